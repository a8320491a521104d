"""GPU parity of the tensor-core 3PCF combination (the delta-weighted Gram of
Algorithms 5 and 7 on tcgen05, split BF16 and split TF32) against the FP64
oracle, through both coefficient layouts it reads: the [bin][x] buffer of a
group that only the 3PCF needs, and the blocked store of the groups the 4PCF
also needs (3PCF and 4PCF in one call).  Edge cases: a grid of one K-block
(8^2 = 64 points), one bin, 20 bins, normalisation.  Tolerances per output
tensor: 1e-4 (split BF16) / 1e-5 (split TF32) of max |zeta|, as for the 4PCF."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-4, "tf32x3": 1e-5}


@pytest.fixture(scope="module")
def sbg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg as s
    build.build()
    return s


def _prec(sbg, name):
    return {"bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3}[name]


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,edges,lmax3,lmax4", [
    (16, [0.5, 1.5, 2.5, 3.5, 5.0, 7.0], 5, None),          # group buffers only
    (16, [0.5, 1.5, 2.5, 3.5, 5.0, 7.0], 4, 2),             # l <= 2 from the blocked store
    (32, list(np.linspace(2.0, 14.0, 11)), 3, None),        # 10 bins
    (32, list(np.linspace(1.0, 15.0, 21)), 2, 1),           # 20 bins, both layouts
    (8, [0.0, 3.5], 2, None),                               # one bin, 8 K-blocks
])
def test_full_3pcf_tensor_core(sbg, name, n, edges, lmax3, lmax4):
    f = synth.lognormal_field(90 + n + len(edges), (n, n, n), 1.5, -11.0 / 3.0, None, np.float32)
    ctx = sbg.Context(0)
    z3, _ = ctx.full(f, edges, lmax3=lmax3, lmax4=lmax4, prec=_prec(sbg, name))
    ref3 = ctx.full(f, edges, lmax3=lmax3)[0]  # the FP32 path of the same call
    ctx.close()
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_full(d, edges, lmax3)
    err = _rel(z3, r3)
    print(f"{name} full 3PCF {n}^3 {len(edges) - 1} bins lmax {lmax3}: {err:.2e} (FP32 {_rel(ref3, r3):.2e})")
    assert err <= TOL[name]


@pytest.mark.parametrize("name", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,edges,mmax,four", [
    (8, [0.5, 1.5, 3.0], 2, False),                         # 64 points: one bf16 K-block
    (64, list(synth.edges_log(2.0, 8.0, 10)), 10, False),
    (64, list(synth.edges_log(2.0, 8.0, 10)), 6, True),     # blocked store
    (128, [2.0, 60.0], 3, False),                           # one bin
])
def test_projected_3pcf_tensor_core(sbg, name, n, edges, mmax, four):
    f = synth.lognormal_field(300 + n + mmax, (n, n), 1.2, -8.0 / 3.0, None, np.float32)
    ctx = sbg.Context(0)
    z3, _ = ctx.projected(f, edges, mmax, npcf=(3, 4) if four else (3,), prec=_prec(sbg, name))
    ctx.close()
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_projected(d, edges, mmax)
    err = _rel(z3[..., 0] + 1j * z3[..., 1], r3)
    print(f"{name} projected 3PCF {n}^2 mmax {mmax}: {err:.2e}")
    assert err <= TOL[name]


def test_normalized_3pcf_tensor_core(sbg):
    f = synth.lognormal_field(77, (16, 16, 16), 1.0, -2.0, None, np.float64)
    edges = [0.5, 1.5, 2.5, 4.0]
    ctx = sbg.Context(0)
    z3, _ = ctx.full(f, edges, lmax3=3, prec=sbg.SBG_PREC_TF32X3, flags=sbg.SBG_SUBTRACT_MEAN | sbg.SBG_NORMALIZED)
    ctx.close()
    d, ngal = O.preprocess(f)
    r3 = O.zeta3_full(d, edges, 3)
    for b1 in range(3):
        for b2 in range(3):
            r3[:, b1, b2] /= O.normalization(d.shape, edges, ngal, 3, [b1, b2])
    assert _rel(z3, r3) <= 1e-5


def test_gram_timeout_then_recovers(sbg):
    f = synth.lognormal_field(5, (16, 16, 16), 1.0, -2.0, None, np.float32)
    edges = [0.5, 1.5, 2.5, 4.0]
    ctx = sbg.Context(0)
    ctx.set_wait_limit(2_000_000, test_stall=1)
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, edges, lmax3=2, prec=sbg.SBG_PREC_BF16X3)   # 3PCF only: only the Gram kernel runs
    assert e.value.status == sbg.SBG_ERR_TIMEOUT
    ctx.set_wait_limit(1_000_000_000, test_stall=0)
    z3, _ = ctx.full(f, edges, lmax3=2, prec=sbg.SBG_PREC_BF16X3)
    d, _ = O.preprocess(f.astype(np.float64))
    assert _rel(z3, O.zeta3_full(d, edges, 2)) <= 1e-4
    ctx.close()
