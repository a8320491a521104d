"""GPU parity of the tensor-core (tcgen05) 4PCF combination, split BF16 and
split TF32, against the FP64 oracle.  Tolerance per output tensor: 1e-4 of
max |zeta| for split BF16, 1e-5 (the FP32 tolerance) for split TF32, whose
short accumulation ranges keep it at FP32 accuracy; the 3PCF and FFTs are
unchanged FP32."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-4
TOL = {"bf16x3": 1e-4, "tf32x3": 1e-5}


def _prec(name):
    from paper_2210_10206_gb300 import sbg
    return sbg.SBG_PREC_BF16X3 if name == "bf16x3" else sbg.SBG_PREC_TF32X3


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    c = sbg.Context(0)
    yield c
    c.close()


def _err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _cplx(z):
    return z[..., 0] + 1j * z[..., 1]


@pytest.mark.parametrize("n,edges,l4,seed", [
    (16, [0.5, 1.5, 2.5, 3.5, 5.0], 2, 51),
    (32, [1.0, 3.0, 5.5, 8.0, 11.0], 3, 52),
    (8, [0.5, 1.5, 2.0, 3.5], 4, 53),
])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_full_4pcf_tensor(ctx, n, edges, l4, seed, prec):
    f = synth.lognormal_field(seed, (n, n, n), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    _, z4 = ctx.full(f, edges, lmax4=l4, prec=_prec(prec))
    d, _ = O.preprocess(f.astype(np.float64))
    assert _err(z4, O.zeta4_full(d, edges, l4)) < TOL[prec]


def test_full_64_cube_tensor_paths_match_fp32_path(ctx):
    from paper_2210_10206_gb300 import sbg
    f = synth.lognormal_field(1002, (64, 64, 64), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    edges = [2.0, 6.0, 10.0, 14.0, 18.0]
    _, a4 = ctx.full(f, edges, lmax4=3, prec=sbg.SBG_PREC_BF16X3)
    _, t4 = ctx.full(f, edges, lmax4=3, prec=sbg.SBG_PREC_TF32X3)
    _, b4 = ctx.full(f, edges, lmax4=3, prec=sbg.SBG_PREC_FP32)
    d, _ = O.preprocess(f.astype(np.float64))
    r4 = O.zeta4_full(d, edges, 3)
    assert _err(b4, r4) < 1e-5
    assert _err(a4, r4) < TOL_BF16
    assert _err(t4, r4) < TOL["tf32x3"]


@pytest.mark.parametrize("n,edges,mmax,seed", [
    (64, [2.0, 5.0, 8.0, 11.0, 14.0], 4, 61),
    (32, list(np.geomspace(1.0, 12.0, 4)), 3, 62),
])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_projected_4pcf_tensor(ctx, n, edges, mmax, seed, prec):
    f = synth.lognormal_field(seed, (n, n), 1.0, -2.0, dtype=np.float32)
    z3, z4 = ctx.projected(f, edges, mmax, prec=_prec(prec))
    d, _ = O.preprocess(f.astype(np.float64))
    assert _err(_cplx(z3), O.zeta3_projected(d, edges, mmax)) < 1e-5
    assert _err(_cplx(z4), O.zeta4_projected(d, edges, mmax)) < TOL[prec]
