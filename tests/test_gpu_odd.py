"""GPU parity of the odd-parity full 4PCF (sbg_full_odd: Eq. mu of Sec. 2.3
with E(Lambda) = -1, reported as the imaginary part of each coefficient)
against the FP64 oracle, in every precision, and its sign flip under a mirror
image of the field.  Tolerances per output tensor, relative to max |zeta_odd|:
1e-5 for FP32 and split TF32, 1e-4 for split BF16."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbgm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    return sbg


def _tol(sbg, prec):
    return 1e-4 if prec == sbg.SBG_PREC_BF16X3 else 1e-5


def _err(z, ref):
    return float(np.abs(z - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("pname", ["fp32", "bf16x3", "tf32x3"])
def test_odd_parity_matches_oracle_16(sbgm, pname):
    sbg = sbgm
    prec = {"fp32": sbg.SBG_PREC_FP32, "bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3}[pname]
    f = synth.lognormal_field(61, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
    edges = [0.5, 2.0, 3.5, 6.0]
    ctx = sbg.Context(0)
    z = ctx.full_odd(f, edges, 3, prec=prec)
    ctx.close()
    d, _ = O.preprocess(f)
    ref = O.zeta4_full_odd(d, edges, 3)
    assert z.shape == ref.shape == (len(O.lambda_list_odd(3)), 3, 3, 3)
    assert _err(z, ref) <= _tol(sbg, prec), (pname, _err(z, ref))


@pytest.mark.parametrize("pname", ["fp32", "bf16x3", "tf32x3"])
def test_odd_parity_benchmark_spectrum_32(sbgm, pname):
    # the benchmark's spectrum and binning at 32^3 (lmax 4, 10 bins 2..15, device field)
    import torch
    sbg = sbgm
    prec = {"fp32": sbg.SBG_PREC_FP32, "bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3}[pname]
    f = synth.lognormal_field(1203, (32, 32, 32), 1.5, -11.0 / 3.0, None, np.float32)
    edges = list(np.linspace(2.0, 15.0, 11))
    ctx = sbg.Context(0)
    z = ctx.full_odd(torch.from_numpy(f).cuda(), edges, 4, prec=prec)
    ctx.close()
    d, _ = O.preprocess(f.astype(np.float64))
    ref = O.zeta4_full_odd(d, edges, 4)
    e = _err(z, ref)
    print(f"\nodd 4PCF 32^3 lmax 4 {pname}: max {e:.3e}")
    assert e <= _tol(sbg, prec), (pname, e)


def test_odd_parity_flips_under_a_mirror_on_gpu(sbgm):
    sbg = sbgm
    f = synth.lognormal_field(62, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
    edges = [0.5, 2.0, 3.5, 6.0]
    ctx = sbg.Context(0)
    z = ctx.full_odd(f, edges, 2)
    zm = ctx.full_odd(np.ascontiguousarray(f[:, ::-1, :]), edges, 2)
    ze = ctx.full(f, edges, lmax4=2)[1]
    sym = f + np.roll(f[:, :, ::-1], 1, axis=2)  # mirror-symmetric in x on the periodic grid
    zs = ctx.full_odd(np.ascontiguousarray(sym), edges, 2)
    ctx.close()
    assert np.abs(z).max() > 0
    assert _err(zm, -z) <= 1e-5
    assert np.abs(zs).max() <= 1e-5 * np.abs(ze).max()


def test_alternating_even_and_odd_calls_reuse_their_plans(sbgm):
    # both table sets stay cached: alternating calls give the same results
    sbg = sbgm
    f = synth.lognormal_field(63, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
    edges = [0.5, 2.0, 3.5, 6.0]
    ctx = sbg.Context(0)
    first_even = ctx.full(f, edges, lmax4=3, prec=sbg.SBG_PREC_BF16X3)[1]
    first_odd = ctx.full_odd(f, edges, 3, prec=sbg.SBG_PREC_BF16X3)
    for _ in range(2):
        e = ctx.full(f, edges, lmax4=3, prec=sbg.SBG_PREC_BF16X3)[1]
        o = ctx.full_odd(f, edges, 3, prec=sbg.SBG_PREC_BF16X3)
        assert np.abs(e - first_even).max() <= 1e-12 * np.abs(first_even).max()
        assert np.abs(o - first_odd).max() <= 1e-12 * np.abs(first_odd).max()
    ctx.close()
