"""GPU parity of sbg_projected_slices: the projected 3PCF and 4PCF of every 2D
slice of a 3D cube (Sec. 4 measures the projected statistics of one slice of a
simulation cube).  Each slice's output matches sbg_projected of that slice and
the oracle's (1e-5 FP32, 1e-4 split BF16, relative to max |zeta| per tensor)."""
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


def _c(z):
    return z[..., 0] + 1j * z[..., 1]


@pytest.mark.parametrize("pname", ["fp32", "bf16x3"])
def test_slices_match_single_fields_and_oracle(sbgm, pname):
    import torch
    sbg = sbgm
    prec = sbg.SBG_PREC_FP32 if pname == "fp32" else sbg.SBG_PREC_BF16X3
    tol = 1e-5 if pname == "fp32" else 1e-4
    cube = synth.lognormal_field(71, (32, 32, 32), 1.2, -2.5, dtype=np.float32)[:12].copy()
    edges = [1.0, 3.0, 5.0, 8.0]
    mmax = 3
    ctx = sbg.Context(0)
    z3, z4 = ctx.projected_slices(torch.from_numpy(cube).cuda(), edges, mmax, prec=prec)
    assert z3.shape == (12, mmax + 1, 3, 3, 2) and z4.shape == (12, 7, 7, 3, 3, 3, 2)
    # the slices run as one slab, whose 4PCF contraction splits each field's
    # sum over x differently from a single-field call: the two agree to the
    # rounding of the combination's arithmetic, and each meets the oracle below
    for i in (0, 5, 11):
        p3, p4 = ctx.projected(cube[i], edges, mmax, prec=prec)
        assert np.abs(z3[i] - p3).max() <= tol * np.abs(p3).max()
        assert np.abs(z4[i] - p4).max() <= tol * np.abs(p4).max()
    ctx.close()
    for i in (0, 11):
        d, _ = O.preprocess(cube[i].astype(np.float64))
        r3 = O.zeta3_projected(d, edges, mmax)
        r4 = O.zeta4_projected(d, edges, mmax)
        assert np.abs(_c(z3[i]) - r3).max() <= tol * np.abs(r3).max()
        assert np.abs(_c(z4[i]) - r4).max() <= tol * np.abs(r4).max()
