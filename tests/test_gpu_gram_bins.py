"""GPU parity of the FP32 3PCF Gram (Algorithm 5 / Eq. zeta3 of Sec. 2.2 and
Algorithm 7 / Eq. proj_3pcf_coeff of Sec. 2.4) across the bin counts that
change its layout: bins form blocks of 4 and each block pair (I <= J) is one
warp, so 1 bin is one block in a CTA of four warps of which one has work, 5
bins are two blocks with a ragged last one, 13 bins four blocks, 20 bins (the
maximum) five blocks and fifteen warps.  Each count is checked reading the
group buffer (3PCF only) and the blocked coefficient store (groups the 4PCF
also uses), against the FP64 oracle: max |zeta_gpu - zeta_oracle| <= 1e-5 max
|zeta_oracle|."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


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


@pytest.mark.parametrize("nb", [1, 5, 13, 20])
def test_full_gram_bins(ctx, nb):
    f = synth.lognormal_field(300 + nb, (32, 32, 32), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    edges = list(np.linspace(1.0, 15.0, nb + 1))
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_full(d, edges, 2)
    # group buffer: 3PCF only
    z3, _ = ctx.full(f, edges, lmax3=2)
    assert _err(z3, r3) < TOL_FP32
    # blocked store: the l <= 1 groups are also 4PCF singles
    z3b, _ = ctx.full(f, edges, lmax3=2, lmax4=1)
    assert _err(z3b, r3) < TOL_FP32


@pytest.mark.parametrize("nb", [1, 5, 13, 20])
def test_projected_gram_bins(ctx, nb):
    f = synth.lognormal_field(400 + nb, (64, 64), 1.0, -2.0, dtype=np.float32)
    edges = list(np.linspace(1.0, 31.0, nb + 1))
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_projected(d, edges, 3)
    z3, _ = ctx.projected(f, edges, 3, npcf=(3,))
    assert _err(_cplx(z3), r3) < TOL_FP32
    z3b, _ = ctx.projected(f, edges, 3, npcf=(3, 4))
    assert _err(_cplx(z3b), r3) < TOL_FP32


@pytest.mark.parametrize("n,nb", [(128, 20), (256, 10)])
def test_gram_large_grids(ctx, n, nb):
    # 3PCF without 4PCF at N = 128 / 256 (groups read from the group buffer at
    # sizes larger than L2); single entries against the FP64 oracle
    f = synth.lognormal_field(500 + n, (n, n, n), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    edges = list(np.linspace(2.0, n / 4, nb + 1))
    z3, _ = ctx.full(f, edges, lmax3=2)
    d, _ = O.preprocess(f.astype(np.float64))
    entries = [(0, 0, nb - 1), (1, 2, 3), (2, nb - 1, nb - 1), (2, 1, nb // 2)]
    want = O.zeta3_full_entries(d, edges, entries)
    scale = np.abs(z3).max()
    for (l, b1, b2), w in zip(entries, want):
        assert abs(z3[l, b1, b2] - w) <= TOL_FP32 * scale, (n, l, b1, b2, z3[l, b1, b2], w)
