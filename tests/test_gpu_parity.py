"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerance (per output tensor): max |zeta_gpu - zeta_oracle|
<= TOL * max |zeta_oracle|, with TOL = 1e-5 for the FP32 path and 1e-4 for the
split-BF16 path."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16 = 1e-4


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


# ------------------------------------------------------------ projected ----

@pytest.mark.parametrize("n,edges,mmax,seed,dtype", [
    (64, [2.0, 5.0, 8.0, 11.0, 14.0], 4, 1001, np.float64),      # 64^2 float64 workload
    (32, list(np.geomspace(1.0, 12.0, 4)), 3, 21, np.float32),     # log bins, ragged counts
    (16, [0.0, 1.0, 2.5, 4.0, 7.5], 2, 22, np.float64),            # edges[0] = 0 excludes the origin
    (8, [0.5, 2.0, 3.9], 2, 23, np.float32),                        # smallest grid, edge just under N/2
])
def test_projected_3pcf_4pcf(ctx, n, edges, mmax, seed, dtype):
    f = synth.lognormal_field(seed, (n, n), 1.0, -2.0, dtype=dtype)
    z3, z4 = ctx.projected(f, edges, mmax)
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_projected(d, edges, mmax)
    r4 = O.zeta4_projected(d, edges, mmax)
    assert _err(_cplx(z3), r3) < TOL_FP32
    assert _err(_cplx(z4), r4) < TOL_FP32
    # entries with |m1 + m2| > mmax are zero
    w = 2 * mmax + 1
    for i in range(w):
        for j in range(w):
            if abs(i + j - 2 * mmax) > mmax:
                assert np.all(z4[i, j] == 0)


def test_projected_single_bin_and_no_mean_subtraction(ctx):
    from paper_2210_10206_gb300 import sbg
    f = synth.particle_field(5, (64, 64), 30)
    edges = [1.0, 9.5]
    z3, z4 = ctx.projected(f, edges, 3, flags=0)
    r3 = O.zeta3_projected(f, edges, 3)
    r4 = O.zeta4_projected(f, edges, 3)
    assert _err(_cplx(z3), r3) < TOL_FP32
    assert _err(_cplx(z4), r4) < TOL_FP32


def test_projected_normalized(ctx):
    from paper_2210_10206_gb300 import sbg
    f = synth.lognormal_field(31, (32, 32), 1.0, -2.0, dtype=np.float64)
    edges = [1.0, 3.0, 6.0, 9.0]
    z3, z4 = ctx.projected(f, edges, 2, flags=sbg.SBG_SUBTRACT_MEAN | sbg.SBG_NORMALIZED)
    d, ngal = O.preprocess(f)
    r3 = O.zeta3_projected(d, edges, 2)
    r4 = O.zeta4_projected(d, edges, 2)
    nb = 3
    for b1 in range(nb):
        for b2 in range(nb):
            r3[:, b1, b2] /= O.normalization(f.shape, edges, ngal, 3, [b1, b2])
            for b3 in range(nb):
                r4[:, :, b1, b2, b3] /= O.normalization(f.shape, edges, ngal, 4, [b1, b2, b3])
    assert _err(_cplx(z3), r3) < TOL_FP32
    assert _err(_cplx(z4), r4) < TOL_FP32


# ----------------------------------------------------------------- full ----

@pytest.mark.parametrize("n,edges,l3,l4,seed", [
    (16, [0.5, 1.5, 2.5, 3.5, 5.0], 4, 2, 41),
    (32, [1.0, 3.0, 5.5, 8.0, 11.0], 3, 3, 42),
    (8, [0.5, 1.5, 2.0, 3.5], 5, 4, 43),
])
def test_full_3pcf_4pcf(ctx, n, edges, l3, l4, seed):
    f = synth.lognormal_field(seed, (n, n, n), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    z3, z4 = ctx.full(f, edges, lmax3=l3, lmax4=l4)
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_full(d, edges, l3)
    r4 = O.zeta4_full(d, edges, l4)
    assert _err(z3, r3) < TOL_FP32
    assert _err(z4, r4) < TOL_FP32


def test_full_64_cube_spans_many_tiles(ctx):
    # 64^3: several CTAs per axis pass, several 4PCF tiles, ragged last tiles
    f = synth.lognormal_field(1002, (64, 64, 64), 1.2, -3.0, cutoff=np.pi / 2, dtype=np.float32)
    edges = [2.0, 6.0, 10.0, 14.0, 18.0]
    z3, z4 = ctx.full(f, edges, lmax3=5, lmax4=3)
    d, _ = O.preprocess(f.astype(np.float64))
    assert _err(z3, O.zeta3_full(d, edges, 5)) < TOL_FP32
    assert _err(z4, O.zeta4_full(d, edges, 3)) < TOL_FP32


def test_full_3pcf_only_and_4pcf_only_agree_with_combined(ctx):
    f = synth.lognormal_field(44, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
    edges = [0.5, 2.0, 3.5, 6.0]
    a3, a4 = ctx.full(f, edges, lmax3=3, lmax4=2)
    b3, _ = ctx.full(f, edges, lmax3=3)
    _, c4 = ctx.full(f, edges, lmax4=2)
    # same sums through two coefficient layouts; FP64 atomics across CTAs add
    # in no fixed order, so agreement is to rounding, not bitwise.  With a 4PCF
    # the m = 0 coefficients come from transforms packed two real results per
    # complex transform (a^b_l0 is real, Eq. almconv with a real kernel), without
    # one from one transform each: the 3PCFs then agree to FP32 rounding
    assert _err(b3, a3) < 1e-6
    assert _err(c4, a4) < 1e-12


def test_full_normalized(ctx):
    from paper_2210_10206_gb300 import sbg
    f = synth.lognormal_field(45, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
    edges = [0.5, 2.0, 3.5, 6.0]
    z3, z4 = ctx.full(f, edges, lmax3=2, lmax4=2, flags=sbg.SBG_SUBTRACT_MEAN | sbg.SBG_NORMALIZED)
    d, ngal = O.preprocess(f)
    r3 = O.zeta3_full(d, edges, 2)
    r4 = O.zeta4_full(d, edges, 2)
    for b1 in range(3):
        for b2 in range(3):
            r3[:, b1, b2] /= O.normalization(f.shape, edges, ngal, 3, [b1, b2])
            for b3 in range(3):
                r4[:, b1, b2, b3] /= O.normalization(f.shape, edges, ngal, 4, [b1, b2, b3])
    assert _err(z3, r3) < TOL_FP32
    assert _err(z4, r4) < TOL_FP32


def test_device_field_matches_host_field(ctx):
    import torch
    f = synth.lognormal_field(46, (32, 32, 32), 1.0, -2.0, dtype=np.float32)
    edges = [1.0, 3.0, 6.0, 9.0]
    h3, h4 = ctx.full(f, edges, lmax3=2, lmax4=2)
    d3, d4 = ctx.full(torch.from_numpy(f).cuda(), edges, lmax3=2, lmax4=2)
    # FP64 atomics across CTAs add in no fixed order: agreement to rounding
    assert _err(d3, h3) < 1e-12 and _err(d4, h4) < 1e-12


def test_shift_and_rotation_invariance_on_gpu(ctx):
    f = synth.lognormal_field(47, (32, 32, 32), 1.0, -2.0, dtype=np.float64)
    edges = [1.0, 3.0, 6.0, 9.0]
    z3, z4 = ctx.full(f, edges, lmax3=3, lmax4=2)
    for t in (np.roll(f, (5, 9, 13), axis=(0, 1, 2)), np.rot90(f, 1, axes=(0, 2))):
        t3, t4 = ctx.full(np.ascontiguousarray(t), edges, lmax3=3, lmax4=2)
        assert _err(t3, z3) < TOL_FP32
        assert _err(t4, z4) < TOL_FP32


def test_errors_are_reported(ctx):
    from paper_2210_10206_gb300 import sbg
    f = np.zeros((16, 16, 16), np.float32)
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, [1.0, 8.0], lmax3=1)            # edges[nbins] >= N/2
    assert e.value.status == -3
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, [2.0, 1.0], lmax3=1)            # not increasing
    assert e.value.status == -3
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(np.zeros((16, 16, 8), np.float32), [1.0, 2.0], lmax3=1)
    assert e.value.status == -2
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(np.zeros((24, 24, 24), np.float32), [1.0, 2.0], lmax3=1)
    assert e.value.status == -2
    with pytest.raises(sbg.SbgError) as e:               # empty bin under normalisation
        ctx.full(f, [1.0, 1.1, 3.0], lmax3=1, flags=sbg.SBG_NORMALIZED)
    assert e.value.status == -4
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, [1.0, 2.0], lmax4=9)
    assert e.value.status == -1
