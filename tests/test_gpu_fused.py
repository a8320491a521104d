"""GPU parity of the fused 3D path taken when the kernel spectra of every
(l, m) group do not fit (the 512^3 3PCF; here forced by a small context
budget): kernel generation fused with the forward transform along x, the
support-only y transform, and the z transform fused with the product with
delta-hat and the inverse z transform (Algorithms 1, 3 with Eq. almconv).
Against the FP64 oracle and against the cached-spectra path of an unbudgeted
context; the launch counts show which path ran (5 kernels per group instead
of 3 for the convolutions)."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg as s
    build.build()
    return s


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# budgets too small for the cached spectra of every group, large enough for one call
@pytest.mark.parametrize("n,edges,lmax3,budget_kb", [
    (32, list(np.linspace(1.0, 14.0, 9)), 5, 8192),    # 8 bins, l <= 5
    (16, [0.0, 7.5], 3, 300),                           # one bin reaching N/2, edges[0] = 0
    (64, list(np.linspace(2.0, 31.5, 6)), 2, 40960),   # support up to N/2: 63 planes of 64
])
def test_fused_3pcf_matches_oracle_and_cached_path(sbg, n, edges, lmax3, budget_kb):
    f = synth.lognormal_field(600 + n, (n, n, n), 1.3, -3.0, None, np.float32)
    tight = sbg.Context(0, budget=budget_kb << 10)
    z3, _ = tight.full(f, edges, lmax3=lmax3)
    z3b, _ = tight.full(f, edges, lmax3=lmax3)
    launches_fused = int(tight.timings()[7])
    tight.close()
    roomy = sbg.Context(0)
    roomy.full(f, edges, lmax3=lmax3)
    c3, _ = roomy.full(f, edges, lmax3=lmax3)
    launches_cached = int(roomy.timings()[7])
    roomy.close()
    ngroups = (lmax3 + 1) * (lmax3 + 2) // 2
    assert launches_fused - launches_cached == 2 * ngroups, (launches_fused, launches_cached)
    d, _ = O.preprocess(f.astype(np.float64))
    r3 = O.zeta3_full(d, edges, lmax3)
    assert _rel(z3, r3) <= 1e-5
    assert np.array_equal(z3, z3b) or _rel(z3b, z3) <= 1e-12
    assert _rel(c3, z3) <= 1e-5


@pytest.mark.parametrize("pname", ["fp32", "bf16x3"])
def test_fused_3pcf_and_4pcf_with_packed_m0(sbg, pname):
    # stored groups (the 4PCF's) go to the blocked store, m = 0 packed two per transform
    n, edges = 32, [0.5, 2.0, 4.0, 6.5, 9.0]
    f = synth.lognormal_field(77, (n, n, n), 1.2, -2.5, None, np.float32)
    prec = sbg.SBG_PREC_FP32 if pname == "fp32" else sbg.SBG_PREC_BF16X3
    ctx = sbg.Context(0, budget=48 << 20)
    z3, z4 = ctx.full(f, edges, lmax3=4, lmax4=2, prec=prec)
    ctx.close()
    d, _ = O.preprocess(f.astype(np.float64))
    tol = 1e-5 if pname == "fp32" else 1e-4
    assert _rel(z3, O.zeta3_full(d, edges, 4)) <= tol
    assert _rel(z4, O.zeta4_full(d, edges, 2)) <= tol
