"""Parity at the benchmark's full size, in the launch configuration bench.py
times (256^3 float32 lognormal field, 10 linear bins 2..32, lmax 4, 4PCF only,
mean subtracted, field resident on the device; FP32, split BF16 and split TF32):
sampled zeta_Lambda^{b1 b2 b3}
entries are recomputed one by one by the FP64 oracle; the whole tensor is
checked for the symmetries that hold at any size."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

# (Lambda, b1, b2, b3) sampled across l-orders, bin ranges and diagonals
ENTRIES = [((0, 0, 0), 1, 4, 8), ((1, 1, 0), 0, 2, 9), ((2, 1, 1), 3, 3, 6)]


@pytest.fixture(scope="module")
def full256():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    f = synth.workload_field("full256")
    edges = synth.WORKLOADS["full256"]["edges"]
    ctx = sbg.Context(0)
    d = torch.from_numpy(f).cuda()
    out = {}
    for name, prec in (("fp32", sbg.SBG_PREC_FP32), ("bf16x3", sbg.SBG_PREC_BF16X3),
                       ("tf32x3", sbg.SBG_PREC_TF32X3)):
        _, z4 = ctx.full(d, edges, lmax4=4, prec=prec)
        out[name] = z4
    ctx.close()
    delta, _ = O.preprocess(f.astype(np.float64))
    ref = O.zeta4_full_entries(delta, edges, ENTRIES)
    return out, ref


def test_sampled_entries_match_oracle(full256):
    out, ref = full256
    lams = O.lambda_list(4)
    for name, tol in (("fp32", 1e-5), ("bf16x3", 1e-4), ("tf32x3", 1e-5)):
        z4 = out[name]
        scale = np.abs(z4).max()
        for (lam, b1, b2, b3), r in zip(ENTRIES, ref):
            got = z4[lams.index(lam), b1, b2, b3]
            assert abs(got - r) <= tol * scale, (name, lam, b1, b2, b3, got, r, scale)


def test_permutation_symmetry_at_full_size(full256):
    out, _ = full256
    lams = O.lambda_list(4)
    for name, tol in (("fp32", 1e-5), ("bf16x3", 1e-4), ("tf32x3", 1e-5)):
        z4 = out[name]
        scale = np.abs(z4).max()
        for i, (l1, l2, l3) in enumerate(lams):
            j = lams.index((l2, l1, l3))
            assert np.abs(z4[i] - np.transpose(z4[j], (1, 0, 2))).max() <= tol * scale
        # split-BF16 and FP32 agree within the split-BF16 tolerance
    assert np.abs(out["bf16x3"] - out["fp32"]).max() <= 1e-4 * np.abs(out["fp32"]).max()
