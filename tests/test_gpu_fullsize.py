"""Parity at the benchmark's full size, in the launch configuration bench.py
times (256^3 float32 lognormal field, 10 linear bins 2..32, lmax 4, 4PCF only,
mean subtracted, field resident on the device; FP32, split BF16 and split TF32).

Expected values are the stored oracle goldens of tests/golden/full256_4pcf.json
(written by tests/golden/make_goldens.py, which calls only the FP64 oracle):
one entry for each of the 42 even Lambda (Eq. mu, Sec. 2.3; Algorithm 6) and
each of the 23 odd Lambda (E(Lambda) = -1), bins drawn from {0, 4, 9}, so every
l = 3 and l = 4 leg and every m3 column block of the tile plan is touched.  The
whole tensor is also checked for the symmetries that hold at any size.
Tolerance per coefficient: 1e-5 (FP32, split TF32) / 1e-4 (split BF16) of
max |zeta| of the tensor."""
import json
import os

import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full256_4pcf.json")
TOLS = (("fp32", 1e-5), ("bf16x3", 1e-4), ("tf32x3", 1e-5))


@pytest.fixture(scope="module")
def full256():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    g = json.load(open(GOLDEN))
    f = synth.workload_field("full256")
    x = f.astype(np.float64)
    # the regenerated input is the one the goldens were computed on
    assert abs(x.sum() - g["field"]["sum"]) <= 1e-9 * np.sqrt(x.size * g["field"]["sumsq"])
    assert abs((x * x).sum() - g["field"]["sumsq"]) <= 1e-9 * g["field"]["sumsq"]
    edges = synth.WORKLOADS["full256"]["edges"]
    assert np.allclose(edges, g["edges"], rtol=0, atol=0)
    ctx = sbg.Context(0)
    d = torch.from_numpy(f).cuda()
    out = {}
    for name, prec in (("fp32", sbg.SBG_PREC_FP32), ("bf16x3", sbg.SBG_PREC_BF16X3),
                       ("tf32x3", sbg.SBG_PREC_TF32X3)):
        _, z4 = ctx.full(d, edges, lmax4=4, prec=prec)
        zo = ctx.full_odd(d, edges, 4, prec=prec)
        out[name] = (z4, zo)
    ctx.close()
    return out, g


def test_every_lambda_matches_oracle_goldens(full256):
    out, g = full256
    lams, lams_odd = O.lambda_list(4), O.lambda_list_odd(4)
    for name, tol in TOLS:
        z4, zo = out[name]
        for key, z, ll in (("even", z4, lams), ("odd", zo, lams_odd)):
            scale = np.abs(z).max()
            worst = 0.0
            for e in g[key]:
                got = z[ll.index(tuple(e["lambda"])), e["bins"][0], e["bins"][1], e["bins"][2]]
                err = abs(got - e["value"]) / scale
                worst = max(worst, err)
                assert err <= tol, (name, key, e, got, scale)
            print(f"{name} {key}: {len(g[key])} golden entries, worst |err|/max|zeta| {worst:.2e}")


def test_permutation_symmetry_at_full_size(full256):
    out, _ = full256
    lams = O.lambda_list(4)
    for name, tol in TOLS:
        z4 = out[name][0]
        scale = np.abs(z4).max()
        for i, (l1, l2, l3) in enumerate(lams):
            j = lams.index((l2, l1, l3))
            assert np.abs(z4[i] - np.transpose(z4[j], (1, 0, 2))).max() <= tol * scale
    # split-BF16 and FP32 agree within the split-BF16 tolerance
    assert np.abs(out["bf16x3"][0] - out["fp32"][0]).max() <= 1e-4 * np.abs(out["fp32"][0]).max()
