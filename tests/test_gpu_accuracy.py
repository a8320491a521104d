"""Error per coefficient of the full 3D 4PCF against the FP64 oracle, for the
FP32, split-BF16 and split-TF32 combination paths, on a 32^3 field with the benchmark's
spectrum (lognormal sigma_G 1.5, P ~ k^-11/3), lmax 4 and 10 bins (2..15).

Reported (printed; run pytest with -s to see them) per precision: the
largest and the 99th-percentile ratio |zeta_gpu - zeta_oracle| / max|zeta|
over all coefficients, and the cancellation ratio
R = max over coefficients of sum_x sum_M |C delta a a a| / max|zeta|, which
says how much of the summed magnitude cancels.  Asserted: the max ratio is
within 1e-5 (FP32, split TF32) / 1e-4 (split BF16)."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

LMAX = 4
EDGES = list(np.linspace(2.0, 15.0, 11))


def _abs_sums(delta, edges, lmax):
    """sum_x sum_M |C^Lambda_M delta a a a| per (Lambda, b1, b2, b3)."""
    nb = len(edges) - 1
    a = {(l, m): np.abs(O.a_full(delta, edges, l, m).reshape(nb, -1))
         for l in range(lmax + 1) for m in range(-l, l + 1)}
    d = np.abs(delta).reshape(1, -1)
    lams = O.lambda_list(lmax)
    out = np.zeros((len(lams), nb, nb, nb))
    for i, (l1, l2, l3) in enumerate(lams):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if abs(m3) > l3:
                    continue
                c = abs(O.coupling(l1, l2, l3, m1, m2, m3))
                if c == 0.0:
                    continue
                out[i] += c * O.triple_sum(d, a[(l1, m1)], a[(l2, m2)], a[(l3, m3)]).real
    return out


def test_error_per_coefficient():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    f = synth.lognormal_field(1203, (32, 32, 32), 1.5, -11.0 / 3.0, None, np.float32)
    delta, _ = O.preprocess(f.astype(np.float64))
    ref = O.zeta4_full(delta, EDGES, LMAX)
    scale = np.abs(ref).max()
    R = _abs_sums(delta, EDGES, LMAX).max() / scale
    ctx = sbg.Context(0)
    for name, prec, tol in (("fp32", sbg.SBG_PREC_FP32, 1e-5), ("bf16x3", sbg.SBG_PREC_BF16X3, 1e-4),
                            ("tf32x3", sbg.SBG_PREC_TF32X3, 1e-5)):
        _, z4 = ctx.full(torch.from_numpy(f).cuda(), EDGES, lmax4=LMAX, prec=prec)
        ratio = np.abs(z4 - ref).ravel() / scale
        print(f"\n4PCF 32^3 lmax {LMAX} {name}: max {ratio.max():.3e}  p99 {np.percentile(ratio, 99):.3e}  "
              f"R {R:.3e}  ({ratio.size} coefficients)")
        assert ratio.max() <= tol, (name, ratio.max())
    ctx.close()
