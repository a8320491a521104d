"""The allocation-free projected 3PCF entry point, for callers that cannot
allocate device memory during a measurement (code running inside a pre-sized
memory pool, or an allocator that must not be re-entered).  Through the C ABI
it is compared with the regular projected entry point and with the FP64
oracle, on three calls in a row: the third is smaller than the second, so
leftovers of a larger call in the shared static array would show."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # same relative tolerance as the FP32 parity tests


def _err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_noalloc_matches_projected_and_oracle_on_three_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    ctx = sbg.Context(0)
    cases = [(64, [2.0, 5.0, 8.0, 11.0, 14.0], 4, 71, torch.float64),
             (128, list(np.geomspace(2.0, 16.0, 6)), 6, 72, torch.float32),
             (64, [1.5, 4.0, 9.0], 2, 73, torch.float32)]
    stream = torch.cuda.current_stream().cuda_stream
    for n, edges, mmax, seed, dt in cases:
        f = synth.lognormal_field(seed, (n, n), 1.0, -2.0, dtype=np.float64)
        d = torch.from_numpy(f).to(device="cuda", dtype=dt)
        ref, _ = ctx.projected(d, edges, mmax, npcf=(3,))
        z = torch.full((mmax + 1, len(edges) - 1, len(edges) - 1, 2), np.nan, dtype=torch.float64, device="cuda")
        sbg.sbg_projected3_noalloc(d, edges, mmax, sbg.SBG_SUBTRACT_MEAN, z, stream)
        torch.cuda.synchronize()
        got = z.cpu().numpy()
        assert _err(got, ref) < TOL
        delta, _ = O.preprocess(d.double().cpu().numpy())
        orc = O.zeta3_projected(delta, edges, mmax)
        assert _err(got[..., 0] + 1j * got[..., 1], orc) < TOL
    # out-of-range sizes are rejected without touching the device
    big = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    z = torch.zeros((2, 1, 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(sbg.SbgError) as e:
        sbg.sbg_projected3_noalloc(big, [1.0, 2.0], 1, 0, z, stream)
    assert e.value.status == -2
    ctx.close()
