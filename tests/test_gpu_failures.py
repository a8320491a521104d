"""Failure paths of the measurement calls, driven from the host (no GPU fault):
a tensor-core kernel whose waits run out returns SBG_ERR_TIMEOUT and leaves the
context usable; a context budget too small for a call returns
SBG_ERR_OUT_OF_MEMORY and a later call within the budget succeeds."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

EDGES = [0.5, 1.5, 2.5, 3.5, 5.0]


@pytest.fixture(scope="module")
def sbg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg as s
    build.build()
    return s


def _field():
    return synth.lognormal_field(31, (16, 16, 16), 1.0, -2.0, dtype=np.float64)


@pytest.mark.parametrize("prec_name", ["SBG_PREC_BF16X3", "SBG_PREC_TF32X3"])
def test_wait_timeout_then_context_recovers(sbg, prec_name):
    prec = getattr(sbg, prec_name)
    f = _field()
    ctx = sbg.Context(0)
    # the MMA issuer is withheld, so the producers' and loaders' waits run out
    ctx.set_wait_limit(2_000_000, test_stall=1)  # 2 ms
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, EDGES, lmax4=2, prec=prec)
    assert e.value.status == sbg.SBG_ERR_TIMEOUT
    # twice in a row: the error word and the barriers start afresh each call
    with pytest.raises(sbg.SbgError) as e:
        ctx.full(f, EDGES, lmax4=2, prec=prec)
    assert e.value.status == sbg.SBG_ERR_TIMEOUT
    # back to normal on the same context: oracle-green
    ctx.set_wait_limit(1_000_000_000, test_stall=0)
    _, z4 = ctx.full(f, EDGES, lmax4=2, prec=prec)
    d, _ = O.preprocess(f)
    ref = O.zeta4_full(d, EDGES, 2)
    assert np.abs(z4 - ref).max() / np.abs(ref).max() < 1e-4
    with pytest.raises(sbg.SbgError):
        ctx.set_wait_limit(0, 0)
    ctx.close()


def test_budget_exceeded_is_out_of_memory(sbg):
    f = _field()
    d, _ = O.preprocess(f)
    ref = O.zeta3_full(d, EDGES, 2)
    # 64 KB cannot hold the staged field, delta and delta-hat of a 16^3 call
    small = sbg.Context(0, budget=64 << 10)
    with pytest.raises(sbg.SbgError) as e:
        small.full(f, EDGES, lmax3=2)
    assert e.value.status == sbg.SBG_ERR_OUT_OF_MEMORY
    small.close()
    # a budget that fits the call works, and the same context keeps working
    ok = sbg.Context(0, budget=256 << 20)
    z3, _ = ok.full(f, EDGES, lmax3=2)
    assert np.abs(z3 - ref).max() / np.abs(ref).max() < 1e-5
    z3b, _ = ok.full(f, EDGES, lmax3=2)
    assert np.array_equal(z3, z3b) or np.abs(z3b - z3).max() < 1e-12 * np.abs(z3).max()
    ok.close()


def test_autotuner_records_its_choices(sbg):
    # the first call of a geometry measures the launch choices and keeps them
    f = _field()
    ctx = sbg.Context(0)
    ctx.full(f, EDGES, lmax4=2, prec=sbg.SBG_PREC_BF16X3)
    rep = sbg.sbg_autotune_report(ctx.h)
    assert any(k.startswith("tc4/") for k in rep), rep
    assert all(v in (0, 1, 2) for k, v in rep.items() if k.startswith("fft/")), rep
    g = synth.lognormal_field(3, (128, 128, 128), 1.0, -2.0, dtype=np.float32)
    ctx.full(g, [2.0, 5.0, 9.0], lmax3=1)
    rep2 = sbg.sbg_autotune_report(ctx.h)
    assert any(k.startswith("fft/128/") for k in rep2), rep2   # strided passes of N >= 128
    assert all(rep2[k] == v for k, v in rep.items())          # earlier choices are kept
    ctx.close()
