"""Host-side checks of the binding's result arrays (no GPU): a caller's array
passed for reuse must be a writable C-contiguous float64 array of exactly the
result's shape, because the library writes every element through its pointer;
anything else is refused before the library is called."""
import numpy as np
import pytest

from paper_2210_10206_gb300 import sbg


def test_out_new_array_is_zeroed():
    a = sbg._out(None, (2, 3, 3), "zeta3")
    assert a.shape == (2, 3, 3) and a.dtype == np.float64 and not a.any()


def test_out_reuses_a_matching_array():
    a = np.ones((4, 2, 2, 2))
    assert sbg._out(a, (4, 2, 2, 2), "zeta4") is a


@pytest.mark.parametrize("bad", [
    np.zeros((2, 3, 4)),                       # wrong shape
    np.zeros((2, 3, 3), dtype=np.float32),     # wrong dtype
    np.zeros((3, 3, 2)).transpose(2, 1, 0),    # not C-contiguous
    [[0.0]],                                   # not an ndarray
])
def test_out_refuses_mismatches(bad):
    with pytest.raises(ValueError):
        sbg._out(bad, (2, 3, 3), "zeta3")


def test_out_refuses_read_only():
    a = np.zeros((2, 3, 3))
    a.flags.writeable = False
    with pytest.raises(ValueError):
        sbg._out(a, (2, 3, 3), "zeta3")


def test_slices_refuses_wrong_out_before_the_library():
    cube = np.zeros((4, 8, 8), dtype=np.float32)
    with pytest.raises(ValueError):
        sbg.sbg_projected_slices(None, cube, [1.0, 2.0, 3.0], 1, sbg.SBG_PREC_FP32,
                                 sbg.SBG_3PCF, zeta3=np.zeros((4, 2, 2, 2)))


def test_batch_refuses_wrong_pair_count():
    with pytest.raises(ValueError):
        sbg.sbg_projected_batch(None, [np.zeros((8, 8))], [[1.0, 2.0]], 1, 1, sbg.SBG_PREC_FP32,
                                sbg.SBG_3PCF, outs=[])
