"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
function that include/sarabande_gb300.h declares, and its host-only calls agree
with the oracle's definitions."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import sarabande_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sbg():
    from paper_2210_10206_gb300 import build, sbg as s
    build.build()
    s.lib()
    return s


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sbg_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(sbg):
    names = _declared()
    assert {"sbg_create", "sbg_full", "sbg_projected", "sbg_projected_batch"} <= names
    lib = ctypes.CDLL(sbg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_lambda_list_matches_oracle(sbg):
    for lmax in range(0, 8):
        assert sbg.sbg_lambda_count(lmax) == len(O.lambda_list(lmax))
        assert [tuple(r) for r in sbg.sbg_lambda_list(lmax)] == O.lambda_list(lmax)
    assert sbg.sbg_lambda_count(3) == 23 and sbg.sbg_lambda_count(4) == 42


def test_odd_lambda_list_matches_oracle(sbg):
    for lmax in range(0, 8):
        assert sbg.sbg_lambda_odd_count(lmax) == len(O.lambda_list_odd(lmax))
        assert [tuple(r) for r in sbg.sbg_lambda_odd_list(lmax)] == O.lambda_list_odd(lmax)
    assert sbg.sbg_lambda_odd_count(1) == 1 and sbg.sbg_lambda_odd_count(4) == 23
    L = sbg.lib()
    assert L.sbg_full_odd(None, None, 0, None, None, 1, 2, 0, 0, None) == -1
    assert L.sbg_projected_slices(None, None, 0, None, None, 1, 2, 0, 3, None, None) == -1


def test_unique_bins_follow_the_papers_1d_index(sbg):
    # nested loops b1 < b2 (< b3) of Algorithm 6's bin loops: lexicographic
    # combinations without repeated bins
    import itertools
    for nb in (1, 2, 3, 10, 20):
        for order, k in ((3, 2), (4, 3)):
            got = [tuple(r) for r in sbg.sbg_unique_bins(nb, order)]
            assert got == list(itertools.combinations(range(nb), k))
    assert len(sbg.sbg_unique_bins(10, 3)) == 45 and len(sbg.sbg_unique_bins(10, 4)) == 120
    with pytest.raises(sbg.SbgError):
        sbg.sbg_unique_bins(10, 5)


def test_unique_gather_picks_the_off_diagonal_entries(sbg):
    import itertools
    rng = np.random.default_rng(3)
    z4 = rng.normal(size=(7, 6, 6, 6))
    u = sbg.sbg_unique_gather(z4, 4)
    idx = list(itertools.combinations(range(6), 3))
    assert u.shape == (7, len(idx))
    assert np.array_equal(u, np.stack([[z4[i][t] for t in idx] for i in range(7)]))
    z3c = rng.normal(size=(4, 5, 5, 2))  # complex (re, im) projected 3PCF layout
    u3 = sbg.sbg_unique_gather(z3c, 3, ncomp=2)
    idx2 = list(itertools.combinations(range(5), 2))
    assert u3.shape == (4, len(idx2), 2)
    assert np.array_equal(u3, np.stack([[z3c[i][t] for t in idx2] for i in range(4)]))


def test_zero_overlap_zeroes_exactly_the_coincident_bins(sbg):
    # the diagonals of the application figure (Sec. 4): b1 = b2 (3PCF), any two
    # bins equal (4PCF); everything else is left bit for bit
    rng = np.random.default_rng(5)
    z4 = rng.normal(size=(3, 6, 6, 6))
    ref = z4.copy()
    assert sbg.sbg_zero_overlap(z4, 4) is z4
    b1, b2, b3 = np.meshgrid(np.arange(6), np.arange(6), np.arange(6), indexing="ij")
    overlap = (b1 == b2) | (b2 == b3) | (b1 == b3)
    assert np.all(z4[:, overlap] == 0.0)
    assert np.array_equal(z4[:, ~overlap], ref[:, ~overlap])
    assert int((~overlap).sum()) == 6 * 5 * 4  # ordered triples of distinct bins
    z3c = rng.normal(size=(4, 5, 5, 2))  # complex projected 3PCF layout
    ref3 = z3c.copy()
    sbg.sbg_zero_overlap(z3c, 3, ncomp=2)
    eye = np.eye(5, dtype=bool)
    assert np.all(z3c[:, eye] == 0.0) and np.array_equal(z3c[:, ~eye], ref3[:, ~eye])
    # the unique gather never reads the zeroed entries
    assert np.array_equal(sbg.sbg_unique_gather(z3c, 3, ncomp=2), sbg.sbg_unique_gather(ref3, 3, ncomp=2))
    L = sbg.lib()
    assert L.sbg_zero_overlap(None, 1, 5, 3, 1) == -1
    bad = np.zeros((2, 2))
    assert L.sbg_zero_overlap(bad.ctypes.data, 1, 2, 5, 1) == -1
    assert L.sbg_zero_overlap(bad.ctypes.data, 1, 21, 3, 1) == -1
    with pytest.raises(ValueError):
        sbg.sbg_zero_overlap(np.zeros((3, 4, 5)), 3)


def test_status_strings_and_argument_errors(sbg):
    assert sbg.sbg_status_string(-3) == "SBG_ERR_BIN_RANGE"
    assert sbg.sbg_status_string(0) == "SBG_OK"
    L = sbg.lib()
    n = ctypes.c_int()
    assert L.sbg_lambda_count(-1, ctypes.byref(n)) == -1
    assert L.sbg_lambda_count(3, None) == -1
    # NULL context is rejected without touching a device
    assert L.sbg_full(None, None, 0, None, None, 1, 0, 0, 0, 1, None, None) == -1
    assert L.sbg_projected(None, None, 0, None, None, 1, 0, 0, 1, None, None) == -1
    L.sbg_destroy(None)


def test_create_without_gpu_fails_cleanly(sbg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    s = sbg.lib().sbg_create(0, 0, ctypes.byref(h))
    assert s in (-1, -6) and not h.value
