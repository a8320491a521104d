"""Host-only checks of the 4PCF tile plan (no GPU): sbg_plan4_info builds the
pair x single tables of the contraction for a geometry and fails with
SBG_ERR_INTERNAL if any output term of Algorithm 6 (full) or Algorithm 8
(projected) finds no computed entry.  The tensor-core plan keeps the smaller of
two coverings of the needed triples: pairs within one half of the bins, or a
greedy set cover."""
import itertools

import pytest

from oracle import sarabande_oracle as O


@pytest.fixture(scope="module")
def sbg():
    from paper_2210_10206_gb300 import build, sbg as s
    build.build()
    s.lib()
    return s


GEOMETRIES = [(3, 1, 0), (3, 1, 4), (3, 2, 1), (3, 3, 5), (3, 5, 2), (3, 8, 4), (3, 10, 3), (3, 10, 4),
              (3, 13, 5), (2, 1, 0), (2, 2, 10), (2, 8, 4), (2, 10, 10), (2, 20, 3)]


@pytest.mark.parametrize("dim,nb,lmax", GEOMETRIES)
def test_every_term_finds_its_entry(sbg, dim, nb, lmax):
    for prec in (sbg.SBG_PREC_FP32, sbg.SBG_PREC_BF16X3, sbg.SBG_PREC_TF32X3):
        nt, nr, cov = sbg.sbg_plan4_info(dim, nb, lmax, prec)
        assert nt >= 1 and nr >= 1 and cov in (0, 1)
    if dim == 3 and lmax >= 1:  # the odd-parity tables of sbg_full_odd
        for prec in (sbg.SBG_PREC_FP32, sbg.SBG_PREC_BF16X3):
            nt, nr, cov = sbg.sbg_plan4_info(dim, nb, lmax, prec, 1)
            assert nt >= 1 and nr >= 1
    # both tensor-core precisions share one plan
    assert sbg.sbg_plan4_info(dim, nb, lmax, sbg.SBG_PREC_BF16X3) == sbg.sbg_plan4_info(dim, nb, lmax,
                                                                                         sbg.SBG_PREC_TF32X3)


def _needed_triples(lmax, nb):
    """Distinct triples of singles (l, m, b) that the even-parity 4PCF of
    Algorithm 6 reads with a nonzero coupling, up to order and M -> -M."""
    seen = set()
    for l1, l2, l3 in O.lambda_list(lmax):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if abs(m3) > l3 or O.coupling(l1, l2, l3, m1, m2, m3) == 0.0:
                    continue
                for b1, b2, b3 in itertools.product(range(nb), repeat=3):
                    t = sorted([(l1, m1, b1), (l2, m2, b2), (l3, m3, b3)])
                    u = sorted([(l1, -m1, b1), (l2, -m2, b2), (l3, -m3, b3)])
                    seen.add(tuple(min(t, u)))
    return len(seen)


def test_greedy_cover_at_the_benchmark_geometry(sbg):
    # 3D, lmax 4, 10 bins: the greedy cover halves the bin-half rows (65
    # tiles); trimming then empties the last tile of block m3 = 2 (445 rows,
    # 4 tiles) by moving the triples its rows cover alone to other blocks
    nt, nr, cov = sbg.sbg_plan4_info(3, 10, 4, sbg.SBG_PREC_BF16X3)
    assert cov == 1
    assert nt <= 29 and nr <= 3700
    # a row of block m3 meets at most nb (lmax - m3 + 1) columns, of which the
    # parity and triangle rules leave at most 3 l3 values at lmax 4: the rows
    # cannot reach every needed triple with fewer than needed / (3 nb) of them
    need = _needed_triples(4, 10)
    assert need == 72510  # of 73060 parity/triangle triples, 550 have only zero couplings
    assert nr * 3 * 10 >= need


def test_fp32_plan_at_the_benchmark_geometry(sbg):
    # the SIMT kernel pays per (row, column) entry: the column-weighted greedy
    # cover computes 134,320 entries per point instead of 239,360 (17,600 rows
    # b1 <= b2 against columns b3 >= b2)
    nt, nr, cov = sbg.sbg_plan4_info(3, 10, 4, sbg.SBG_PREC_FP32)
    assert cov == 1 and nr < 17600


def test_plan_argument_errors(sbg):
    for args in ((4, 10, 4), (1, 10, 4), (3, 0, 4), (3, 21, 4), (3, 10, 6), (3, 10, -1), (2, 10, 11)):
        with pytest.raises(sbg.SbgError):
            sbg.sbg_plan4_info(*args, sbg.SBG_PREC_BF16X3)
    with pytest.raises(sbg.SbgError):
        sbg.sbg_plan4_info(3, 10, 4, 2)  # precision 2 is not built
    with pytest.raises(sbg.SbgError):
        sbg.sbg_plan4_info(2, 10, 4, sbg.SBG_PREC_BF16X3, 1)  # odd parity is a 3D output


def test_trimmed_projected_plan(sbg):
    # 2D, mmax 10, 10 bins: the greedy cover's 27 tiles trim to 25 (block
    # m3 = 1 was 4 rows over 7 tiles, block m3 = 2 60 rows over 5)
    nt, nr, cov = sbg.sbg_plan4_info(2, 10, 10, sbg.SBG_PREC_BF16X3)
    assert cov == 1 and nt <= 25
