"""Pins of the FP64 C++ oracle (oracle/sarabande_oracle.cpp) against things
other than itself: numpy's FFT for its own FFT, sympy for its 3j, brute-force
neighbour sums with scipy's Y_lm for its coefficients, direct counting over
particle pairs (Sec. 4.3), and the pinned Python oracle for every output on
small grids (power-of-two and other sides).  CPU only."""
import math

import numpy as np
import pytest

from oracle import cpp as C
from oracle import sarabande_oracle as O
import tests.test_oracle_pins as pins

RNG = np.random.default_rng(2468)


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def test_fft_matches_numpy():
    for shape in [(8, 8, 8), (16, 16, 16), (32, 32), (12, 12, 12), (6, 10)]:
        x = RNG.normal(size=shape) + 1j * RNG.normal(size=shape)
        assert _rel(C.fftn(x, -1), np.fft.fftn(x)) < 1e-13
        assert _rel(C.fftn(x, +1), np.fft.ifftn(x) * x.size) < 1e-13


def test_wigner3j_matches_sympy():
    for j1, j2, j3, m1, m2 in [(1, 1, 0, 1, -1), (2, 3, 4, -2, 1), (4, 4, 4, 2, -3), (10, 10, 10, 3, -7),
                               (5, 3, 2, 0, 0), (3, 3, 3, 1, 1), (2, 2, 2, 1, 1)]:
        assert abs(C.wigner3j(j1, j2, j3, m1, m2, -m1 - m2) - pins._sympy_3j(j1, j2, j3, m1, m2, -m1 - m2)) < 1e-14
    assert C.wigner3j(1, 1, 3, 0, 0, 0) == 0.0


def test_coefficients_match_direct_neighbour_sums():
    d = RNG.normal(size=(10, 10, 10))
    edges = [0.5, 1.5, 2.5, 3.5]
    offs = pins._offsets_in_bins(d.shape, edges)
    for l, m in [(0, 0), (1, -1), (2, 1), (3, -2), (3, 3)]:
        for b in range(3):
            ref = sum(np.conj(pins._scipy_Y(l, m, r)) * pins._shift(d, r) for r in offs[b])
            assert _rel(C.coefficient(d, edges, l, m, b), ref) < 1e-12
    d2 = RNG.normal(size=(18, 18))
    e2 = [0.5, 2.5, 4.0, 6.5]
    offs2 = pins._offsets_in_bins(d2.shape, e2)
    for m in (-3, 0, 2):
        for b in range(3):
            ref = sum(np.exp(-1j * m * math.atan2(r[0], r[1])) * pins._shift(d2, r) for r in offs2[b])
            assert _rel(C.coefficient(d2, e2, 0, m, b), ref) < 1e-12


def test_projected_3pcf_matches_particle_counting():
    from paper_2210_10206_gb300 import synth
    n, mmax = 64, 3
    f = synth.particle_field(19, (n, n), 30)
    edges = list(np.linspace(2.0, 20.0, 6))
    z = C.zeta3_projected(f, edges, mmax)
    pos = np.argwhere(f > 0)
    e2 = O.snapped_edges_sq(edges)
    ref = pins._dc_projected3(pos, n, e2, len(edges) - 1, mmax)
    assert _rel(z, ref) < 1e-12


@pytest.mark.parametrize("n", [8, 12])
def test_full_outputs_match_python_oracle(n):
    d = RNG.normal(size=(n, n, n))
    d -= d.mean()
    edges = [0.5, 1.5, 2.5, 3.9]
    assert _rel(C.zeta3_full(d, edges, 3), O.zeta3_full(d, edges, 3)) < 1e-12
    assert _rel(C.zeta4_full(d, edges, 2), O.zeta4_full(d, edges, 2)) < 1e-12
    assert _rel(C.zeta4_full(d, edges, 2, odd=True), O.zeta4_full_odd(d, edges, 2)) < 1e-12
    assert C.lambda_list(3) == O.lambda_list(3)
    assert C.lambda_list(3, odd=True) == O.lambda_list_odd(3)


def test_full_4pcf_combination_on_given_points():
    # the combination step alone, over a subset of the points (the bench's
    # timing sample), against the Python oracle's triple sums on the same points
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    nb, lmax, npts = 3, 2, 200
    a = np.stack([np.stack([O.a_coefficient(d, k) for k in O.kernel_full(d.shape, edges, l, m)]).reshape(nb, -1)
                  for l in range(lmax + 1) for m in range(-l, l + 1)])
    w = d.reshape(1, -1)[:, :npts]
    got = C.zeta4_combine(w, a[:, :, :npts], lmax)
    ai = {(l, m): a[l * l + l + m, :, :npts] for l in range(lmax + 1) for m in range(-l, l + 1)}
    ref = np.zeros_like(got)
    for i, (l1, l2, l3) in enumerate(O.lambda_list(lmax)):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -m1 - m2
                if abs(m3) > l3:
                    continue
                ref[i] += (O.coupling(l1, l2, l3, m1, m2, m3) * O.triple_sum(w, ai[(l1, m1)], ai[(l2, m2)],
                                                                             ai[(l3, m3)])).real
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("n", [16, 18])
def test_projected_outputs_match_python_oracle(n):
    d = RNG.normal(size=(n, n))
    edges = [0.5, 2.0, 3.5, 5.0, 7.5]
    assert _rel(C.zeta3_projected(d, edges, 4), O.zeta3_projected(d, edges, 4)) < 1e-12
    assert _rel(C.zeta4_projected(d, edges[:4], 2), O.zeta4_projected(d, edges[:4], 2)) < 1e-12
