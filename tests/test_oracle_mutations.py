"""Planted mistakes: each plausible error in the oracle must make at least one
pin fail.  The mistakes are planted in the oracle (monkeypatched, on the CPU);
nothing here touches the CUDA path."""
import numpy as np
import pytest

from oracle import sarabande_oracle as O
import tests.test_oracle_pins as pins


def _fails(fn):
    try:
        fn()
    except AssertionError:
        return True
    return False


def test_convolution_instead_of_correlation_is_caught(monkeypatch):
    # Algorithms 2 and 4 read literally: the kernel e^{+i m phi} (not its
    # conjugate) convolved, FFT^-1(FFT(delta) * FFT(e^{i m phi} Theta))
    def conv(delta, kernel):
        return np.fft.ifftn(np.fft.fftn(delta) * np.fft.fftn(np.conj(kernel)))
    monkeypatch.setattr(O, "a_coefficient", conv)
    assert _fails(pins.test_c_projected_matches_direct_sum_and_conjugate_symmetry)
    assert _fails(pins.test_zeta3_projected_brute_force)


def test_dropped_parity_prefactor_is_caught(monkeypatch):
    orig = O.zeta3_full

    def no_sign(delta, edges, lmax, return_imag=False):
        z = orig(delta, edges, lmax)
        return z * np.array([(-1) ** l for l in range(lmax + 1)])[:, None, None]
    monkeypatch.setattr(O, "zeta3_full", no_sign)
    assert _fails(pins.test_zeta3_full_addition_theorem_brute_force)


def test_wrong_coupling_sign_is_caught(monkeypatch):
    orig = O.wigner3j

    def bad(j1, j2, j3, m1, m2, m3):
        v = orig(j1, j2, j3, m1, m2, m3)
        return -v if m1 < 0 else v
    monkeypatch.setattr(O, "wigner3j", bad)
    assert _fails(pins.test_wigner3j_matches_sympy)
    assert _fails(pins.test_zeta4_full_brute_force_triple_sums)


def test_missing_conjugate_on_second_bin_is_caught(monkeypatch):
    orig = O.c_projected

    def bad_c(delta, edges, m):
        c = orig(delta, edges, m)
        return c if m >= 0 else np.conj(c) * (-1) ** m   # Algorithm 8's (-1)^m c_{|m|}
    monkeypatch.setattr(O, "c_projected", bad_c)
    assert _fails(pins.test_zeta4_projected_brute_force)


def test_off_by_one_bin_edge_is_caught(monkeypatch):
    orig = O.bin_masks

    def loose(shape, edges):
        g = O.offset_grids(shape)
        r2 = sum(c * c for c in g).astype(np.float64)
        e2 = O.snapped_edges_sq(edges)
        return [(r2 >= e2[b]) & (r2 <= e2[b + 1]) for b in range(len(edges) - 1)]
    monkeypatch.setattr(O, "bin_masks", loose)
    assert _fails(pins.test_bin_counts_match_explicit_offsets)


def test_odd_parity_sign_and_part_are_caught(monkeypatch):
    # E(Lambda) dropped (the odd sum taken with +1), or the real part reported
    orig = O.zeta4_full_odd

    def no_parity_sign(delta, edges, lmax, return_real=False):
        r = orig(delta, edges, lmax, return_real)
        return (-r[0], -r[1]) if return_real else -r
    monkeypatch.setattr(O, "zeta4_full_odd", no_parity_sign)
    assert _fails(pins.test_zeta4_full_odd_brute_force_triple_sums)
    monkeypatch.setattr(O, "zeta4_full_odd", orig)

    def real_part(delta, edges, lmax, return_real=False):
        im, re = orig(delta, edges, lmax, True)
        return (re, im) if return_real else re
    monkeypatch.setattr(O, "zeta4_full_odd", real_part)
    assert _fails(pins.test_zeta4_full_odd_brute_force_triple_sums)


def test_normalization_mistakes_are_caught(monkeypatch):
    # the normalisation of Sec. 2.5 with a bin volume one cell off, the
    # continuous shell in place of the cell count, nbar per unit length instead
    # of per cell, and one nbar V factor too many
    orig_counts = O.bin_cell_counts
    orig_norm = O.normalization

    def plus_one(shape, edges):
        return orig_counts(shape, edges) + 1
    monkeypatch.setattr(O, "bin_cell_counts", plus_one)
    assert _fails(pins.test_normalization_constant_field_closed_form)
    monkeypatch.setattr(O, "bin_cell_counts", orig_counts)

    def continuous(shape, edges):
        e = np.asarray(edges, dtype=np.float64)
        if len(shape) == 3:
            return 4 * np.pi / 3 * (e[1:] ** 3 - e[:-1] ** 3)
        return np.pi * (e[1:] ** 2 - e[:-1] ** 2)
    monkeypatch.setattr(O, "bin_cell_counts", continuous)
    assert _fails(pins.test_normalization_constant_field_closed_form)
    monkeypatch.setattr(O, "bin_cell_counts", orig_counts)

    def nbar_per_length(shape, edges, n_gal, order, bins):
        return orig_norm(shape, edges, n_gal, order, bins) * (shape[0] ** (len(shape) - 1)) ** (order - 1)
    monkeypatch.setattr(O, "normalization", nbar_per_length)
    assert _fails(pins.test_normalization_constant_field_closed_form)
    assert _fails(pins.test_normalized_projected_3pcf_approaches_particle_counting)

    def extra_factor(shape, edges, n_gal, order, bins):
        return orig_norm(shape, edges, n_gal, order, list(bins) + [bins[0]])
    monkeypatch.setattr(O, "normalization", extra_factor)
    assert _fails(pins.test_normalization_constant_field_closed_form)
    assert _fails(pins.test_normalized_full_3pcf_approaches_particle_counting)


def test_ngal_before_mean_subtraction_is_caught(monkeypatch):
    orig = O.preprocess

    def early(field, subtract_mean=True):
        d, _ = orig(field, subtract_mean)
        return d, float((np.asarray(field, dtype=np.float64) + 1.0).sum())
    monkeypatch.setattr(O, "preprocess", early)
    assert _fails(pins.test_ngal_after_mean_subtraction_is_grid_size)
