"""Pins of the FP64 oracle against things other than itself: library routines
(scipy spherical harmonics, sympy 3j, numpy Legendre/arctan2), brute-force
direct sums over neighbour offsets (the paper's direct-counting validation,
Sec. 4.3), closed forms, invariants and symmetries.  CPU only."""
import math

import numpy as np
import pytest

from oracle import sarabande_oracle as O

RNG = np.random.default_rng(12345)


# ------------------------------------------------------------ helpers ----

def _offsets_in_bins(shape, edges):
    """Explicit list of integer offsets per bin by plain loops (independent of
    the oracle's vectorised masks)."""
    e2 = [float(e) ** 2 for e in edges]
    half = [n // 2 for n in shape]
    out = [[] for _ in range(len(edges) - 1)]
    rng = [range(-h + 1, h) for h in half]  # edges < N/2: -N/2 never in a bin
    import itertools
    for r in itertools.product(*rng):
        q = sum(c * c for c in r)
        for b in range(len(edges) - 1):
            if e2[b] < q <= e2[b + 1]:
                out[b].append(r)
    return out


def _shift(delta, r):
    """delta(x + r) as an array over x."""
    return np.roll(delta, shift=[-c for c in r], axis=tuple(range(delta.ndim)))


def _scipy_Y(l, m, r):
    from scipy.special import sph_harm_y
    z, y, x = (float(c) for c in r)
    rr = math.sqrt(x * x + y * y + z * z)
    theta = math.acos(z / rr)
    phi = math.atan2(y, x)
    return complex(sph_harm_y(l, m, theta, phi))


def _sympy_3j(j1, j2, j3, m1, m2, m3):
    from sympy.physics.wigner import wigner_3j
    return float(wigner_3j(j1, j2, j3, m1, m2, m3))


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------ basis and couplings ----

def test_sph_harm_matches_scipy():
    pts = RNG.normal(size=(40, 3))
    for l in range(0, 11):
        for m in range(-l, l + 1):
            mine = O.sph_harm(l, m, pts[:, 0], pts[:, 1], pts[:, 2])
            ref = np.array([_scipy_Y(l, m, p) for p in pts])
            assert np.max(np.abs(mine - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (l, m)


def test_sph_harm_addition_theorem_on_grid_directions():
    # sum_m |Y_lm|^2 = (2l+1)/(4 pi) at every direction (P6)
    z, y, x = O.offset_grids((9, 9, 9))
    keep = (x * x + y * y + z * z) > 0
    for l in range(0, 11):
        s = sum(np.abs(O.sph_harm(l, m, z[keep], y[keep], x[keep])) ** 2 for m in range(-l, l + 1))
        assert np.allclose(s, (2 * l + 1) / (4 * math.pi), rtol=1e-12, atol=0)


def test_wigner3j_matches_sympy():
    for j1 in range(0, 5):
        for j2 in range(0, 5):
            for j3 in range(abs(j1 - j2), min(j1 + j2, 6) + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = -m1 - m2
                        if abs(m3) > j3:
                            continue
                        a = O.wigner3j(j1, j2, j3, m1, m2, m3)
                        b = _sympy_3j(j1, j2, j3, m1, m2, m3)
                        assert abs(a - b) < 1e-14, (j1, j2, j3, m1, m2, m3, a, b)


def test_wigner3j_closed_forms_and_orthogonality():
    for l in range(0, 11):
        for m in range(-l, l + 1):
            # (l l 0; m -m 0) = (-1)^(l-m) / sqrt(2l+1)
            assert abs(O.wigner3j(l, l, 0, m, -m, 0) - (-1) ** (l - m) / math.sqrt(2 * l + 1)) < 1e-14
    for j1 in range(4):
        for j2 in range(4):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m3 in range(-j3, j3 + 1):
                    # sum over m1, m2 at fixed m3 = 1/(2 j3 + 1)
                    s = sum(O.wigner3j(j1, j2, j3, m1, -m1 - m3, m3) ** 2
                            for m1 in range(-j1, j1 + 1) if abs(m1 + m3) <= j2)
                    assert abs(s - 1.0 / (2 * j3 + 1)) < 1e-13


def test_lambda_list_counts_and_order():
    assert len(O.lambda_list(3)) == 23
    assert len(O.lambda_list(4)) == 42
    lam = O.lambda_list(2)
    assert lam[0] == (0, 0, 0)
    for (l1, l2, l3) in lam:
        assert (l1 + l2 + l3) % 2 == 0 and abs(l1 - l2) <= l3 <= min(l1 + l2, 2)


# ------------------------------------------------------------- binning ----

def test_bin_counts_match_explicit_offsets():
    for shape, edges in [((16, 16, 16), [0.5, 1.5, 2.5, 4.0]), ((32, 32), [2, 5, 8, 11, 14]),
                         ((64, 64), [2, 5, 8, 11, 14])]:
        expl = [len(v) for v in _offsets_in_bins(shape, edges)]
        assert list(O.bin_cell_counts(shape, edges)) == expl


def test_edge_snapping_log_bins():
    # log-spaced edges land a few ulp off integer squares (e.g. 2*sqrt(2)^2 = 8)
    e = np.geomspace(2.0, 64.0, 11)
    e2 = O.snapped_edges_sq(e)
    for v in e2:
        if abs(v - round(v)) < 1e-6:
            assert v == round(v)
    assert O.snapped_edges_sq([2 * math.sqrt(2)])[0] == 8.0


# ---------------------------------------------- convolution coefficients --

def test_a_fft_equals_direct_sum_3d():
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    for (l, m) in [(0, 0), (1, 0), (1, 1), (2, -1), (3, 2), (4, -4)]:
        ks = O.kernel_full(d.shape, edges, l, m)
        for k in ks:
            assert _rel(O.a_coefficient(d, k), O.brute_a(d, k)) < 1e-12


def test_a_is_a_correlation_not_a_convolution():
    # a(x) = sum_r K(r) delta(x+r): a delta spike at x0 gives a(x0 - r) = K(r)
    d = np.zeros((8, 8, 8))
    d[1, 2, 3] = 1.0
    k = O.kernel_full(d.shape, [0.5, 1.5], 1, 1)[0]
    a = O.a_coefficient(d, k)
    r = (0, 0, 1)  # (z, y, x)
    assert abs(a[1 - r[0], 2 - r[1], 3 - r[2]] - k[r]) < 1e-14
    assert abs(k[r] - np.conj(_scipy_Y(1, 1, r))) < 1e-14


def test_c_projected_matches_direct_sum_and_conjugate_symmetry():
    d = RNG.normal(size=(16, 16))
    edges = [0.5, 2.0, 3.5, 5.0]
    for m in range(0, 5):
        c = O.c_projected(d, edges, m)
        cm = O.c_projected(d, edges, -m)
        for b, k in enumerate(O.kernel_projected(d.shape, edges, m)):
            assert _rel(c[b], O.brute_a(d, k)) < 1e-12
        # c_{-m} = c_m^* for real delta (Sec. 2.2)
        assert _rel(cm, np.conj(c)) < 1e-12


# ---------------------------------------------------------- 3PCF pins ----

def _pair_sums(delta, offs1, offs2):
    """F[i, j] = sum_x delta(x) delta(x + r1_i) delta(x + r2_j)."""
    s1 = np.stack([_shift(delta, r) for r in offs1]).reshape(len(offs1), -1)
    s2 = np.stack([_shift(delta, r) for r in offs2]).reshape(len(offs2), -1)
    return (s1 * delta.reshape(1, -1)) @ s2.T


def test_zeta3_full_addition_theorem_brute_force():
    # P2: zeta_l = (-1)^l sqrt(2l+1)/(4 pi) sum_x delta sum_{r1,r2} delta delta L_l(r1.r2)
    from numpy.polynomial import legendre
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.0, 2.5]
    offs = _offsets_in_bins(d.shape, edges)
    z = O.zeta3_full(d, edges, 4)
    for b1 in range(3):
        for b2 in range(3):
            F = _pair_sums(d, offs[b1], offs[b2])
            u1 = np.array(offs[b1], float)
            u1 /= np.linalg.norm(u1, axis=1, keepdims=True)
            u2 = np.array(offs[b2], float)
            u2 /= np.linalg.norm(u2, axis=1, keepdims=True)
            cos = np.clip(u1 @ u2.T, -1, 1)
            for l in range(5):
                L = legendre.legval(cos, [0] * l + [1])
                ref = (-1) ** l * math.sqrt(2 * l + 1) / (4 * math.pi) * np.sum(F * L)
                assert abs(z[l, b1, b2] - ref) <= 1e-12 * max(1.0, np.abs(z).max()), (l, b1, b2)


def test_zeta3_full_reality_and_symmetry():
    d = RNG.normal(size=(8, 8, 8))
    zr, zi = O.zeta3_full(d, [0.5, 1.5, 2.5, 3.5], 3, return_imag=True)
    assert np.abs(zi).max() <= 1e-12 * np.abs(zr).max()
    assert np.allclose(zr, np.transpose(zr, (0, 2, 1)), rtol=1e-12, atol=1e-12 * np.abs(zr).max())


def test_zeta3_projected_brute_force():
    d = RNG.normal(size=(16, 16))
    edges = [0.5, 2.0, 3.5, 5.0]
    offs = _offsets_in_bins(d.shape, edges)
    z = O.zeta3_projected(d, edges, 4)
    for b1 in range(3):
        for b2 in range(3):
            F = _pair_sums(d, offs[b1], offs[b2])
            p1 = np.array([math.atan2(r[0], r[1]) for r in offs[b1]])
            p2 = np.array([math.atan2(r[0], r[1]) for r in offs[b2]])
            for m in range(5):
                ph = np.exp(-1j * m * p1)[:, None] * np.exp(1j * m * p2)[None, :]
                ref = np.sum(F * ph)
                assert abs(z[m, b1, b2] - ref) <= 1e-12 * np.abs(z).max(), (m, b1, b2)
    # zeta^{b2 b1}_m = conj zeta^{b1 b2}_m
    assert _rel(z, np.conj(np.transpose(z, (0, 2, 1)))) < 1e-12


def test_ell0_special_case():
    # P3: zeta_0^{b1 b2} = (1/4pi) sum delta S_b1 S_b2 with S_b = sum_{r in b} delta(x+r)
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    offs = _offsets_in_bins(d.shape, edges)
    S = [sum(_shift(d, r) for r in ob) for ob in offs]
    z = O.zeta3_full(d, edges, 0)
    for b1 in range(3):
        for b2 in range(3):
            assert abs(z[0, b1, b2] - np.sum(d * S[b1] * S[b2]) / (4 * math.pi)) < 1e-12 * np.abs(z).max()
    z4 = O.zeta4_full(d, edges, 0)
    for b1 in range(3):
        for b2 in range(3):
            for b3 in range(3):
                ref = np.sum(d * S[b1] * S[b2] * S[b3]) * (4 * math.pi) ** -1.5
                assert abs(z4[0, b1, b2, b3] - ref) < 1e-12 * np.abs(z4).max()


# ---------------------------------------------------------- 4PCF pins ----

def _P_lambda(lam, u1, u2, u3):
    """Isotropic basis P_Lambda at direction triples from scipy Y and sympy 3j
    (Sec. 2.3), independent of the oracle's Y and 3j."""
    l1, l2, l3 = lam
    Y1 = {m: np.array([_scipy_Y(l1, m, r) for r in u1]) for m in range(-l1, l1 + 1)}
    Y2 = {m: np.array([_scipy_Y(l2, m, r) for r in u2]) for m in range(-l2, l2 + 1)}
    Y3 = {m: np.array([_scipy_Y(l3, m, r) for r in u3]) for m in range(-l3, l3 + 1)}
    P = np.zeros((len(u1), len(u2), len(u3)), dtype=complex)
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            m3 = -m1 - m2
            if abs(m3) > l3:
                continue
            c = (-1) ** (l1 + l2 + l3) * _sympy_3j(l1, l2, l3, m1, m2, m3)
            P += c * Y1[m1][:, None, None] * Y2[m2][None, :, None] * Y3[m3][None, None, :]
    return P


def test_zeta4_full_brute_force_triple_sums():
    # P1 for the 4PCF: zeta_Lambda = sum_x delta sum_{r1,r2,r3} delta delta delta P_Lambda
    d = RNG.normal(size=(6, 6, 6))
    edges = [0.5, 1.5, 2.0]
    offs = _offsets_in_bins(d.shape, edges)
    lmax = 2
    z = O.zeta4_full(d, edges, lmax)
    lams = O.lambda_list(lmax)
    sh = [np.stack([_shift(d, r) for r in ob]).reshape(len(ob), -1) for ob in offs]
    dd = d.reshape(-1)
    for b1 in range(2):
        for b2 in range(2):
            for b3 in range(2):
                F = np.einsum("x,ix,jx,kx->ijk", dd, sh[b1], sh[b2], sh[b3])
                for i, lam in enumerate(lams):
                    P = _P_lambda(lam, offs[b1], offs[b2], offs[b3])
                    ref = np.sum(F * P)
                    assert abs(ref.imag) < 1e-10 * max(1.0, abs(ref.real))
                    assert abs(z[i, b1, b2, b3] - ref.real) <= 1e-12 * np.abs(z).max(), (lam, b1, b2, b3)


def test_lambda_list_odd_enumeration():
    # every odd (l1, l2, l3) obeying the triangle rule with each l <= lmax, once,
    # in the loop order of Algorithm 6 (l1, then l2, then l3 ascending)
    import itertools
    for lmax in range(0, 6):
        want = sorted(t for t in itertools.product(range(lmax + 1), repeat=3)
                      if sum(t) % 2 == 1 and abs(t[0] - t[1]) <= t[2] <= t[0] + t[1])
        got = O.lambda_list_odd(lmax)
        assert got == want, lmax
    assert O.lambda_list_odd(0) == [] and O.lambda_list_odd(1) == [(1, 1, 1)]


def test_zeta4_full_odd_brute_force_triple_sums():
    # P1 for the odd-parity 4PCF.  The a-coefficients carry Y* (Eq. almconv),
    # so sum_M C a a a = sum_x delta sum_{r1,r2,r3} delta delta delta
    # conj(P_Lambda); for odd Lambda conj(P_Lambda) = -P_Lambda (P is
    # imaginary), and E(Lambda) = -1 of Eq. mu cancels that sign:
    # zeta = sum delta delta delta delta P_Lambda, reported as its imaginary part
    d = RNG.normal(size=(6, 6, 6))
    edges = [0.5, 1.5, 2.0]
    offs = _offsets_in_bins(d.shape, edges)
    lmax = 2
    z, zr = O.zeta4_full_odd(d, edges, lmax, return_real=True)
    lams = O.lambda_list_odd(lmax)
    assert len(lams) == 4 and np.abs(z).max() > 0
    sh = [np.stack([_shift(d, r) for r in ob]).reshape(len(ob), -1) for ob in offs]
    dd = d.reshape(-1)
    for b1 in range(2):
        for b2 in range(2):
            for b3 in range(2):
                F = np.einsum("x,ix,jx,kx->ijk", dd, sh[b1], sh[b2], sh[b3])
                for i, lam in enumerate(lams):
                    ref = np.sum(F * _P_lambda(lam, offs[b1], offs[b2], offs[b3]))
                    assert abs(ref.real) < 1e-10 * max(1.0, abs(ref.imag))
                    assert abs(z[i, b1, b2, b3] - ref.imag) <= 1e-12 * np.abs(z).max(), (lam, b1, b2, b3)
    assert np.abs(zr).max() <= 1e-12 * np.abs(z).max()


def test_zeta4_full_odd_parity_under_mirror_and_rotations():
    # odd Lambda: a mirror flips the sign, proper rotations and shifts keep it;
    # a mirror-symmetric field has no odd-parity 4PCF
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    z = O.zeta4_full_odd(d, edges, 2)
    assert np.abs(z).max() > 0
    for t in [np.roll(d, (2, 1, 3), axis=(0, 1, 2)), np.rot90(d, 1, axes=(0, 1)), np.rot90(d, 1, axes=(1, 2))]:
        assert _rel(O.zeta4_full_odd(np.ascontiguousarray(t), edges, 2), z) < 1e-11
    for ax in range(3):
        m = np.ascontiguousarray(np.flip(d, axis=ax))
        assert _rel(O.zeta4_full_odd(m, edges, 2), -z) < 1e-11
    sym = d + np.roll(np.flip(d, axis=2), 1, axis=2)  # f(z, y, -x) = f(z, y, x) on the periodic grid
    assert np.abs(O.zeta4_full_odd(sym, edges, 2)).max() <= 1e-11 * np.abs(O.zeta4_full(sym, edges, 2)).max()


def test_zeta4_full_l3_zero_reduces_to_weighted_3pcf():
    # P4: zeta_{l l 0}^{b1 b2 b3}[delta] = 3PCF_l^{b1 b2} with primary weight delta*S_b3/sqrt(4pi)
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    offs = _offsets_in_bins(d.shape, edges)
    lmax = 2
    z4 = O.zeta4_full(d, edges, lmax)
    lams = O.lambda_list(lmax)
    for b3 in range(3):
        S3 = sum(_shift(d, r) for r in offs[b3])
        w = d * S3 / math.sqrt(4 * math.pi)
        for l in range(lmax + 1):
            i = lams.index((l, l, 0))
            for b1 in range(3):
                for b2 in range(3):
                    # 3PCF with primary weight w and the same a-coefficients of delta
                    s = 0
                    for m in range(-l, l + 1):
                        a = O.a_full(d, edges, l, m)
                        s += np.sum(w * a[b1] * np.conj(a[b2]))
                    ref = ((-1) ** l / math.sqrt(2 * l + 1) * s).real
                    assert abs(z4[i, b1, b2, b3] - ref) < 1e-12 * np.abs(z4).max()


def test_zeta4_full_reality_and_permutation_symmetry():
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    zr, zi = O.zeta4_full(d, edges, 2, return_imag=True)
    assert np.abs(zi).max() <= 1e-12 * np.abs(zr).max()
    lams = O.lambda_list(2)
    for i, (l1, l2, l3) in enumerate(lams):
        j = lams.index((l2, l1, l3))
        assert _rel(zr[i], np.transpose(zr[j], (1, 0, 2))) < 1e-11 or np.abs(zr[i]).max() < 1e-12


def test_zeta4_projected_brute_force():
    d = RNG.normal(size=(12, 12))
    edges = [0.5, 1.5, 2.5]
    offs = _offsets_in_bins(d.shape, edges)
    mmax = 2
    z = O.zeta4_projected(d, edges, mmax)
    sh = [np.stack([_shift(d, r) for r in ob]).reshape(len(ob), -1) for ob in offs]
    ph = [np.array([math.atan2(r[0], r[1]) for r in ob]) for ob in offs]
    dd = d.reshape(-1)
    for b1 in range(2):
        for b2 in range(2):
            for b3 in range(2):
                F = np.einsum("x,ix,jx,kx->ijk", dd, sh[b1], sh[b2], sh[b3])
                for m1 in range(-mmax, mmax + 1):
                    for m2 in range(-mmax, mmax + 1):
                        m3 = -m1 - m2
                        if abs(m3) > mmax:
                            assert z[m1 + mmax, m2 + mmax, b1, b2, b3] == 0
                            continue
                        E = (np.exp(-1j * m1 * ph[b1])[:, None, None] * np.exp(-1j * m2 * ph[b2])[None, :, None]
                             * np.exp(-1j * m3 * ph[b3])[None, None, :])
                        ref = np.sum(F * E)
                        assert abs(z[m1 + mmax, m2 + mmax, b1, b2, b3] - ref) <= 1e-12 * np.abs(z).max()
    # zeta_{-m1,-m2} = conj zeta_{m1,m2}
    assert _rel(z[::-1, ::-1], np.conj(z)) < 1e-12


# ------------------------------------------------------------ invariants --

def test_shift_rotation_mirror_invariance_full():
    d = RNG.normal(size=(8, 8, 8))
    edges = [0.5, 1.5, 2.5, 3.5]
    z3 = O.zeta3_full(d, edges, 3)
    z4 = O.zeta4_full(d, edges, 2)
    for t in [np.roll(d, (1, 3, 5), axis=(0, 1, 2)), np.rot90(d, 1, axes=(0, 1)),
              np.rot90(d, 1, axes=(1, 2)), np.rot90(d, 1, axes=(0, 2)), d[:, :, ::-1]]:
        t = np.ascontiguousarray(t)
        assert _rel(O.zeta3_full(t, edges, 3), z3) < 1e-11
        assert _rel(O.zeta4_full(t, edges, 2), z4) < 1e-11


def test_shift_rotation_mirror_projected():
    d = RNG.normal(size=(16, 16))
    edges = [0.5, 2.0, 3.5, 5.0]
    z3 = O.zeta3_projected(d, edges, 4)
    z4 = O.zeta4_projected(d, edges, 2)
    for t in [np.roll(d, (3, 7), axis=(0, 1)), np.rot90(d, 1)]:
        t = np.ascontiguousarray(t)
        assert _rel(O.zeta3_projected(t, edges, 4), z3) < 1e-11
        assert _rel(O.zeta4_projected(t, edges, 2), z4) < 1e-11
    t = np.ascontiguousarray(d[:, ::-1])  # mirror x -> -x conjugates projected outputs
    assert _rel(O.zeta3_projected(t, edges, 4), np.conj(z3)) < 1e-11
    assert _rel(O.zeta4_projected(t, edges, 2), np.conj(z4)) < 1e-11


# ------------------------------------------------------ ensemble / particles --

def test_gaussian_random_field_mean_3pcf_vanishes():
    # P10: for a Gaussian field the ensemble-mean 3PCF is zero
    from paper_2210_10206_gb300 import synth
    edges = [1.5, 3.0, 4.5]
    zs = []
    for s in range(48):
        g = synth.gaussian_field(500 + s, (16, 16, 16), -2.0)
        zs.append(O.zeta3_full(g - g.mean(), edges, 2))
    zs = np.array(zs)
    mean, err = zs.mean(0), zs.std(0) / math.sqrt(len(zs))
    assert np.all(np.abs(mean) < 4.5 * err + 1e-12)
    # and a lognormal field of the same spectrum has a clearly non-zero mean zeta_0
    ln = []
    for s in range(16):
        f = synth.lognormal_field(500 + s, (16, 16, 16), 1.0, -2.0, dtype=np.float64)
        ln.append(O.zeta3_full(f, edges, 0)[0])
    ln = np.array(ln)
    assert np.max(np.abs(ln.mean(0)) / (ln.std(0) / 4.0)) > 4.0


def _min_image(d, n):
    d = np.mod(d + n // 2, n) - n // 2
    return d


def test_particle_direct_counting_full_3pcf_4pcf():
    # P11 / Sec. 4.3: unit-weight cells vs direct counting over particle pairs/triples
    from numpy.polynomial import legendre
    from paper_2210_10206_gb300 import synth
    shape = (48, 48, 48)
    f = synth.particle_field(11, shape, 40)
    edges = list(np.linspace(2.0, 20.0, 5))
    z3 = O.zeta3_full(f, edges, 2)
    z4 = O.zeta4_full(f, edges, 2)
    pos = np.argwhere(f > 0)
    e2 = O.snapped_edges_sq(edges)
    nb = len(edges) - 1
    ref3 = np.zeros_like(z3)
    ref4 = np.zeros_like(z4)
    lams = O.lambda_list(2)
    for p in pos:
        sep = _min_image(pos - p, shape[0])
        q2 = (sep ** 2).sum(1)
        nbr = [sep[(q2 > e2[b]) & (q2 <= e2[b + 1])] for b in range(nb)]
        unit = [v / np.linalg.norm(v, axis=1, keepdims=True) if len(v) else v for v in nbr]
        for b1 in range(nb):
            for b2 in range(nb):
                if len(nbr[b1]) == 0 or len(nbr[b2]) == 0:
                    continue
                cos = np.clip(unit[b1] @ unit[b2].T, -1, 1)
                for l in range(3):
                    ref3[l, b1, b2] += ((-1) ** l * math.sqrt(2 * l + 1) / (4 * math.pi)
                                        * legendre.legval(cos, [0] * l + [1]).sum())
                for b3 in range(nb):
                    if len(nbr[b3]) == 0:
                        continue
                    for i, lam in enumerate(lams):
                        ref4[i, b1, b2, b3] += _P_lambda(lam, nbr[b1], nbr[b2], nbr[b3]).sum().real
    assert _rel(z3, ref3) < 1e-12
    assert _rel(z4, ref4) < 1e-12


def test_particle_direct_counting_projected():
    from paper_2210_10206_gb300 import synth
    shape = (128, 128)
    f = synth.particle_field(13, shape, 41)
    edges = list(np.linspace(2.0, 40.0, 11))
    mmax = 3
    z3 = O.zeta3_projected(f, edges, mmax)
    z4 = O.zeta4_projected(f, edges, 2)
    pos = np.argwhere(f > 0)
    e2 = O.snapped_edges_sq(edges)
    nb = len(edges) - 1
    r3 = np.zeros_like(z3)
    r4 = np.zeros_like(z4)
    for p in pos:
        sep = _min_image(pos - p, shape[0])
        q2 = (sep ** 2).sum(1)
        phis = [np.arctan2(sep[:, 0], sep[:, 1])[(q2 > e2[b]) & (q2 <= e2[b + 1])] for b in range(nb)]
        for m in range(mmax + 1):
            c = np.array([np.exp(-1j * m * ph).sum() for ph in phis])
            r3[m] += c[:, None] * np.conj(c)[None, :]
        cm = {m: np.array([np.exp(-1j * m * ph).sum() for ph in phis]) for m in range(-2, 3)}
        for m1 in range(-2, 3):
            for m2 in range(-2, 3):
                m3 = -m1 - m2
                if abs(m3) > 2:
                    continue
                r4[m1 + 2, m2 + 2] += np.einsum("i,j,k->ijk", cm[m1], cm[m2], cm[m3])
    assert _rel(z3, r3) < 1e-12
    assert _rel(z4, r4) < 1e-12


# ---------------------------------------------------------- normalisation --

def test_normalization_constant_field_closed_form():
    # For a constant field delta = c (no mean subtraction) every binned
    # coefficient is known in closed form: a^b_00 = c V_b Y_00, c^b_0 = c V_b
    # with V_b the number of cells of bin b, N_gal = N_g (1 + c) and
    # nbar = 1 + c (Eq. num_gals with L = N).  The normalised monopoles are then
    # independent of the bins:  3PCF  c^3 / ((1 + c)^3 4 pi)  (full) and
    # c^3 / (1 + c)^3 (projected); 4PCF (000) c^4 / ((1 + c)^4 (4 pi)^{3/2}).
    # Any other bin measure (a cell more or less, the continuous shell), a
    # wrong nbar or a wrong number of factors breaks these identities.
    c = 0.75
    shape3 = (12, 12, 12)
    edges3 = [0.0, 1.5, 2.9, 4.5, 5.5]
    d3, ngal3 = O.preprocess(np.full(shape3, c), subtract_mean=False)
    assert ngal3 == pytest.approx(12 ** 3 * (1 + c), rel=1e-14)
    z3 = O.zeta3_full(d3, edges3, 0)[0]
    z4 = O.zeta4_full(d3, edges3, 0)[0]
    nb = len(edges3) - 1
    for b1 in range(nb):
        for b2 in range(nb):
            n3 = O.normalization(shape3, edges3, ngal3, 3, [b1, b2])
            assert z3[b1, b2] / n3 == pytest.approx(c ** 3 / ((1 + c) ** 3 * 4 * math.pi), rel=1e-12)
            for b3 in range(nb):
                n4 = O.normalization(shape3, edges3, ngal3, 4, [b1, b2, b3])
                assert z4[b1, b2, b3] / n4 == pytest.approx(c ** 4 / ((1 + c) ** 4 * (4 * math.pi) ** 1.5),
                                                            rel=1e-12)
    shape2 = (24, 24)
    edges2 = [0.5, 2.0, 4.5, 7.0, 11.0]
    d2, ngal2 = O.preprocess(np.full(shape2, c), subtract_mean=False)
    p3 = O.zeta3_projected(d2, edges2, 0)[0]
    for b1 in range(nb):
        for b2 in range(nb):
            n = O.normalization(shape2, edges2, ngal2, 3, [b1, b2])
            assert p3[b1, b2].real / n == pytest.approx(c ** 3 / (1 + c) ** 3, rel=1e-12)
            assert abs(p3[b1, b2].imag) < 1e-9 * abs(p3[b1, b2].real)


def test_ngal_after_mean_subtraction_is_grid_size():
    # Eq. num_gals evaluated after the mean is removed (Sec. 4.1) is exactly N_g,
    # whatever the field's mean was; without subtraction it counts the field
    from paper_2210_10206_gb300 import synth
    f = synth.particle_field(21, (32, 32), 50)
    _, ngal = O.preprocess(f, subtract_mean=True)
    assert ngal == pytest.approx(32 * 32, rel=1e-13)
    _, ngal_raw = O.preprocess(f, subtract_mean=False)
    assert ngal_raw == pytest.approx(32 * 32 + 50, rel=1e-13)


def _dc_projected3(pos, n, e2, nb, mmax):
    """Direct counting over particle pairs around each primary (Sec. 4.3)."""
    r = np.zeros((mmax + 1, nb, nb), dtype=np.complex128)
    for p in pos:
        sep = _min_image(pos - p, n)
        q2 = (sep ** 2).sum(1)
        phis = [np.arctan2(sep[:, 0], sep[:, 1])[(q2 > e2[b]) & (q2 <= e2[b + 1])] for b in range(nb)]
        for m in range(mmax + 1):
            cm = np.array([np.exp(-1j * m * ph).sum() for ph in phis])
            r[m] += cm[:, None] * np.conj(cm)[None, :]
    return r


def test_normalized_projected_3pcf_approaches_particle_counting():
    # Sec. 2.5 / Sec. 4.3 (Fig. normalization_projected): 41 unit-weight
    # particles; the grid coefficients divided by N = N_gal prod nbar A_bin with
    # A_bin = cell count (Eq. proj_b_area, proj_norm) against direct counting
    # divided by the particle code's normalisation, whose bin areas are the
    # continuous annuli pi (r+^2 - r-^2) and nbar = N_part / L^2.  Unnormalised
    # they agree to rounding; normalised they differ by the lattice's
    # approximation of each annulus, which shrinks as the cells get smaller
    # (box and bins scaled together).
    from paper_2210_10206_gb300 import synth
    errs = []
    for n in (64, 128, 256, 512):
        edges = np.linspace(n / 32.0, 0.45 * n, 11)
        f = synth.particle_field(13, (n, n), 41)
        pos = np.argwhere(f > 0)
        npart = len(pos)
        nb, mmax = 10, 2
        grid = O.zeta3_projected(f, edges, mmax)
        dc = _dc_projected3(pos, n, O.snapped_edges_sq(edges), nb, mmax)
        assert _rel(grid, dc) < 1e-12
        nbar = npart / float(n * n)
        area = math.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
        gn = np.empty_like(grid)
        dn = np.empty_like(dc)
        for b1 in range(nb):
            for b2 in range(nb):
                gn[:, b1, b2] = grid[:, b1, b2] / O.normalization((n, n), edges, npart, 3, [b1, b2])
                dn[:, b1, b2] = dc[:, b1, b2] / (npart * nbar * area[b1] * nbar * area[b2])
        errs.append(_rel(gn, dn))
    # measured 9.5e-2, 4.8e-2, 1.7e-2, 3.5e-3 for 64^2 .. 512^2
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 3e-2 and errs[3] < 1e-2, errs
    assert errs[0] / errs[3] > 10, errs


def test_normalized_full_3pcf_approaches_particle_counting():
    # the same check in 3D (Sec. 2.5, shells (4 pi / 3)(r+^3 - r-^3)), monopole
    from paper_2210_10206_gb300 import synth
    errs = []
    for n in (32, 64, 128):
        edges = np.linspace(n / 16.0, 0.45 * n, 5)
        f = synth.particle_field(17, (n, n, n), 104)
        pos = np.argwhere(f > 0)
        npart = len(pos)
        nb = 4
        grid = O.zeta3_full(f, edges, 0)[0]
        e2 = O.snapped_edges_sq(edges)
        dc = np.zeros((nb, nb))
        for p in pos:
            q2 = (_min_image(pos - p, n) ** 2).sum(1)
            cnt = np.array([((q2 > e2[b]) & (q2 <= e2[b + 1])).sum() for b in range(nb)], dtype=np.float64)
            dc += np.outer(cnt, cnt) / (4 * math.pi)   # l = 0: Y00^2 = 1 / (4 pi)
        assert _rel(grid, dc) < 1e-12
        nbar = npart / float(n ** 3)
        vol = 4 * math.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
        gn = np.array([[grid[b1, b2] / O.normalization((n, n, n), edges, npart, 3, [b1, b2]) for b2 in range(nb)]
                       for b1 in range(nb)])
        dn = dc / (npart * nbar ** 2 * np.outer(vol, vol))
        errs.append(_rel(gn, dn))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-2, errs


def test_single_entry_oracle_matches_full_tensor():
    # the one-entry path used for spot checks at full size equals the full tensor
    d = RNG.normal(size=(16, 16, 16))
    edges = [0.5, 1.5, 2.5, 3.5, 5.0]
    z4 = O.zeta4_full(d, edges, 2)
    lams = O.lambda_list(2)
    entries = [((0, 0, 0), 0, 1, 2), ((1, 1, 2), 3, 0, 1), ((2, 2, 2), 2, 2, 3), ((2, 1, 1), 1, 3, 3)]
    got = O.zeta4_full_entries(d, edges, entries)
    for (lam, b1, b2, b3), g in zip(entries, got):
        assert abs(g - z4[lams.index(lam), b1, b2, b3]) < 1e-12 * np.abs(z4).max()
    k = O.kernel_full(d.shape, edges, 2, -1)
    assert np.array_equal(O.kernel_full_bin(d.shape, edges, 2, -1, 2), k[2])


def test_single_entry_oracles_match_full_tensors():
    # the one-entry paths that write the full-size goldens equal the full
    # tensors: the odd-parity option, and the 3PCF entries built from m >= 0
    d = RNG.normal(size=(16, 16, 16))
    edges = [0.5, 1.5, 2.5, 3.5, 5.0]
    zo = O.zeta4_full_odd(d, edges, 2)
    lams = O.lambda_list_odd(2)
    entries = [((1, 1, 1), 0, 1, 2), ((1, 2, 2), 3, 0, 1), ((2, 1, 2), 2, 2, 3), ((2, 2, 1), 1, 3, 3)]
    got = O.zeta4_full_entries(d, edges, entries, odd=True)
    for (lam, b1, b2, b3), g in zip(entries, got):
        assert abs(g - zo[lams.index(lam), b1, b2, b3]) < 1e-12 * np.abs(zo).max()
    z3 = O.zeta3_full(d, edges, 4)
    e3 = [(0, 0, 0), (1, 2, 1), (2, 3, 3), (3, 0, 3), (4, 1, 2)]
    for (l, b1, b2), g in zip(e3, O.zeta3_full_entries(d, edges, e3)):
        assert abs(g - z3[l, b1, b2]) < 1e-12 * np.abs(z3).max()


def test_projected_entry_oracle_matches_full_tensors():
    d = RNG.normal(size=(24, 24))
    edges = [0.5, 2.0, 3.5, 5.0, 7.5]
    z3 = O.zeta3_projected(d, edges, 3)
    z4 = O.zeta4_projected(d, edges, 3)
    e3 = [(0, 1, 2), (3, 3, 0), (2, 2, 2)]
    e4 = [((1, 2), 0, 1, 3), ((-3, 1), 2, 2, 0), ((3, -3), 1, 0, 1), ((0, 0), 3, 3, 3)]
    g3, g4 = O.zeta_projected_entries(d, edges, e3, e4)
    for (m, b1, b2), g in zip(e3, g3):
        assert abs(g - z3[m, b1, b2]) < 1e-12 * np.abs(z3).max()
    for ((m1, m2), b1, b2, b3), g in zip(e4, g4):
        assert abs(g - z4[m1 + 3, m2 + 3, b1, b2, b3]) < 1e-12 * np.abs(z4).max()
