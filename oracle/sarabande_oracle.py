"""FP64 CPU oracle for the SARABANDE 3/4PCF hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` import it.  It shares no code with the CUDA path.

It is a plain, slow restatement of the definitions of Sunseri et al. 2022
(arXiv 2210.10206), in float64 / complex128, with numpy's FFT as the only
library step.  Each function cites the passage it follows.

Conventions adopted where the paper is silent or inconsistent (each is listed
with its reason in the design notes of the repository):

* Offsets are minimum-image integer vectors of the periodic grid, origin at
  index 0; array index (i, j, k) of a C-order 3D array maps to (z, y, x) and
  (i, j) of a 2D array to (y, x).  Box side = N cells, cell volume 1 (Sec. 4.2).
* Bin b holds offsets with  e_b^2 < |r|^2 <= e_{b+1}^2  (Algorithm 1 mask),
  with squared edges snapped to the nearest integer when within 1e-9 relative.
* The binned coefficient is a correlation, a(x) = sum_r K(r) delta(x + r)
  (Eq. almconv and its footnote), with K = Y*_lm Theta^b (3D) or
  e^{-i m phi} Theta^b (2D, Eq. c_m def kernel).  Masks are 0/1: the 1/V_b of
  Eq. bin_volume_unity is not applied (Algorithm 1 applies none either).
* Outputs are raw sums over grid points (Algorithms 5-8), not volume averages.
* Full 3PCF keeps the (-1)^l / sqrt(2l+1) prefactor of Eq. alm_to_zeta_clean;
  the projected 3PCF omits the 1/(2 pi)^2 of Eq. proj_3pcf_coeff (Algorithm 7
  omits it).
* Full 4PCF: even-parity Lambda in the loop order of Algorithm 6, the full sum
  over M with |m3| <= l3, coupling C^Lambda_M = (-1)^(l1+l2+l3) (3j) (Sec. 2.3).
  Odd-parity Lambda (l1 + l2 + l3 odd) take E(Lambda) = -1 of Eq. mu; their
  M-sum is imaginary for a real delta and is reported as its imaginary part.
* Projected 4PCF: c_{-m} taken from its own kernel e^{+i m phi} (equal to
  conj(c_m), Sec. 2.2), all (m1, m2) with |m1|, |m2|, |m1 + m2| <= mmax.

Y_lm: orthonormal, Condon-Shortley phase, theta from +z, phi = atan2(y, x).
"""

from fractions import Fraction
import math

import numpy as np

__all__ = [
    "snapped_edges_sq", "offset_grids", "bin_masks", "bin_cell_counts",
    "sph_harm", "kernel_full", "kernel_projected", "a_coefficient",
    "a_full", "c_projected", "zeta3_full", "zeta4_full", "zeta3_projected",
    "zeta4_projected", "lambda_list", "wigner3j", "coupling",
    "normalization", "preprocess", "brute_a", "zeta4_full_entries", "kernel_full_bin",
    "lambda_list_odd", "zeta4_full_odd", "zeta3_full_entries", "zeta_projected_entries",
]


# ---------------------------------------------------------------- binning --

def snapped_edges_sq(edges):
    """Squared bin edges in float64; a square within 1e-9 (relative) of an
    integer is replaced by that integer so that the strict/loose inequalities
    of the Algorithm 1 mask (r_min < r <= r_max) act on exact integers."""
    e2 = np.asarray(edges, dtype=np.float64) ** 2
    out = e2.copy()
    for i, v in enumerate(e2):
        rv = round(v)
        if abs(v - rv) <= 1e-9 * max(v, 1.0):
            out[i] = float(rv)
    return out


def offset_grids(shape):
    """Minimum-image integer offsets, one array per axis, broadcast to `shape`
    (origin at index 0; the centred grid of Algorithms 1-2 after ifftshift)."""
    axes = [np.fft.fftfreq(n, 1.0 / n).round().astype(np.int64) for n in shape]
    return np.meshgrid(*axes, indexing="ij")


def bin_masks(shape, edges):
    """Boolean masks Theta^b over the offset grid, b = 0..nbins-1
    (Algorithm 1: r_min(b) < |r| <= r_max(b); Algorithm 2 in 2D)."""
    g = offset_grids(shape)
    r2 = sum(c * c for c in g).astype(np.float64)
    e2 = snapped_edges_sq(edges)
    return [(r2 > e2[b]) & (r2 <= e2[b + 1]) for b in range(len(edges) - 1)]


def bin_cell_counts(shape, edges):
    """N_cells in each bin, used by the bin volume of Eq. radial_binning /
    the bin area of Eq. proj_b_area (cell size 1)."""
    return np.array([int(m.sum()) for m in bin_masks(shape, edges)], dtype=np.int64)


# -------------------------------------------------------- basis functions --

def _reduced_legendre(l, m, t):
    """(-1)^m d^m P_l/dt^m (t), i.e. the associated Legendre function with the
    Condon-Shortley phase divided by (1 - t^2)^(m/2); m >= 0.  Standard
    three-term recurrence in l at fixed m."""
    p_mm = np.full_like(t, ((-1) ** m) * float(math.prod(range(1, 2 * m, 2))))
    if l == m:
        return p_mm
    p_m1 = (2 * m + 1) * t * p_mm
    if l == m + 1:
        return p_m1
    a, b = p_mm, p_m1
    for ll in range(m + 2, l + 1):
        a, b = b, ((2 * ll - 1) * t * b - (ll + m - 1) * a) / (ll - m)
    return b


def sph_harm(l, m, z, y, x):
    """Orthonormal Y_lm at Cartesian points (z, y, x), r > 0.

    Y_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta) e^{i m phi}; with
    sin(theta) e^{i phi} = (x + i y)/r this is N_lm Pred_l^m(z/r) ((x+iy)/r)^m.
    Negative m: Y_{l,-m} = (-1)^m conj(Y_lm)."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(x * x + y * y + z * z)
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4.0 * math.pi)
                     * math.factorial(l - am) / math.factorial(l + am))
    val = norm * _reduced_legendre(l, am, z / r) * ((x + 1j * y) / r) ** am
    if m < 0:
        val = ((-1) ** am) * np.conj(val)
    return val


def kernel_full(shape, edges, l, m):
    """K^b_lm(r) = Y*_lm(r_hat) Theta^b(|r|) for every bin b (Eq. almconv,
    Algorithm 1), shape [nbins, *shape], complex128."""
    z, y, x = offset_grids(shape)
    masks = bin_masks(shape, edges)
    out = np.zeros((len(masks),) + tuple(shape), dtype=np.complex128)
    for b, mk in enumerate(masks):
        # Y is evaluated only on the cells of the bin (r > 0 there)
        out[b][mk] = np.conj(sph_harm(l, m, z[mk], y[mk], x[mk]))
    return out


def kernel_full_bin(shape, edges, l, m, b):
    """K^b_lm of kernel_full for the single bin b."""
    z, y, x = offset_grids(shape)
    mk = bin_masks(shape, edges)[b]
    out = np.zeros(tuple(shape), dtype=np.complex128)
    out[mk] = np.conj(sph_harm(l, m, z[mk], y[mk], x[mk]))
    return out


def kernel_projected(shape, edges, m):
    """K^b_m(rho) = e^{-i m phi} Theta^b(rho) (Eq. c_m def kernel), with
    e^{i m phi} = ((x + i y)/rho)^m (Algorithm 2 notes); negative m allowed."""
    y, x = offset_grids(shape)
    masks = bin_masks(shape, edges)
    out = np.zeros((len(masks),) + tuple(shape), dtype=np.complex128)
    for b, mk in enumerate(masks):
        xb, yb = x[mk].astype(np.float64), y[mk].astype(np.float64)
        u = (xb + 1j * yb) / np.sqrt(xb * xb + yb * yb)   # rho > 0 inside a bin
        out[b][mk] = np.conj(u) ** m if m >= 0 else u ** (-m)
    return out


# ------------------------------------------------------------- convolution --

def a_coefficient(delta, kernel, delta_hat=None):
    """a(x) = sum_r K(r) delta(x + r) on the periodic grid (Eq. almconv, a
    correlation per its footnote), evaluated as IFFT(FFT(delta) * G) with
    G(k) = sum_r K(r) e^{+2 pi i k.r/N} = N_g * IFFT(K)(k) (Algorithms 3-4).
    `delta_hat` may pass FFT(delta) when it is already at hand."""
    ng = delta.size
    dh = np.fft.fftn(delta) if delta_hat is None else delta_hat
    return np.fft.ifftn(dh * (np.fft.ifftn(kernel) * ng))


def brute_a(delta, kernel):
    """The same correlation by direct summation over the kernel support
    (no FFT); for tiny grids in tests."""
    out = np.zeros(delta.shape, dtype=np.complex128)
    for idx in zip(*np.nonzero(kernel)):
        # delta(x + r) = roll(delta, -r)(x)
        out += kernel[idx] * np.roll(delta, shift=[-int(i) for i in _signed(idx, delta.shape)],
                                     axis=tuple(range(delta.ndim)))
    return out


def _signed(idx, shape):
    return [i if i < n - i else i - n for i, n in zip(idx, shape)]


def a_full(delta, edges, l, m):
    """a^b_lm(x) for all bins b: [nbins, *shape] (Eq. almconv, Algorithm 3)."""
    return np.stack([a_coefficient(delta, k) for k in kernel_full(delta.shape, edges, l, m)])


def c_projected(delta, edges, m):
    """c^b_m(x) for all bins b (Eqs. discretize_cmb, c_m def kernel; Algorithm 4)."""
    return np.stack([a_coefficient(delta, k) for k in kernel_projected(delta.shape, edges, m)])


# ------------------------------------------------------------- preprocess --

def preprocess(field, subtract_mean=True):
    """delta <- delta - mean(delta) when requested (Sec. 4.1: the mean is
    subtracted for all measurements); returns (delta, N_gal) with
    N_gal = sum(delta + 1) (Eq. num_gals)."""
    d = np.asarray(field, dtype=np.float64)
    if subtract_mean:
        d = d - d.mean()
    return d, float((d + 1.0).sum())


# ---------------------------------------------------------------- 3PCF ----

def zeta3_full(delta, edges, lmax, return_imag=False):
    """zeta_l^{b1 b2} = (-1)^l/sqrt(2l+1) sum_x delta(x) sum_{m=-l..l}
    a^{b1}_lm(x) a^{b2}_lm(x)^*  (Eq. alm_to_zeta_clean summed over x as in
    Algorithm 5).  Shape [lmax+1, nb, nb]; negative m from their own kernels."""
    nb = len(edges) - 1
    z = np.zeros((lmax + 1, nb, nb), dtype=np.complex128)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            a = a_full(delta, edges, l, m).reshape(nb, -1)
            wa = a * delta.reshape(1, -1)
            z[l] += wa @ np.conj(a).T
        z[l] *= (-1) ** l / math.sqrt(2 * l + 1)
    return (z.real, z.imag) if return_imag else z.real


def zeta3_projected(delta, edges, mmax):
    """zeta_m^{b1 b2} = sum_x delta(x) c^{b1}_m(x) c^{b2}_m(x)^*
    (Eq. proj_3pcf_coeff without 1/(2 pi)^2, Algorithm 7), m = 0..mmax.
    Shape [mmax+1, nb, nb] complex."""
    nb = len(edges) - 1
    z = np.zeros((mmax + 1, nb, nb), dtype=np.complex128)
    for m in range(mmax + 1):
        c = c_projected(delta, edges, m).reshape(nb, -1)
        z[m] = (c * delta.reshape(1, -1)) @ np.conj(c).T
    return z


# ---------------------------------------------------------------- 4PCF ----

def lambda_list(lmax):
    """Even-parity Lambda = (l1, l2, l3) in the loop order of Algorithm 6:
    l1, l2 in 0..lmax, l3 from |l1-l2| to min(l1+l2, lmax), l1+l2+l3 even."""
    out = []
    for l1 in range(lmax + 1):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if (l1 + l2 + l3) % 2 == 0:
                    out.append((l1, l2, l3))
    return out


def lambda_list_odd(lmax):
    """Odd-parity Lambda = (l1, l2, l3): the loops of Algorithm 6 (l1, l2 in
    0..lmax, l3 from |l1-l2| to min(l1+l2, lmax)) keeping l1+l2+l3 odd, the
    Lambda with E(Lambda) = -1 in Eq. mu (Sec. 2.3)."""
    out = []
    for l1 in range(lmax + 1):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if (l1 + l2 + l3) % 2 == 1:
                    out.append((l1, l2, l3))
    return out


def wigner3j(j1, j2, j3, m1, m2, m3):
    """Wigner 3j symbol by the Racah formula in exact rational arithmetic,
    returned as float (the 3j of the coupling in Sec. 2.3)."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if not (abs(j1 - j2) <= j3 <= j1 + j2):
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = math.factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pre = tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(j1 + j2 - j3 - k) * f(j1 - m1 - k) * f(j2 + m2 - k)
               * f(j3 - j2 + m1 + k) * f(j3 - j1 - m2 + k))
        s += Fraction((-1) ** k, den)
    sign = (-1) ** (j1 - j2 - m3)
    # sqrt of an exact rational, then the exact rational sum
    return float(sign * s) * math.sqrt(pre.numerator / pre.denominator) if pre else 0.0


def coupling(l1, l2, l3, m1, m2, m3):
    """C^Lambda_M = (-1)^(l1+l2+l3) (l1 l2 l3; m1 m2 m3) (Sec. 2.3)."""
    return ((-1) ** (l1 + l2 + l3)) * wigner3j(l1, l2, l3, m1, m2, m3)


def _all_a(delta, edges, lmax):
    """a^b_lm for l <= lmax and every m in -l..l, flattened over x."""
    nb = len(edges) - 1
    return {(l, m): a_full(delta, edges, l, m).reshape(nb, -1)
            for l in range(lmax + 1) for m in range(-l, l + 1)}


def zeta4_full(delta, edges, lmax, return_imag=False):
    """zeta^{b1 b2 b3}_{l1 l2 l3} = Re sum_x delta(x) sum_M C^Lambda_M
    a^{b1}_{l1 m1} a^{b2}_{l2 m2} a^{b3}_{l3 m3}, m3 = -(m1 + m2), |m3| <= l3
    (Eq. mu of Sec. 2.3 with E(Lambda) = +1; even Lambda of Algorithm 6).
    Shape [nLambda, nb, nb, nb], all bin triples."""
    nb = len(edges) - 1
    lams = lambda_list(lmax)
    a = _all_a(delta, edges, lmax)
    d = delta.reshape(1, -1)
    z = np.zeros((len(lams), nb, nb, nb), dtype=np.complex128)
    for i, (l1, l2, l3) in enumerate(lams):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if abs(m3) > l3:
                    continue
                c = coupling(l1, l2, l3, m1, m2, m3)
                if c == 0.0:
                    continue
                z[i] += c * triple_sum(d, a[(l1, m1)], a[(l2, m2)], a[(l3, m3)])
    return (z.real, z.imag) if return_imag else z.real


def zeta4_full_odd(delta, edges, lmax, return_real=False):
    """Odd-parity 4PCF: zeta^{b1 b2 b3}_{l1 l2 l3} = sum_x delta(x) sum_M
    E(Lambda) C^Lambda_M a^{b1}_{l1 m1} a^{b2}_{l2 m2} a^{b3}_{l3 m3} with
    E(Lambda) = -1 (Eq. mu of Sec. 2.3), m3 = -(m1 + m2), |m3| <= l3, for the
    odd Lambda of lambda_list_odd.  For a real delta the terms M and -M are
    each other's negated conjugates, so the sum is imaginary: the coefficient is
    returned as its imaginary part (with return_real, also the real part, which
    is zero up to rounding).  Shape [nLambda_odd, nb, nb, nb], all bin triples."""
    nb = len(edges) - 1
    lams = lambda_list_odd(lmax)
    a = _all_a(delta, edges, lmax)
    d = delta.reshape(1, -1)
    z = np.zeros((len(lams), nb, nb, nb), dtype=np.complex128)
    for i, (l1, l2, l3) in enumerate(lams):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if abs(m3) > l3:
                    continue
                c = coupling(l1, l2, l3, m1, m2, m3)
                if c == 0.0:
                    continue
                z[i] -= c * triple_sum(d, a[(l1, m1)], a[(l2, m2)], a[(l3, m3)])  # E(Lambda) = -1
    return (z.imag, z.real) if return_real else z.imag


def triple_sum(d, a1, a2, a3):
    """sum_x d(x) a1[b1](x) a2[b2](x) a3[b3](x) for all bin triples: the
    summand of Eq. mu (Sec. 2.3) / Eq. proj_4pcf_coeff at one (M) term.
    a_i: [nb, X]; d: [1, X].  Returns [nb, nb, nb]."""
    nb = a1.shape[0]
    p = (d * a1)[:, None, :] * a2[None, :, :]
    return (p.reshape(nb * nb, -1) @ a3.T).reshape(nb, nb, nb)


def zeta4_full_entries(delta, edges, entries, odd=False, cache=None):
    """The same coefficients as zeta4_full (odd=False) or zeta4_full_odd
    (odd=True: E(Lambda) = -1, imaginary part) for a list of single entries
    ((l1, l2, l3), b1, b2, b3), each computed on its own from only the
    a-arrays it needs (for spot checks at sizes where the full tensor is out
    of reach).  `cache` may pass a dict that keeps a-arrays across calls."""
    cache = {} if cache is None else cache
    dh = np.fft.fftn(delta)

    def a_of(l, m, b):
        if (l, m, b) not in cache:
            k = kernel_full_bin(delta.shape, edges, l, m, b)
            cache[(l, m, b)] = a_coefficient(delta, k, dh).ravel()
        return cache[(l, m, b)]

    d = delta.ravel()
    out = []
    for (l1, l2, l3), b1, b2, b3 in entries:
        s = 0.0 + 0.0j
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if abs(m3) > l3:
                    continue
                c = coupling(l1, l2, l3, m1, m2, m3)
                if c == 0.0:
                    continue
                s += c * np.sum(d * a_of(l1, m1, b1) * a_of(l2, m2, b2) * a_of(l3, m3, b3))
        out.append(-s.imag if odd else s.real)
    return np.array(out)


def zeta3_full_entries(delta, edges, entries):
    """zeta_l^{b1 b2} of zeta3_full for a list of single entries (l, b1, b2),
    each from the a-arrays of its two bins at m = 0..l only: for a real delta
    a_{l,-m} = (-1)^m conj(a_lm) (Sec. 2.1), so the terms m and -m of
    Eq. alm_to_zeta_clean are complex conjugates and sum to twice the real part.
    The arrays of one m are made, used and dropped in turn, so that one entry
    holds at most two grid-sized arrays (spot checks at 512^3)."""
    dh = np.fft.fftn(delta)
    d = delta.ravel()
    out = []
    for l, b1, b2 in entries:
        s = 0.0
        for m in range(l + 1):
            a1 = a_coefficient(delta, kernel_full_bin(delta.shape, edges, l, m, b1), dh).ravel()
            a2 = a1 if b2 == b1 else a_coefficient(delta, kernel_full_bin(delta.shape, edges, l, m, b2), dh).ravel()
            t = np.sum(d * a1 * np.conj(a2))
            s += t.real if m == 0 else 2.0 * t.real
            del a1, a2
        out.append(s * (-1) ** l / math.sqrt(2 * l + 1))
    return np.array(out)


def zeta_projected_entries(delta, edges, entries3, entries4):
    """Single entries of zeta3_projected, (m, b1, b2), and of zeta4_projected,
    ((m1, m2), b1, b2, b3) with |m1 + m2| <= mmax, each from the c arrays of the
    m values it needs (every m from its own kernel, as in c_projected); for spot
    checks of large batches.  Returns two complex arrays."""
    cache = {}

    def c_of(m):
        if m not in cache:
            cache[m] = c_projected(delta, edges, m).reshape(len(edges) - 1, -1)
        return cache[m]

    d = delta.ravel()
    z3 = [np.sum(d * c_of(m)[b1] * np.conj(c_of(m)[b2])) for m, b1, b2 in entries3]
    z4 = [np.sum(d * c_of(m1)[b1] * c_of(m2)[b2] * c_of(-(m1 + m2))[b3]) for (m1, m2), b1, b2, b3 in entries4]
    return np.array(z3, dtype=np.complex128), np.array(z4, dtype=np.complex128)


def zeta4_projected(delta, edges, mmax):
    """zeta^{b1 b2 b3}_{m1 m2} = sum_x delta c^{b1}_{m1} c^{b2}_{m2}
    c^{b3}_{-(m1+m2)} (Eq. proj_4pcf_coeff; Algorithm 8 with c_{-m} from its
    own kernel and |m3| <= mmax kept).  Shape [2mmax+1, 2mmax+1, nb, nb, nb],
    index m + mmax; entries with |m1 + m2| > mmax are 0."""
    nb = len(edges) - 1
    c = {m: c_projected(delta, edges, m).reshape(nb, -1) for m in range(-mmax, mmax + 1)}
    d = delta.reshape(1, -1)
    w = 2 * mmax + 1
    z = np.zeros((w, w, nb, nb, nb), dtype=np.complex128)
    for m1 in range(-mmax, mmax + 1):
        for m2 in range(-mmax, mmax + 1):
            m3 = -(m1 + m2)
            if abs(m3) > mmax:
                continue
            z[m1 + mmax, m2 + mmax] = triple_sum(d, c[m1], c[m2], c[m3])
    return z


# ---------------------------------------------------------- normalisation --

def normalization(shape, edges, n_gal, order, bins):
    """N = N_gal prod_{i=1}^{order-1} nbar V_bin,i with nbar = N_gal / L^d,
    L = N (cell units) and V_bin = cell count (Eqs. radial_binning, num_gals,
    and the normalisation coefficient of Sec. 2.5; areas in 2D, Eq. proj_norm).
    `bins` lists the order-1 bin indices."""
    counts = bin_cell_counts(shape, edges)
    nbar = n_gal / float(np.prod(shape))
    out = n_gal
    for b in bins:
        out *= nbar * counts[b]
    return out
