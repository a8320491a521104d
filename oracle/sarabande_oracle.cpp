// FP64 C++ oracle of the SARABANDE 3/4PCF hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this file;
// only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
// reference legs load it (through oracle/cpp.py).  It shares no code with the
// CUDA path.
//
// A plain, slow restatement of the definitions of Sunseri et al. 2022 (arXiv
// 2210.10206) in double / std::complex<double>, with its own FFT (iterative
// radix-2 for powers of two, a direct O(N^2) DFT per axis otherwise) and OpenMP
// over independent lines and grid points.  The conventions are those of
// oracle/sarabande_oracle.py:
//  * offsets are minimum-image integer vectors, origin at index 0; C-order
//    index (i, j, k) <-> (z, y, x), 2D (i, j) <-> (y, x); box side N, cell 1;
//  * bin b holds |r|^2 in (e_b^2, e_{b+1}^2] (Algorithm 1 mask), squared edges
//    snapped to the nearest integer within 1e-9 relative;
//  * a(x) = sum_r K(r) delta(x + r), a correlation (Eq. almconv and its
//    footnote), K = conj(Y_lm) Theta_b in 3D, e^{-i m phi} Theta_b in 2D, 0/1
//    masks; negative m from their own kernels;
//  * outputs are raw sums over grid points (Algorithms 5-8); the full 3PCF has
//    (-1)^l / sqrt(2l+1) (Eq. alm_to_zeta_clean); the projected 3PCF no
//    1/(2 pi)^2; the full 4PCF sums every M with |m3| <= l3 and the coupling
//    (-1)^(l1+l2+l3) (3j) of Sec. 2.3, E(Lambda) = +1 (even, real part) or -1
//    (odd, imaginary part); the projected 4PCF keeps every (m1, m2) with
//    |m1|, |m2|, |m1 + m2| <= mmax (Eq. proj_4pcf_coeff), zero elsewhere.
// Y_lm: orthonormal, Condon-Shortley phase, theta from +z, phi = atan2(y, x).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846264338327950288;

// ------------------------------------------------------------------ FFT ----
// One length-n transform of a strided line: X_k = sum_j x_j exp(sign 2 pi i j k / n).
bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

void fft_line(cd* buf, int64_t n, int sign, const std::vector<cd>& w) {
  // w[j] = exp(sign 2 pi i j / n), j < n
  if (is_pow2(n)) {
    // bit-reversal permutation, then log2(n) butterfly stages
    for (int64_t i = 1, j = 0; i < n; ++i) {
      int64_t bit = n >> 1;
      for (; j & bit; bit >>= 1) j ^= bit;
      j ^= bit;
      if (i < j) std::swap(buf[i], buf[j]);
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
      const int64_t step = n / len;
      for (int64_t s = 0; s < n; s += len)
        for (int64_t k = 0; k < len / 2; ++k) {
          const cd u = buf[s + k], v = buf[s + k + len / 2] * w[k * step];
          buf[s + k] = u + v;
          buf[s + k + len / 2] = u - v;
        }
    }
  } else {
    std::vector<cd> out(n);
    for (int64_t k = 0; k < n; ++k) {
      cd acc = 0.0;
      for (int64_t j = 0; j < n; ++j) acc += buf[j] * w[(j * k) % n];
      out[k] = acc;
    }
    for (int64_t k = 0; k < n; ++k) buf[k] = out[k];
  }
}

// In-place unnormalised DFT of a C-order array of `dims` (1..3 axes).
void fftn(cd* a, const std::vector<int64_t>& dims, int sign) {
  int64_t total = 1;
  for (int64_t d : dims) total *= d;
  for (size_t ax = 0; ax < dims.size(); ++ax) {
    const int64_t n = dims[ax];
    int64_t inner = 1;
    for (size_t k = ax + 1; k < dims.size(); ++k) inner *= dims[k];
    const int64_t outer = total / (n * inner);
    std::vector<cd> w(n);
    for (int64_t j = 0; j < n; ++j) w[j] = std::polar(1.0, sign * 2.0 * kPi * (double)j / (double)n);
#pragma omp parallel
    {
      std::vector<cd> line(n);
#pragma omp for schedule(static)
      for (int64_t t = 0; t < outer * inner; ++t) {
        const int64_t o = t / inner, i = t % inner;
        cd* base = a + o * n * inner + i;
        for (int64_t j = 0; j < n; ++j) line[j] = base[j * inner];
        fft_line(line.data(), n, sign, w);
        for (int64_t j = 0; j < n; ++j) base[j * inner] = line[j];
      }
    }
  }
}

// ------------------------------------------------------------- binning ----
std::vector<double> snapped_sq(const double* edges, int nb) {
  std::vector<double> e2(nb + 1);
  for (int i = 0; i <= nb; ++i) {
    double v = edges[i] * edges[i];
    const double r = std::round(v);
    if (std::fabs(v - r) <= 1e-9 * std::max(v, 1.0)) v = r;
    e2[i] = v;
  }
  return e2;
}

// bin of an integer squared length, or -1 (Algorithm 1: r_min < r <= r_max)
int bin_of(double r2, const std::vector<double>& e2) {
  const int nb = (int)e2.size() - 1;
  for (int b = 0; b < nb; ++b)
    if (r2 > e2[b] && r2 <= e2[b + 1]) return b;
  return -1;
}

int64_t signed_offset(int64_t i, int64_t n) { return i < n - i ? i : i - n; }

// ---------------------------------------------------- spherical harmonics --
// Y_lm(r_hat) at a non-zero integer offset (x, y, z), any m in -l..l.
cd ylm(int l, int m, double x, double y, double z) {
  const int am = std::abs(m);
  const double r = std::sqrt(x * x + y * y + z * z);
  const double t = z / r;
  // associated Legendre with the Condon-Shortley phase, divided by
  // (1 - t^2)^(am/2): start at P_am^am, then the recurrence in l
  double pmm = 1.0;
  for (int k = 1; k <= am; ++k) pmm *= -(2.0 * k - 1.0);
  double p = pmm;
  if (l > am) {
    double pm1 = (2.0 * am + 1.0) * t * pmm;
    double pl2 = pmm, pl1 = pm1;
    for (int ll = am + 2; ll <= l; ++ll) {
      const double pn = ((2.0 * ll - 1.0) * t * pl1 - (ll + am - 1.0) * pl2) / (double)(ll - am);
      pl2 = pl1;
      pl1 = pn;
    }
    p = pl1;
  }
  // normalisation sqrt((2l+1)/(4 pi) (l-am)!/(l+am)!)
  double ratio = 1.0;
  for (int k = l - am + 1; k <= l + am; ++k) ratio /= (double)k;
  const double norm = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio);
  // sin^am(theta) e^{i am phi} = ((x + i y) / r)^am
  cd e = 1.0;
  const cd u(x / r, y / r);
  for (int k = 0; k < am; ++k) e *= u;
  cd v = norm * p * e;
  if (m < 0) v = ((am & 1) ? -1.0 : 1.0) * std::conj(v);
  return v;
}

// --------------------------------------------------------------- Wigner 3j --
// Racah's single-sum formula; factorials from a long double table (l <= 10
// keeps every factorial below 32!).
struct FactTable {
  long double t[64];
  FactTable() {
    t[0] = 1.0L;
    for (int i = 1; i < 64; ++i) t[i] = t[i - 1] * (long double)i;
  }
};

long double fact(int n) {
  static const FactTable table;  // initialised once, thread-safe
  return table.t[n];
}

double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  const long double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const long double root = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                                     fact(j3 + m3) * fact(j3 - m3));
  long double sum = 0.0L;
  for (int k = 0; k <= j1 + j2 + j3; ++k) {
    const int d[6] = {k, j1 + j2 - j3 - k, j1 - m1 - k, j2 + m2 - k, j3 - j2 + m1 + k, j3 - j1 - m2 + k};
    bool ok = true;
    for (int v : d) ok = ok && v >= 0;
    if (!ok) continue;
    long double den = 1.0L;
    for (int v : d) den *= fact(v);
    sum += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  const int ph = j1 - j2 - m3;
  return (double)((((ph % 2) + 2) % 2 ? -1.0L : 1.0L) * root * sum);
}

// ----------------------------------------------------------- coefficients --
struct Grid {
  int dim;
  int64_t n, ng;
  std::vector<int64_t> dims;
};

Grid make_grid(int dim, int64_t n) {
  Grid g;
  g.dim = dim;
  g.n = n;
  g.dims.assign(dim, n);
  g.ng = 1;
  for (int i = 0; i < dim; ++i) g.ng *= n;
  return g;
}

// offset (x, y, z) of flat index i (z = 0 in 2D)
void offset_of(const Grid& g, int64_t i, double& x, double& y, double& z) {
  if (g.dim == 3) {
    z = (double)signed_offset(i / (g.n * g.n), g.n);
    y = (double)signed_offset((i / g.n) % g.n, g.n);
    x = (double)signed_offset(i % g.n, g.n);
  } else {
    z = 0.0;
    y = (double)signed_offset(i / g.n, g.n);
    x = (double)signed_offset(i % g.n, g.n);
  }
}

// The binned kernel of one (l, m, b) (3D) or (m, b) (2D, l ignored):
// conj(Y_lm) Theta_b, or e^{-i m phi} Theta_b with e^{i phi} = (x + i y)/rho.
std::vector<cd> kernel(const Grid& g, const std::vector<double>& e2, int l, int m, int b) {
  std::vector<cd> k(g.ng, cd(0.0, 0.0));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < g.ng; ++i) {
    double x, y, z;
    offset_of(g, i, x, y, z);
    const double r2 = x * x + y * y + z * z;
    if (bin_of(r2, e2) != b) continue;
    if (g.dim == 3) {
      k[i] = std::conj(ylm(l, m, x, y, z));
    } else {
      const double rho = std::sqrt(r2);
      const cd u(x / rho, y / rho);
      cd v = 1.0;
      const int am = std::abs(m);
      for (int q = 0; q < am; ++q) v *= u;
      k[i] = m >= 0 ? std::conj(v) : v;  // e^{-i m phi}
    }
  }
  return k;
}

// a(x) = sum_r K(r) delta(x + r) = FFT_+(dhat * G) / N_g with G = FFT_+(K)
// and dhat = FFT_-(delta).
std::vector<cd> coefficient(const Grid& g, const std::vector<cd>& dhat, std::vector<cd> k) {
  fftn(k.data(), g.dims, +1);
  const double inv = 1.0 / (double)g.ng;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < g.ng; ++i) k[i] *= dhat[i] * inv;
  fftn(k.data(), g.dims, +1);
  return k;
}

std::vector<cd> delta_hat(const Grid& g, const double* delta) {
  std::vector<cd> d(g.ng);
  for (int64_t i = 0; i < g.ng; ++i) d[i] = delta[i];
  fftn(d.data(), g.dims, -1);
  return d;
}

// sum_x w(x) p(x) for complex arrays, in per-thread partial sums
cd weighted_sum(int64_t ng, const double* w, const cd* a, const cd* b, const cd* c) {
  double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
  for (int64_t i = 0; i < ng; ++i) {
    cd v = w[i] * a[i] * b[i];
    if (c) v *= c[i];
    re += v.real();
    im += v.imag();
  }
  return cd(re, im);
}

}  // namespace

extern "C" {

// Unnormalised in-place DFT of a complex C-order array (interleaved re, im):
// X_k = sum_j x_j exp(sign 2 pi i j.k / N) over `ndim` axes of sizes dims.
int oc_fftn(double* data, int ndim, const int64_t* dims, int sign) {
  if (!data || ndim < 1 || ndim > 3 || (sign != 1 && sign != -1)) return -1;
  std::vector<int64_t> d(dims, dims + ndim);
  fftn(reinterpret_cast<cd*>(data), d, sign);
  return 0;
}

// Binned coefficient a^b_lm(x) (3D, Eq. almconv) or c^b_m(x) (2D, dim 2, l
// ignored) of a real field; out: N^dim complex (interleaved).
int oc_coefficient(const double* delta, int dim, int64_t n, const double* edges, int nb, int l, int m, int b,
                   double* out) {
  if (!delta || !edges || !out || (dim != 2 && dim != 3) || n < 2 || nb < 1 || b < 0 || b >= nb) return -1;
  const Grid g = make_grid(dim, n);
  const std::vector<double> e2 = snapped_sq(edges, nb);
  const std::vector<cd> dh = delta_hat(g, delta);
  const std::vector<cd> a = coefficient(g, dh, kernel(g, e2, l, m, b));
  std::memcpy(out, a.data(), sizeof(cd) * g.ng);
  return 0;
}

// Full 3PCF zeta_l^{b1 b2} = (-1)^l/sqrt(2l+1) sum_x delta sum_m a^{b1}_lm
// conj(a^{b2}_lm) (Eq. alm_to_zeta_clean, Algorithm 5), every m from its own
// kernel; streamed over (l, m).  out: [lmax+1][nb][nb].
int oc_zeta3_full(const double* delta, int64_t n, const double* edges, int nb, int lmax, double* out) {
  if (!delta || !edges || !out || n < 2 || nb < 1 || lmax < 0) return -1;
  const Grid g = make_grid(3, n);
  const std::vector<double> e2 = snapped_sq(edges, nb);
  const std::vector<cd> dh = delta_hat(g, delta);
  for (int l = 0; l <= lmax; ++l) {
    std::vector<cd> acc((size_t)nb * nb, cd(0.0, 0.0));
    for (int m = -l; m <= l; ++m) {
      std::vector<std::vector<cd>> a(nb);
      for (int b = 0; b < nb; ++b) a[b] = coefficient(g, dh, kernel(g, e2, l, m, b));
      for (int b1 = 0; b1 < nb; ++b1)
        for (int b2 = 0; b2 < nb; ++b2) {
          std::vector<cd> c2(g.ng);
          for (int64_t i = 0; i < g.ng; ++i) c2[i] = std::conj(a[b2][i]);
          acc[(size_t)b1 * nb + b2] += weighted_sum(g.ng, delta, a[b1].data(), c2.data(), nullptr);
        }
    }
    const double pre = ((l & 1) ? -1.0 : 1.0) / std::sqrt(2.0 * l + 1.0);
    for (int i = 0; i < nb * nb; ++i) out[(size_t)l * nb * nb + i] = pre * acc[i].real();
  }
  return 0;
}

// Projected 3PCF zeta_m^{b1 b2} = sum_x delta c^{b1}_m conj(c^{b2}_m)
// (Eq. proj_3pcf_coeff without 1/(2 pi)^2, Algorithm 7), m = 0..mmax.
// out: [mmax+1][nb][nb][2].
int oc_zeta3_projected(const double* delta, int64_t n, const double* edges, int nb, int mmax, double* out) {
  if (!delta || !edges || !out || n < 2 || nb < 1 || mmax < 0) return -1;
  const Grid g = make_grid(2, n);
  const std::vector<double> e2 = snapped_sq(edges, nb);
  const std::vector<cd> dh = delta_hat(g, delta);
  for (int m = 0; m <= mmax; ++m) {
    std::vector<std::vector<cd>> c(nb);
    for (int b = 0; b < nb; ++b) c[b] = coefficient(g, dh, kernel(g, e2, 0, m, b));
    for (int b1 = 0; b1 < nb; ++b1)
      for (int b2 = 0; b2 < nb; ++b2) {
        std::vector<cd> c2(g.ng);
        for (int64_t i = 0; i < g.ng; ++i) c2[i] = std::conj(c[b2][i]);
        const cd z = weighted_sum(g.ng, delta, c[b1].data(), c2.data(), nullptr);
        double* o = out + (((size_t)m * nb + b1) * nb + b2) * 2;
        o[0] = z.real();
        o[1] = z.imag();
      }
  }
  return 0;
}

// Number of Lambda = (l1, l2, l3) of Algorithm 6's loops (l1, l2 in 0..lmax,
// l3 from |l1 - l2| to min(l1 + l2, lmax)) with l1 + l2 + l3 of the given
// parity (0 even, 1 odd); list (3 ints each) if not NULL.
int oc_lambda_list(int lmax, int parity, int* list) {
  int k = 0;
  for (int l1 = 0; l1 <= lmax; ++l1)
    for (int l2 = 0; l2 <= lmax; ++l2)
      for (int l3 = std::abs(l1 - l2); l3 <= std::min(l1 + l2, lmax); ++l3)
        if ((l1 + l2 + l3) % 2 == parity) {
          if (list) {
            list[3 * k] = l1;
            list[3 * k + 1] = l2;
            list[3 * k + 2] = l3;
          }
          ++k;
        }
  return k;
}

double oc_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) { return wigner3j(j1, j2, j3, m1, m2, m3); }

// The combination step of the full 4PCF (Eq. mu, Sec. 2.3; Algorithm 6) from
// given coefficient arrays: for each Lambda of the given parity
// zeta^{b1 b2 b3} = sum_x delta sum_M E C^Lambda_M a^{b1}_{l1 m1} a^{b2}_{l2 m2}
// a^{b3}_{l3 m3}, m3 = -(m1 + m2), |m3| <= l3, C = (-1)^(l1+l2+l3) (3j);
// even (odd = 0, E = +1): the real part; odd (odd = 1, E = -1): the imaginary
// part; every bin triple.  a: [(lmax+1)^2][nb][npts] complex (interleaved),
// (l, m) at index l*l + l + m, m = -l..l; delta: [npts].
// out: [nLambda][nb][nb][nb].
int oc_zeta4_combine(const double* delta, const double* a_interleaved, int64_t npts, int nb, int lmax, int odd,
                     double* out) {
  if (!delta || !a_interleaved || !out || npts < 1 || nb < 1 || lmax < 0 || (odd != 0 && odd != 1)) return -1;
  const cd* a = reinterpret_cast<const cd*>(a_interleaved);
  const int nl = oc_lambda_list(lmax, odd, nullptr);
  std::vector<int> lams(3 * (size_t)nl);
  oc_lambda_list(lmax, odd, lams.data());
  // the (Lambda, M) terms with a non-zero coupling
  struct Term {
    int li;
    size_t i1, i2, i3;
    double c;
  };
  std::vector<Term> terms;
  for (int li = 0; li < nl; ++li) {
    const int l1 = lams[3 * li], l2 = lams[3 * li + 1], l3 = lams[3 * li + 2];
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int m2 = -l2; m2 <= l2; ++m2) {
        const int m3 = -(m1 + m2);
        if (std::abs(m3) > l3) continue;
        const double c = (((l1 + l2 + l3) & 1) ? -1.0 : 1.0) * wigner3j(l1, l2, l3, m1, m2, m3);
        if (c == 0.0) continue;
        terms.push_back({li, (size_t)(l1 * l1 + l1 + m1) * nb * npts, (size_t)(l2 * l2 + l2 + m2) * nb * npts,
                         (size_t)(l3 * l3 + l3 + m3) * nb * npts, c});
      }
  }
  const size_t nb3 = (size_t)nb * nb * nb;
  std::vector<cd> acc((size_t)nl * nb3, cd(0.0, 0.0));
#pragma omp parallel
  {
    // per-thread sums over its points, added together at the end
    std::vector<cd> part((size_t)nl * nb3, cd(0.0, 0.0));
    std::vector<cd> p12((size_t)nb * nb);
#pragma omp for schedule(static)
    for (int64_t x = 0; x < npts; ++x) {
      const double w = delta[x];
      for (const Term& t : terms) {
        for (int b1 = 0; b1 < nb; ++b1) {
          const cd p1 = t.c * w * a[t.i1 + (size_t)b1 * npts + x];
          for (int b2 = 0; b2 < nb; ++b2) p12[(size_t)b1 * nb + b2] = p1 * a[t.i2 + (size_t)b2 * npts + x];
        }
        cd* o = part.data() + (size_t)t.li * nb3;
        for (int b12 = 0; b12 < nb * nb; ++b12)
          for (int b3 = 0; b3 < nb; ++b3) o[(size_t)b12 * nb + b3] += p12[b12] * a[t.i3 + (size_t)b3 * npts + x];
      }
    }
#pragma omp critical
    for (size_t i = 0; i < part.size(); ++i) acc[i] += part[i];
  }
  for (size_t i = 0; i < acc.size(); ++i) out[i] = odd ? -acc[i].imag() : acc[i].real();
  return 0;
}

// Full 4PCF of a field: every a^b_lm (every m, its own kernel) by FFT, then
// the combination above over all grid points.  out: [nLambda][nb][nb][nb].
int oc_zeta4_full(const double* delta, int64_t n, const double* edges, int nb, int lmax, int odd, double* out) {
  if (!delta || !edges || !out || n < 2 || nb < 1 || lmax < 0 || (odd != 0 && odd != 1)) return -1;
  const Grid g = make_grid(3, n);
  const std::vector<double> e2 = snapped_sq(edges, nb);
  const std::vector<cd> dh = delta_hat(g, delta);
  const int nlm = (lmax + 1) * (lmax + 1);
  std::vector<cd> a((size_t)nlm * nb * g.ng);
  for (int l = 0; l <= lmax; ++l)
    for (int m = -l; m <= l; ++m)
      for (int b = 0; b < nb; ++b) {
        const std::vector<cd> c = coefficient(g, dh, kernel(g, e2, l, m, b));
        std::memcpy(a.data() + ((size_t)(l * l + l + m) * nb + b) * g.ng, c.data(), sizeof(cd) * g.ng);
      }
  return oc_zeta4_combine(delta, reinterpret_cast<const double*>(a.data()), g.ng, nb, lmax, odd, out);
}

// Projected 4PCF zeta^{b1 b2 b3}_{m1 m2} = sum_x delta c^{b1}_{m1} c^{b2}_{m2}
// c^{b3}_{-(m1+m2)} (Eq. proj_4pcf_coeff, Algorithm 8 with c_{-m} from its own
// kernel), |m1|, |m2|, |m1 + m2| <= mmax, zero elsewhere.
// out: [2mmax+1][2mmax+1][nb][nb][nb][2], index m + mmax.
int oc_zeta4_projected(const double* delta, int64_t n, const double* edges, int nb, int mmax, double* out) {
  if (!delta || !edges || !out || n < 2 || nb < 1 || mmax < 0) return -1;
  const Grid g = make_grid(2, n);
  const std::vector<double> e2 = snapped_sq(edges, nb);
  const std::vector<cd> dh = delta_hat(g, delta);
  const int w = 2 * mmax + 1;
  std::vector<std::vector<cd>> c((size_t)w * nb);
  for (int m = -mmax; m <= mmax; ++m)
    for (int b = 0; b < nb; ++b) c[(size_t)(m + mmax) * nb + b] = coefficient(g, dh, kernel(g, e2, 0, m, b));
  const size_t nb3 = (size_t)nb * nb * nb;
  std::memset(out, 0, sizeof(double) * 2 * nb3 * w * w);
  for (int m1 = -mmax; m1 <= mmax; ++m1)
    for (int m2 = -mmax; m2 <= mmax; ++m2) {
      const int m3 = -(m1 + m2);
      if (std::abs(m3) > mmax) continue;
      double* o = out + ((size_t)(m1 + mmax) * w + (m2 + mmax)) * nb3 * 2;
      for (int b1 = 0; b1 < nb; ++b1)
        for (int b2 = 0; b2 < nb; ++b2)
          for (int b3 = 0; b3 < nb; ++b3) {
            const cd z = weighted_sum(g.ng, delta, c[(size_t)(m1 + mmax) * nb + b1].data(),
                                      c[(size_t)(m2 + mmax) * nb + b2].data(), c[(size_t)(m3 + mmax) * nb + b3].data());
            o[(((size_t)b1 * nb + b2) * nb + b3) * 2] = z.real();
            o[(((size_t)b1 * nb + b2) * nb + b3) * 2 + 1] = z.imag();
          }
    }
  return 0;
}

// Threads the OpenMP loops use (1 without OpenMP).
int oc_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
