// Kernel generation fused with the forward FFT, and the spectral product fused
// between the last forward and the first inverse pass, for 3D groups whose
// kernel spectra are not cached (the kernel spectra of every (l, m) do not fit
// in HBM, e.g. the 512^3 l <= 10 3PCF): per (l, m) group of nb bins,
//
//   pass A (x, contiguous): K^b_lm = conj(Y_lm) Theta_b (Algorithm 1) is
//       evaluated in FP64 on the fly for the x-lines (z, y) that meet the
//       kernel support (y^2 + z^2 <= e_nb^2) and transformed along x; no other
//       line is touched (they are zero);
//   pass B (y, strided): the planes |z| <= e_nb, reading only the entries of
//       lines that pass A wrote;
//   pass C (z, strided): per column, the forward transform along z of every
//       bin's kernel (reading only the planes pass B wrote), the product with
//       delta-hat (one read of delta-hat per group, kept in shared memory for
//       all bins), and the inverse transform along z (Algorithms 3-4: the
//       convolution a = IFFT(delta-hat x FFT(K)), in the correlation convention
//       of Eq. almconv: G(k) = sum_r K(r) e^{+i k.r} / N_g);
//   then the inverse y and x passes of sbg_fft.cu.
//
// Compared with generating every spectrum in HBM (memset, kgen3d, three
// forward passes, three inverse passes) this moves no zero lines and never
// writes or reads the kernel spectra G.  Real m = 0 arrays are packed two per
// inverse transform as in the other path (delta-hat (G_2j + i G_2j+1)).
#include "sbg_fft_core.cuh"
#include "sbg_kernels.cuh"

namespace sbg {

namespace {

__device__ __forceinline__ int min_img(int i, int n) { return i < n - i ? i : i - n; }

// conj(Y_lm(r_hat)) norm scale at the integer offset (x, y, z), r2 = |r|^2 > 0,
// in FP64: the reduced associated Legendre recurrence times ((x + i y)/r)^m
__device__ __noinline__ float2 kernel_value(int l, int m, double norm_scale, int x, int y, int z, double r2) {
  const double r = sqrt(r2);
  const double t = z / r;
  double pmm = (m & 1) ? -1.0 : 1.0;
  for (int k = 1; k < 2 * m; k += 2) pmm *= k;
  double p = pmm;
  if (l > m) {
    double a = pmm, bb = (2 * m + 1) * t * pmm;
    for (int ll = m + 2; ll <= l; ++ll) {
      const double c = ((2 * ll - 1) * t * bb - (ll + m - 1) * a) / (ll - m);
      a = bb;
      bb = c;
    }
    p = bb;
  }
  const double ur = x / r, ui = y / r;
  double er = 1.0, ei = 0.0;
  for (int k = 0; k < m; ++k) {
    const double tr = er * ur - ei * ui;
    ei = er * ui + ei * ur;
    er = tr;
  }
  const double s = norm_scale * p;
  return make_float2((float)(s * er), (float)(-s * ei));
}

// One transform (sign +1) of TL lines of N points, T = min(R1, R2) threads per
// line, in the two steps of sbg_fft.cu: thread (line l, index j) loads points
// n = n1 + R1 n2 through ld(n), exchanges through `ex`, and stores k = k2 + R2 k1
// through st(k, value).  STRIDED: lines adjacent in the thread index (j = t / TL),
// otherwise points adjacent (j = t % T).  Every thread of the CTA calls it.
template <int N, int TL, bool STRIDED, class LD, class ST>
__device__ __forceinline__ void line_fft(float2* ex, const float2* __restrict__ tw, int l, int j, LD ld, ST st) {
  constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2, T = R1 < R2 ? R1 : R2;
  constexpr int R2S = STRIDED ? R2 : R2 + 1, LS = R1 * R2S + 1;
  auto sidx = [&](int n1, int k2) { return STRIDED ? (n1 * R2 + k2) * TL + l : l * LS + n1 * R2S + k2; };
#pragma unroll
  for (int q = 0; q < R1 / T; ++q) {
    const int n1 = j + T * q;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = ld(n1 + R1 * n2);
    Dft<R2, 1>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) ex[sidx(n1, k2)] = k2 ? cmul(v[k2], __ldg(tw + ((n1 * k2) & (N - 1)))) : v[k2];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < R2 / T; ++q) {
    const int k2 = j + T * q;
    float2 u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) u[n1] = ex[sidx(n1, k2)];
    Dft<R1, 1>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) st(k2 + R2 * k1, u[k1]);
  }
}

template <int N> struct FusedGeo {
  static constexpr int T = Plan<N>::R1 < Plan<N>::R2 ? Plan<N>::R1 : Plan<N>::R2;
  static constexpr int TLA = N <= 32 ? 8 : 256 / T;  // pass A: x-lines per CTA
  static constexpr int TLB = N >= 16 ? 16 : 8;       // pass B: lines per CTA (adjacent x; 128-byte runs)
  static constexpr int TLS = 8;                      // pass C: lines per CTA (adjacent x)
  static constexpr int LSA = Plan<N>::R1 * (Plan<N>::R2 + 1) + 1;
  static constexpr int SMEM_A = TLA * LSA * 8;
  static constexpr int SMEM_B = TLB * N * 8;
  static constexpr int SMEM_C = 3 * TLS * N * 8;     // exchange, kernel column, delta-hat column
  // pass C in place: each n1 row of the exchange layout is padded by 8 float2
  // (16 banks), so the warp's four n1 rows fall on distinct bank halves
  static constexpr int EXPAD = Plan<N>::R1 * 8;
};

// Pass A: the x-lines (z, y) of `lines` (row index z N + y), bin b = blockIdx.y:
// generate K^b_lm along x and transform; out[b][z][y][:] for those lines only.
template <int N>
__global__ void __launch_bounds__(FusedGeo<N>::TLA * FusedGeo<N>::T)
kgen_fft_x_kernel(int l, int m, double norm_scale, const double* __restrict__ e2, const int* __restrict__ lines,
                  int nlines, const float2* __restrict__ tw, float2* __restrict__ out, long long ng) {
  using G = FusedGeo<N>;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x, j = t % G::T, li = t / G::T;
  const int L = blockIdx.x * G::TLA + li;
  const bool valid = L < nlines;
  const int row = valid ? lines[L] : 0;
  const int z = min_img(row / N, N), y = min_img(row % N, N);
  const int yz2 = y * y + z * z;
  const int b = blockIdx.y;
  // Bin membership e2[b] < |r|^2 <= e2[b+1] in integer arithmetic: for an
  // integer |r|^2 it holds exactly when floor(e2[b]) < |r|^2 <= floor(e2[b+1])
  // (|r|^2 <= 3 (N/2)^2 fits an int).  Only the kernel values take FP64, whose
  // rate on this part is a small fraction of the FP32 rate.
  const int lo = (int)floor(e2[b]), hi = (int)floor(e2[b + 1]);
  float2* o = out + (long long)b * ng + (long long)row * N;
  line_fft<N, G::TLA, false>(
      ex, tw, li, j,
      [&](int n) {
        const int x = min_img(n, N);
        const int r2 = yz2 + x * x;
        return (valid && r2 > lo && r2 <= hi) ? kernel_value(l, m, norm_scale, x, y, z, (double)r2)
                                               : make_float2(0.f, 0.f);
      },
      [&](int k, float2 v) {
        if (valid) o[k] = v;
      });
}

// Pass B: y-lines of the planes |z| <= R (plane p = blockIdx.x / (N / TLB), z = p - R),
// TLB adjacent x per CTA, bin blockIdx.y, in place; entry (z, y) is read only if
// y^2 + z^2 <= e2nb (pass A wrote that x-line).
template <int N>
__global__ void __launch_bounds__(FusedGeo<N>::TLB * FusedGeo<N>::T)
disk_fft_y_kernel(double e2nb, int R, const float2* __restrict__ tw, float2* __restrict__ buf, long long ng) {
  using G = FusedGeo<N>;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x, j = t / G::TLB, li = t % G::TLB;
  const int xg = blockIdx.x % (N / G::TLB), p = blockIdx.x / (N / G::TLB);
  const int z = p - R, zi = z < 0 ? z + N : z;
  const int x = xg * G::TLB + li;
  float2* col = buf + (long long)blockIdx.y * ng + (long long)zi * N * N + x;
  // y^2 + z^2 <= e2nb for integers, in integer arithmetic (as in pass A)
  const int z2 = z * z, r2max = (int)floor(e2nb);
  line_fft<N, G::TLB, true>(
      ex, tw, li, j,
      [&](int n) {
        const int y = min_img(n, N);
        return (y * y + z2 <= r2max) ? col[(long long)n * N] : make_float2(0.f, 0.f);
      },
      [&](int k, float2 v) { col[(long long)k * N] = v; });
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Pass C: columns (y, x0 .. x0 + TL - 1) along z, every bin of the group: forward
// transform of the kernel column (planes |z| <= R only), times delta-hat, inverse
// transform, to out.  npack > 0: real arrays packed two per transform, output j
// holding delta-hat (G_2j + i G_2j+1) (G_2j+1 taken as 0 past npack).  The 2R + 1
// support rows of bin b + 1 are copied (cp.async) into one of two staging buffers
// while bin b is transformed.
template <int N>
__global__ void __launch_bounds__(FusedGeo<N>::TLS * FusedGeo<N>::T)
fused_fft_z_kernel(int R, int nb, int npack, const float2* __restrict__ tw, const float2* __restrict__ kin,
                   const float2* __restrict__ dhat, float2* __restrict__ out, long long ng) {
  using G = FusedGeo<N>;
  constexpr int TL = G::TLS;
  extern __shared__ float2 smem[];
  float2* ex = smem;
  float2* C = smem + TL * N;   // the kernel column's spectrum, [k][line]
  float2* D = C + TL * N;      // delta-hat, [k][line]
  float2* stg = D + TL * N;    // two staging buffers of the support rows, [2][2R + 1][line]
  const int rows = 2 * R + 1;
  const int t = threadIdx.x, j = t / TL, li = t % TL;
  const int xg = blockIdx.x % (N / TL), yy = blockIdx.x / (N / TL);
  const long long cbase = (long long)yy * N + (long long)xg * TL;  // (0, y, x0)
  // rows z = -R .. R of bin b into staging buffer b & 1 (TL x 8 bytes = TL / 2 chunks per row)
  auto prefetch = [&](int b) {
    float2* dst = stg + (b & 1) * rows * TL;
    const float2* src = kin + (long long)b * ng + cbase;
    for (int c = t; c < rows * (TL / 2); c += blockDim.x) {
      const int r = c / (TL / 2), q = c % (TL / 2);
      const int z = r - R, zi = z < 0 ? z + N : z;
      cp_async16(dst + r * TL + 2 * q, src + (long long)zi * N * N + 2 * q);
    }
    cp_async_commit();
  };
  prefetch(0);
  for (int i = t; i < N * TL; i += blockDim.x) {
    const int k = i / TL, c = i % TL;
    D[i] = __ldg(dhat + (long long)k * N * N + cbase + c);
  }
  for (int b = 0; b < nb; ++b) {
    const int o = npack ? b / 2 : b;
    const int s = npack ? b % 2 : 0;
    if (b + 1 < nb) prefetch(b + 1);
    else cp_async_commit();  // an empty group keeps the wait count uniform
    cp_async_wait1();         // bin b's rows have landed (this thread's copies)
    __syncthreads();          // ... everyone's; the exchange buffer and C are free
    const float2* sb = stg + (b & 1) * rows * TL;
    line_fft<N, TL, true>(
        ex, tw, li, j,
        [&](int n) {
          const int z = min_img(n, N);
          return (z >= -R && z <= R) ? sb[(z + R) * TL + li] : make_float2(0.f, 0.f);
        },
        [&](int k, float2 v) {
          if (s == 0) {
            C[k * TL + li] = v;
          } else {  // C += i v
            const float2 c = C[k * TL + li];
            C[k * TL + li] = make_float2(c.x - v.y, c.y + v.x);
          }
        });
    const bool last = !npack || s == 1 || b == nb - 1;
    if (!last) continue;
    __syncthreads();
    float2* oc = out + (long long)o * ng + cbase + li;
    line_fft<N, TL, true>(
        ex, tw, li, j, [&](int n) { return cmul(C[n * TL + li], D[n * TL + li]); },
        [&](int k, float2 v) { oc[(long long)k * N * N] = v; });
  }
}

// Pass C without packed pairs, in place: the forward transform's outputs,
// times delta-hat, go back into the exchange buffer in natural order, and the
// inverse transform starts from there, so no kernel-column buffer is kept.
// One staging buffer of the support rows, refilled for the next bin once the
// first forward step has read it: exchange + delta-hat + staging is 73 KB per
// CTA at N = 512 with |z| <= 62, three CTAs per SM (pass C with the column
// buffer fits two).  Each thread gathers its points in registers before the
// buffer is rewritten (six barriers per bin).
template <int N>
__global__ void __launch_bounds__(FusedGeo<N>::TLS * FusedGeo<N>::T)
fused_fft_z_ip_kernel(int R, int nb, const float2* __restrict__ tw, const float2* __restrict__ kin,
                      const float2* __restrict__ dhat, float2* __restrict__ out, long long ng) {
  using G = FusedGeo<N>;
  constexpr int TL = G::TLS, R1 = Plan<N>::R1, R2 = Plan<N>::R2, T = G::T;
  extern __shared__ float2 smem[];
  float2* ex = smem;                   // exchange layout n1 (R2 TL + 8) + k2 TL + line, or natural k TL + line
  float2* D = ex + TL * N + G::EXPAD;  // delta-hat, [k][line]
  float2* stg = D + TL * N;            // staging of the support rows, [2R + 1][line]
  const int rows = 2 * R + 1;
  const int t = threadIdx.x, j = t / TL, li = t % TL;
  const int xg = blockIdx.x % (N / TL), yy = blockIdx.x / (N / TL);
  const long long cbase = (long long)yy * N + (long long)xg * TL;  // (0, y, x0)
  auto sidx = [&](int n1, int k2) { return n1 * (R2 * TL + 8) + k2 * TL + li; };
  auto prefetch = [&](int b) {
    float2* dst = stg;
    const float2* src = kin + (long long)b * ng + cbase;
    for (int c = t; c < rows * (TL / 2); c += blockDim.x) {
      const int r = c / (TL / 2), q = c % (TL / 2);
      const int z = r - R, zi = z < 0 ? z + N : z;
      cp_async16(dst + r * TL + 2 * q, src + (long long)zi * N * N + 2 * q);
    }
    cp_async_commit();
  };
  // delta-hat of the CTA's lines (16-byte copies, in bin 0's copy group)
  for (int c = t; c < N * (TL / 2); c += blockDim.x) {
    const int k = c / (TL / 2), q = c % (TL / 2);
    cp_async16(D + k * TL + 2 * q, dhat + (long long)k * N * N + cbase + 2 * q);
  }
  prefetch(0);
  float2 v[R1 / T][R2];
  float2 u[R2 / T][R1];
  for (int b = 0; b < nb; ++b) {
    cp_async_wait0();         // bin b's rows have landed (this thread's copies)
    __syncthreads();          // ... everyone's; the previous bin has read the exchange buffer
    const float2* sb = stg;
    // forward, step 1 (from the staged support rows; zero outside |z| <= R)
#pragma unroll
    for (int q = 0; q < R1 / T; ++q) {
      const int n1 = j + T * q;
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        const int z = min_img(n1 + R1 * n2, N);
        v[q][n2] = (z >= -R && z <= R) ? sb[(z + R) * TL + li] : make_float2(0.f, 0.f);
      }
      Dft<R2, 1>::run(v[q]);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) ex[sidx(n1, k2)] = k2 ? cmul(v[q][k2], __ldg(tw + ((n1 * k2) & (N - 1)))) : v[q][k2];
    }
    __syncthreads();
    // the staging buffer is read: the next bin's rows land while this one is transformed
    if (b + 1 < nb) prefetch(b + 1);
    // forward, step 2, into registers
#pragma unroll
    for (int q = 0; q < R2 / T; ++q) {
      const int k2 = j + T * q;
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[q][n1] = ex[sidx(n1, k2)];
      Dft<R1, 1>::run(u[q]);
    }
    __syncthreads();  // every exchange value read
    // the product with delta-hat, natural order k = k2 + R2 k1
#pragma unroll
    for (int q = 0; q < R2 / T; ++q)
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int k = j + T * q + R2 * k1;
        ex[k * TL + li] = cmul(u[q][k1], D[k * TL + li]);
      }
    __syncthreads();
    // inverse, step 1, gathered into registers
#pragma unroll
    for (int q = 0; q < R1 / T; ++q) {
      const int n1 = j + T * q;
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) v[q][n2] = ex[(n1 + R1 * n2) * TL + li];
      Dft<R2, 1>::run(v[q]);
    }
    __syncthreads();  // every product read
#pragma unroll
    for (int q = 0; q < R1 / T; ++q) {
      const int n1 = j + T * q;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) ex[sidx(n1, k2)] = k2 ? cmul(v[q][k2], __ldg(tw + ((n1 * k2) & (N - 1)))) : v[q][k2];
    }
    __syncthreads();
    // inverse, step 2, to the coefficient array
    float2* oc = out + (long long)b * ng + cbase + li;
#pragma unroll
    for (int q = 0; q < R2 / T; ++q) {
      const int k2 = j + T * q;
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[q][n1] = ex[sidx(n1, k2)];
      Dft<R1, 1>::run(u[q]);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) oc[(long long)(k2 + R2 * k1) * N * N] = u[q][k1];
    }
  }
}

template <int N>
cudaError_t launch_n(const FusedGroup& g, cudaStream_t st) {
  using G = FusedGeo<N>;
  cudaError_t e;
  if ((e = ensure_smem_attr<kgen_fft_x_kernel<N>>(G::SMEM_A)) != cudaSuccess) return e;
  if ((e = ensure_smem_attr<disk_fft_y_kernel<N>>(G::SMEM_B)) != cudaSuccess) return e;
  if ((e = ensure_smem_attr<fused_fft_z_kernel<N>>(G::SMEM_C + 2 * N * G::TLS * 8)) != cudaSuccess) return e;
  const long long ng = (long long)N * N * N;
  if (g.nlines > 0) {
    dim3 ga((unsigned)((g.nlines + G::TLA - 1) / G::TLA), (unsigned)g.nb);
    kgen_fft_x_kernel<N><<<ga, G::TLA * G::T, G::SMEM_A, st>>>(g.l, g.m, g.norm_scale, g.e2, g.lines, g.nlines, g.tw,
                                                               g.kbuf, ng);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 gb((unsigned)((2 * g.R + 1) * (N / G::TLB)), (unsigned)g.nb);
    disk_fft_y_kernel<N><<<gb, G::TLB * G::T, G::SMEM_B, st>>>(g.e2nb, g.R, g.tw, g.kbuf, ng);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (g.npack == 0) {
    // 2 TLS N exchange / delta-hat values (+ the exchange padding) and the
    // staging of at most N + 1 rows
    if ((e = ensure_smem_attr<fused_fft_z_ip_kernel<N>>(2 * G::TLS * N * 8 + G::EXPAD * 8 + (N + 1) * G::TLS * 8)) !=
        cudaSuccess)
      return e;
    // |z| <= N / 2 covers every plane (z = +-N/2 is the same plane, staged twice)
    const int rz = g.R < N / 2 ? g.R : N / 2;
    const int smem_ip = 2 * G::TLS * N * 8 + G::EXPAD * 8 + (2 * rz + 1) * G::TLS * 8;
    fused_fft_z_ip_kernel<N><<<(unsigned)(N * (N / G::TLS)), G::TLS * G::T, smem_ip, st>>>(rz, g.nb, g.tw, g.kbuf,
                                                                                             g.dhat, g.out, ng);
    return cudaGetLastError();
  }
  const int smem_c = G::SMEM_C + 2 * (2 * g.R + 1) * G::TLS * 8;
  fused_fft_z_kernel<N><<<(unsigned)(N * (N / G::TLS)), G::TLS * G::T, smem_c, st>>>(
      g.R, g.nb, g.npack, g.tw, g.kbuf, g.dhat, g.out, ng);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_group(int n, const FusedGroup& g, cudaStream_t st) {
  if (g.nb < 1 || g.R < 0 || 2 * g.R + 1 > n || (g.npack && (g.npack > g.nb))) return cudaErrorInvalidValue;
  switch (n) {
    case 8: return launch_n<8>(g, st);
    case 16: return launch_n<16>(g, st);
    case 32: return launch_n<32>(g, st);
    case 64: return launch_n<64>(g, st);
    case 128: return launch_n<128>(g, st);
    case 256: return launch_n<256>(g, st);
    case 512: return launch_n<512>(g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbg
