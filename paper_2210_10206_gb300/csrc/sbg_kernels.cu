// Preprocessing, kernel generation, 3PCF Gram, FP32 SIMT 4PCF contraction and
// FP64 finalisation kernels.
#include <algorithm>

#include "sbg_kernels.cuh"
#include "sbg_tcgen05.cuh"

namespace sbg {

// ------------------------------------------------------------------ reduce --
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_add_d(double v, double* dst) {
  __shared__ double part[32];
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    v = warp_sum_d(v);
    if (lane == 0) atomicAdd(dst, v);
  }
}

// field f = blockIdx.y of a slab: its n values start at f * n; acc[2f] collects
// the sum and acc[2f + 1] N_gal
__global__ void sum_kernel(const void* in, int is_f64, long long n, double* acc) {
  const long long f0 = (long long)blockIdx.y * n;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += is_f64 ? reinterpret_cast<const double*>(in)[f0 + i] : (double)reinterpret_cast<const float*>(in)[f0 + i];
  block_add_d(s, acc + 2 * blockIdx.y);
}

__global__ void convert_kernel(const void* in, int is_f64, long long n, const double* acc, int subtract,
                               float* out, double* ngal) {
  const long long f0 = (long long)blockIdx.y * n;
  const double mean = subtract ? acc[2 * blockIdx.y] / (double)n : 0.0;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = is_f64 ? reinterpret_cast<const double*>(in)[f0 + i] : (double)reinterpret_cast<const float*>(in)[f0 + i];
    v -= mean;
    out[f0 + i] = (float)v;
    s += v + 1.0;
  }
  block_add_d(s, ngal + 2 * blockIdx.y);
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)device_sms() * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// CTAs per field of a slab of nfld fields: the single-field grid, shared out
static dim3 grid_fields(long long n, int nfld) {
  long long b = grid_for(n, 256);
  if (nfld > 1) b = std::max<long long>(1, std::min<long long>(b, ((long long)device_sms() * 16 + nfld - 1) / nfld));
  return dim3((unsigned)b, (unsigned)nfld);
}

cudaError_t launch_sum(const void* in, int is_f64, long long n, double* acc, cudaStream_t st, int nfld) {
  if (nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  sum_kernel<<<grid_fields(n, nfld), 256, 0, st>>>(in, is_f64, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* in, int is_f64, long long n, const double* acc, int subtract, float* out,
                           cudaStream_t st, int nfld) {
  if (nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  convert_kernel<<<grid_fields(n, nfld), 256, 0, st>>>(in, is_f64, n, acc, subtract, out,
                                                        const_cast<double*>(acc) + 1);
  return cudaGetLastError();
}

// ---------------------------------------------------------- kernel generation --
__device__ __forceinline__ int min_image(int i, int n) { return i < n - i ? i : i - n; }

__device__ __forceinline__ int find_bin(double r2, const double* e2, int nb) {
  if (!(r2 > e2[0]) || r2 > e2[nb]) return -1;
  int b = 0;
  while (b < nb - 1 && r2 > e2[b + 1]) ++b;
  return b;
}

// conj(Y_lm) * Theta_b on the minimum-image offset grid (Algorithm 1); Y_lm from the
// reduced associated Legendre recurrence times ((x + i y)/r)^m, in FP64.
__global__ void kgen3d_kernel(int n, int l, int m, double norm, const double* __restrict__ e2, int nb, double scale,
                              float2* __restrict__ out) {
  const long long ng = (long long)n * n * n;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= ng) return;
  const int ix = (int)(cell % n), iy = (int)((cell / n) % n), iz = (int)(cell / ((long long)n * n));
  const int x = min_image(ix, n), y = min_image(iy, n), z = min_image(iz, n);
  const double r2 = (double)x * x + (double)y * y + (double)z * z;
  const int b = find_bin(r2, e2, nb);
  if (b < 0) return;
  const double r = sqrt(r2);
  const double t = z / r;
  // reduced associated Legendre (-1)^m d^m P_l/dt^m
  double pmm = (m & 1) ? -1.0 : 1.0;
  for (int k = 1; k < 2 * m; k += 2) pmm *= k;
  double p = pmm;
  if (l > m) {
    double a = pmm, bb = (2 * m + 1) * t * pmm;
    for (int ll = m + 2; ll <= l; ++ll) {
      double c = ((2 * ll - 1) * t * bb - (ll + m - 1) * a) / (ll - m);
      a = bb;
      bb = c;
    }
    p = bb;
  }
  double ur = x / r, ui = y / r, er = 1.0, ei = 0.0;
  for (int k = 0; k < m; ++k) {
    const double tr = er * ur - ei * ui;
    ei = er * ui + ei * ur;
    er = tr;
  }
  const double s = norm * p * scale;
  out[(long long)b * ng + cell] = make_float2((float)(s * er), (float)(-s * ei));
}

// conj(((x + i y)/rho)^m) * Theta_b (Algorithm 2)
__global__ void kgen2d_kernel(int n, int m, const double* __restrict__ e2, int nb, double scale,
                              float2* __restrict__ out) {
  const long long ng = (long long)n * n;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= ng) return;
  const int x = min_image((int)(cell % n), n), y = min_image((int)(cell / n), n);
  const double r2 = (double)x * x + (double)y * y;
  const int b = find_bin(r2, e2, nb);
  if (b < 0) return;
  const double r = sqrt(r2);
  double ur = x / r, ui = y / r, er = 1.0, ei = 0.0;
  for (int k = 0; k < m; ++k) {
    const double tr = er * ur - ei * ui;
    ei = er * ui + ei * ur;
    er = tr;
  }
  out[(long long)b * ng + cell] = make_float2((float)(er * scale), (float)(-ei * scale));
}

cudaError_t launch_kgen3d(int n, int l, int m, double norm_lm, const double* e2_dev, int nb, double scale,
                          float2* out, cudaStream_t st) {
  const long long ng = (long long)n * n * n;
  kgen3d_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(n, l, m, norm_lm, e2_dev, nb, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_kgen2d(int n, int m, const double* e2_dev, int nb, double scale, float2* out, cudaStream_t st) {
  const long long ng = (long long)n * n;
  kgen2d_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(n, m, e2_dev, nb, scale, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gram3 --
// S[b1][b2] += sum_x delta(x) a_b1(x) conj(a_b2(x)) for b1 <= b2 (Algorithm 5's
// delta-weighted products of the coefficients, Eq. zeta3 of Sec. 2.2).  One CTA
// sweeps a contiguous x-range in chunks of 128 points, staged in shared memory
// by cp.async through a ring of kGramStages chunks (three in flight while one
// is summed).  The bins (at most 20) form blocks of 4; warp w owns block pair
// w (I <= J; at most 15) and its lanes take every 32nd point, so each lane
// holds a 4 x 4 tile of pair sums (16 complex, FP32 with packed f32x2 FMAs: 8
// operand loads per 16 products).  Every kGramFlush chunks a warp reduce-scatter hands
// lane k the warp's total of tile element k, which it adds to an FP64
// register; at the end each lane adds its element to S (FP64 atomics).
constexpr int kGramChunk = 128;
constexpr int kGramMaxNb = 20;
constexpr int kGramFlush = 4;   // chunks (16 points per lane) between FP64 flushes
constexpr int kGramStages = 4;  // ring of staged chunks

__device__ __forceinline__ void gram_cp(void* dst, const void* src, bool ok, int bytes) {
  // bytes 4 / 8 / 16; a copy outside the range reads nothing and writes zeros
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = ok ? bytes : 0;
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__global__ void __launch_bounds__(512, 2) gram3_kernel(const float2* __restrict__ a, long long ng, int nb,
                                                    const float* __restrict__ delta, double* __restrict__ S,
                                                    int nsingle, int single0, long long s_stride) {
  // field f = blockIdx.y of a slab: its bins follow field f - 1's (group
  // buffer) or its points do (blocked store); its delta and S likewise
  const long long fx = (long long)blockIdx.y * ng;
  if (!nsingle) a += (long long)blockIdx.y * nb * ng;
  delta += fx;
  S += (long long)blockIdx.y * s_stride;
  const int nbb = (nb + 3) / 4, nrow = 4 * nbb;
  // stage: nrow rows of kGramChunk (re, im), then kGramChunk deltas; rows nb ..
  // of the last block stay zero
  extern __shared__ __align__(16) uint8_t gsm[];
  const int stage_bytes = nrow * kGramChunk * 8 + kGramChunk * 4;
  auto srow = [&](int st, int b) { return reinterpret_cast<float2*>(gsm + st * stage_bytes) + b * kGramChunk; };
  auto sdel = [&](int st) { return reinterpret_cast<float*>(gsm + st * stage_bytes + nrow * kGramChunk * 8); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // x-ranges of whole chunks: x0 and x1 are multiples of 4 (ng is), so the
  // 16-byte copies below never straddle x1
  const long long per = ((ng + gridDim.x - 1) / gridDim.x + kGramChunk - 1) / kGramChunk * kGramChunk;
  const long long x0 = blockIdx.x * per, x1 = min(ng, x0 + per);
  const int nch = x0 < x1 ? (int)((x1 - x0 + kGramChunk - 1) / kGramChunk) : 0;
  for (int i = threadIdx.x; i < kGramStages * (nrow - nb) * kGramChunk; i += blockDim.x) {
    const int st = i / ((nrow - nb) * kGramChunk), r = i % ((nrow - nb) * kGramChunk);
    srow(st, nb + r / kGramChunk)[r % kGramChunk] = make_float2(0.f, 0.f);
  }
  // this warp's block pair (none for warps past the last one)
  int bI = -1, bJ = -1;
  for (int i = 0, q = warp; i < nbb && q >= 0; ++i) {
    if (q < nbb - i) {
      bI = i;
      bJ = i + q;
    }
    q -= nbb - i;
  }
  // copies of chunk c into stage c % kGramStages, one commit group per chunk
  auto issue = [&](int c) {
    if (c < nch) {
      const int st = c % kGramStages;
      const long long xc = x0 + (long long)c * kGramChunk;
      if (nsingle) {
        // blocked store: per 32-point block 32 Re then 32 Im floats of a single
        for (int i = threadIdx.x; i < nb * kGramChunk; i += blockDim.x) {
          const int b = i / kGramChunk, xx = i % kGramChunk;
          const long long x = xc + xx;
          const bool ok = x < x1;
          const float* f = reinterpret_cast<const float*>(a) + blocked_re(fx + (ok ? x : x0), single0 + b, nsingle);
          float2* dst = srow(st, b) + xx;
          gram_cp(&dst->x, f, ok, 4);
          gram_cp(&dst->y, f + 32, ok, 4);
        }
      } else {
        // group buffer: bins of ng complex, two points per 16-byte copy
        for (int i = threadIdx.x; i < nb * kGramChunk / 2; i += blockDim.x) {
          const int b = i / (kGramChunk / 2), xx = 2 * (i % (kGramChunk / 2));
          const long long x = xc + xx;  // even, and x1 is a multiple of 4
          const bool ok = x < x1;
          gram_cp(srow(st, b) + xx, a + (long long)b * ng + (ok ? x : x0), ok, 16);
        }
      }
      for (int i = threadIdx.x; i < kGramChunk / 4; i += blockDim.x) {
        const long long x = xc + 4 * i;
        const bool ok = x < x1;
        gram_cp(sdel(st) + 4 * i, delta + (ok ? x : x0), ok, 16);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  uint64_t acc[16];
  double dacc = 0.0;
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0ull;
  // lane k of the warp gets the warp's total of element k of the 32 floats
  auto flush = [&]() {
    float v[32];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      upk(acc[e], v[2 * e], v[2 * e + 1]);
      acc[e] = 0ull;
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
      const int o = 16 >> lv;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int e = 0; e < o; ++e) {
        const float send = up ? v[e] : v[e + o];
        const float keep = up ? v[e + o] : v[e];
        v[e] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    dacc += (double)v[0];
  };
  __syncthreads();  // zero rows written
#pragma unroll
  for (int c = 0; c < kGramStages - 1; ++c) issue(c);
  int nflush = 0;
  for (int c = 0; c < nch; ++c) {
    asm volatile("cp.async.wait_group %0;" ::"n"(kGramStages - 2) : "memory");
    __syncthreads();  // chunk c landed for every thread; chunk c - 1 has been summed
    issue(c + kGramStages - 1);
    const int st = c % kGramStages;
    const float* sd = sdel(st);
    if (bI >= 0) {
      const float2* s1 = srow(st, 4 * bI);
      const float2* s2 = srow(st, 4 * bJ);
#pragma unroll 2
      for (int m = 0; m < kGramChunk / 32; ++m) {
        const int xx = lane + 32 * m;
        const float d = sd[xx];
        const uint64_t dd = pk(d, d);
        uint64_t w[4], wr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 u = s1[i * kGramChunk + xx];
          w[i] = mul2(pk(u.x, u.y), dd);    // delta u
          wr[i] = mul2(pk(u.y, -u.x), dd);  // delta (Im u, -Re u)
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 v = s2[j * kGramChunk + xx];
          const uint64_t vr = pk(v.x, v.x), vi = pk(v.y, v.y);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            // (Re, Im) of delta u conj(v) = w Re v + (Im w, -Re w) Im v
            acc[4 * i + j] = fma2(w[i], vr, acc[4 * i + j]);
            acc[4 * i + j] = fma2(wr[i], vi, acc[4 * i + j]);
          }
        }
      }
    }
    if (++nflush == kGramFlush) {
      flush();
      nflush = 0;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (nflush) flush();
  if (bI >= 0) {
    // lane = 2 (4 i + j) + component
    const int e = lane >> 1, c = lane & 1, i = e >> 2, j = e & 3;
    const int b1 = 4 * bI + i, b2 = 4 * bJ + j;
    if (b1 <= b2 && b2 < nb) atomicAdd(&S[((long long)b1 * nb + b2) * 2 + c], dacc);
  }
}

cudaError_t launch_gram3(const float2* a, long long ng, int nb, const float* delta, double* S, int nsingle,
                         int single0, cudaStream_t st, int nfld, long long s_stride) {
  if (nb < 1 || nb > kGramMaxNb || nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  // 16-byte copies of the group buffer and of delta
  if (!nsingle && (((uintptr_t)a & 15) || (ng & 1))) return cudaErrorInvalidValue;
  if (((uintptr_t)delta & 15) || (ng & 3)) return cudaErrorInvalidValue;
  const int nbb = (nb + 3) / 4, nbp = nbb * (nbb + 1) / 2;
  const int threads = std::max(32 * nbp, 128);  // a warp per block pair, at least 4 to stage
  const int smem = kGramStages * (4 * nbb * kGramChunk * 8 + kGramChunk * 4);
  // the attribute is set once per device: to the largest stage ring
  constexpr int kMaxSmem = kGramStages * (4 * ((kGramMaxNb + 3) / 4) * kGramChunk * 8 + kGramChunk * 4);
  cudaError_t e = ensure_smem_attr<gram3_kernel>(kMaxSmem);
  if (e != cudaSuccess) return e;
  // chunks per CTA: about 4 on small grids; on large ones as many CTAs as fit
  long long blocks = (ng + 4 * kGramChunk - 1) / (4 * kGramChunk);
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram3_kernel, threads, smem)) != cudaSuccess) return e;
  const long long cap = std::max<long long>(1, ((long long)device_sms() * std::max(per_sm, 1) + nfld - 1) / nfld);
  if (blocks > cap) blocks = cap;
  gram3_kernel<<<dim3((unsigned)blocks, nfld), threads, smem, st>>>(a, ng, nb, delta, S, nsingle, single0, s_stride);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ simt4 --
// T[r][c] = sum_x delta(x) f1_r(x) f2_r(x) a_c(x): the pair-by-single contraction
// of the 4PCF (Eq. mu of Sec. 2.3, Eq. proj_4pcf_coeff) as an FP32 SIMT GEMM over
// x with the pair operand formed on chip.  Per 32-point chunk the tile's row
// singles, its column singles and delta are copied with cp.async into one of two
// raw buffers while the previous chunk is computed; then the pair products
// P_r = sign delta f1 f2 and the transposed columns are formed in shared memory
// and each thread accumulates a 4x4 block of rows x cols.  FP32 over 512-point
// spans, FP64 across spans and CTAs.
constexpr int kX = 32;          // points per chunk
constexpr int kSpan = 16;       // chunks per FP32 span
constexpr int kRawF = 68;       // floats per raw row: Re x0..31, Im x0..31, pad (16-byte multiple)

__device__ __forceinline__ void simt_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

template <int TCG>
struct SimtSmem {
  static constexpr int TR = 4 * (256 / TCG), TC = 4 * TCG;
  static constexpr int kRawU = kSimtMaxUniq * kRawF;  // floats of one raw row-single buffer
  static constexpr int kRawC = TC * kRawF;             // floats of one raw column buffer
  static constexpr int kRaw = kRawU + kRawC + kX;      // one raw buffer (+ delta)
  static constexpr size_t kBytes = (size_t)(2 * kRaw) * 4 + (size_t)(kX * TR + kX * TC) * 8;
};

template <int TCG, bool CPLX>
__global__ void __launch_bounds__(256) simt4_kernel(const float2* __restrict__ astore, long long ng,
                                                    const float* __restrict__ delta, const Tile4* __restrict__ tiles,
                                                    const Row4* __restrict__ rows, const int* __restrict__ cols,
                                                    const int* __restrict__ uniq, int nsplit, int nsingle,
                                                    double* __restrict__ T, int imag, int splits_per_field,
                                                    long long t_field_stride) {
  // a slab of fields: x-split blockIdx.y belongs to field blockIdx.y / splits_per_field
  if (splits_per_field) T += (long long)(blockIdx.y / splits_per_field) * t_field_stride;
  using SM = SimtSmem<TCG>;
  constexpr int TR = SM::TR, TC = SM::TC;
  extern __shared__ float4 smem4[];
  float* raw = reinterpret_cast<float*>(smem4);                       // [2][kRaw]
  float2* Ps = reinterpret_cast<float2*>(raw + 2 * SM::kRaw);         // [kX][TR]
  float2* Cs = Ps + kX * TR;                                          // [kX][TC]

  const Tile4 tl = tiles[blockIdx.x];
  // the plan keeps tiles within the staging buffers; a tile that is not is skipped
  if (tl.nuniq > kSimtMaxUniq || tl.ncols > TC || tl.nrows > TR) return;
  const int tid = threadIdx.x;
  const int cg = tid % TCG, rg = tid / TCG;
  const long long per = ((ng / kX + nsplit - 1) / nsplit) * kX;
  const long long x0 = blockIdx.y * per, x1 = min(ng, x0 + per);

  // copy chunk xc (raw blocked rows: 16 chunks of 16 B per single) into buffer b
  auto stage = [&](long long xc, int b) {
    float* ru = raw + b * SM::kRaw;
    float* rc = ru + SM::kRawU;
    float* rd = rc + SM::kRawC;
    const float* base = reinterpret_cast<const float*>(astore) + (xc / kX) * (long long)nsingle * 64;
    const int nu = tl.nuniq * 16, nc = tl.ncols * 16;
    for (int i = tid; i < nu + nc + 8; i += 256) {
      if (i < nu) {
        simt_cp16(ru + (i >> 4) * kRawF + (i & 15) * 4, base + uniq[tl.uniq0 + (i >> 4)] * 64 + (i & 15) * 4);
      } else if (i < nu + nc) {
        const int k = i - nu;
        simt_cp16(rc + (k >> 4) * kRawF + (k & 15) * 4, base + cols[tl.col0 + (k >> 4)] * 64 + (k & 15) * 4);
      } else {
        const int k = i - nu - nc;
        simt_cp16(rd + k * 4, delta + xc + k * 4);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  float acc[4][4][CPLX ? 2 : 1];
  double dacc[4][4][CPLX ? 2 : 1];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < (CPLX ? 2 : 1); ++c) { acc[i][k][c] = 0.f; dacc[i][k][c] = 0.0; }

  int span = 0, b = 0;
  if (x0 < x1) stage(x0, 0);
  for (long long xc = x0; xc < x1; xc += kX, b ^= 1) {
    // prefetch the next chunk into the other buffer (its last readers finished
    // before the barrier that ended the previous iteration)
    if (xc + kX < x1) {
      stage(xc + kX, b ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* ru = raw + b * SM::kRaw;
    const float* rc = ru + SM::kRawU;
    const float* rd = rc + SM::kRawC;
    // columns, transposed to [x][c] (zero past the tile's columns); imag: a is
    // stored as (Im a, -Re a), so that the real accumulation gives Im(P a)
    for (int i = tid; i < TC * kX; i += 256) {
      const int c = i % TC, xx = i / TC;
      float2 v = make_float2(0.f, 0.f);
      if (c < tl.ncols) {
        const float re = rc[c * kRawF + xx], im = rc[c * kRawF + 32 + xx];
        v = imag ? make_float2(im, -re) : make_float2(re, im);
      }
      Cs[xx * TC + c] = v;
    }
    // pair products P_r(x) = sign * delta * f1 * f2
    for (int i = tid; i < TR * kX; i += 256) {
      const int r = i % TR, xx = i / TR;
      float2 p = make_float2(0.f, 0.f);
      if (r < tl.nrows) {
        const Row4 rw = rows[tl.row0 + r];
        float2 f1 = make_float2(ru[rw.u1 * kRawF + xx], ru[rw.u1 * kRawF + 32 + xx]);
        float2 f2 = make_float2(ru[rw.u2 * kRawF + xx], ru[rw.u2 * kRawF + 32 + xx]);
        if (rw.flags & 1) f1.y = -f1.y;
        if (rw.flags & 2) f2.y = -f2.y;
        const float s = rw.sign * rd[xx];
        p = cmul(f1, f2);
        p.x *= s;
        p.y *= s;
      }
      Ps[xx * TR + r] = p;
    }
    __syncthreads();
    // operands of point xx + 1 are loaded while point xx is accumulated
    const float4* pr0 = reinterpret_cast<const float4*>(Ps + rg * 4);
    const float4* cr0 = reinterpret_cast<const float4*>(Cs + cg * 4);
    float4 np01 = pr0[0], np23 = pr0[1], nc01 = cr0[0], nc23 = cr0[1];
#pragma unroll 4
    for (int xx = 0; xx < kX; ++xx) {
      const float4 p01 = np01, p23 = np23, c01 = nc01, c23 = nc23;
      if (xx + 1 < kX) {
        const float4* pr = reinterpret_cast<const float4*>(Ps + (xx + 1) * TR + rg * 4);
        const float4* cr = reinterpret_cast<const float4*>(Cs + (xx + 1) * TC + cg * 4);
        np01 = pr[0];
        np23 = pr[1];
        nc01 = cr[0];
        nc23 = cr[1];
      }
      const float2 P[4] = {{p01.x, p01.y}, {p01.z, p01.w}, {p23.x, p23.y}, {p23.z, p23.w}};
      const float2 C[4] = {{c01.x, c01.y}, {c01.z, c01.w}, {c23.x, c23.y}, {c23.z, c23.w}};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[i][k][0] = fmaf(P[i].x, C[k].x, fmaf(-P[i].y, C[k].y, acc[i][k][0]));
          if (CPLX) acc[i][k][CPLX ? 1 : 0] = fmaf(P[i].x, C[k].y, fmaf(P[i].y, C[k].x, acc[i][k][CPLX ? 1 : 0]));
        }
    }
    if (++span == kSpan) {
      span = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < (CPLX ? 2 : 1); ++c) { dacc[i][k][c] += acc[i][k][c]; acc[i][k][c] = 0.f; }
    }
    __syncthreads();  // Ps, Cs and this raw buffer are free for the next chunk
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = rg * 4 + i;
    if (r >= tl.nrows) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = cg * 4 + k;
      if (c >= tl.ncols) continue;
#pragma unroll
      for (int q = 0; q < (CPLX ? 2 : 1); ++q) {
        const double v = dacc[i][k][q] + acc[i][k][q];
        atomicAdd(&T[(tl.tout + (long long)r * tl.ncols + c) * (CPLX ? 2 : 1) + q], v);
      }
    }
  }
}

template <int TCG, bool CPLX>
static cudaError_t simt4_t(const float2* astore, long long ng, const float* delta, const Tile4* tiles, int ntiles,
                          const Row4* rows, const int* cols, const int* uniq, int nsplit, int nsingle, double* T,
                          int nsm, int imag, cudaStream_t st, int nfld, long long t_field_stride) {
  const size_t smem = SimtSmem<TCG>::kBytes;
  auto kern = simt4_kernel<TCG, CPLX>;
  {
    cudaError_t e = ensure_smem_attr<simt4_kernel<TCG, CPLX>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  int spf = 0;  // x-splits per field of a slab
  if (nfld > 1) {
    // a slab: every field is split alike (a power of two dividing its
    // K-blocks), the split count chosen for the best fill of the resident slots
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)nsm * (per_sm > 0 ? per_sm : 1), fchunks = ng / nfld / kX;
    double best = -1.0;
    spf = 1;
    for (long long k = 1; k <= fchunks && k <= 64; k *= 2) {
      const long long units = (long long)ntiles * nfld * k;
      if (units > 65535LL * ntiles) break;
      const double fill = (double)units / (double)(slots * ((units + slots - 1) / slots));
      if (fill > best + 1e-3) {
        best = fill;
        spf = (int)k;
      }
      if (units >= 4 * slots) break;
    }
    nsplit = nfld * spf;
  } else if (nsplit <= 0) {
    // x-splits per tile so that the CTAs fill whole waves of the resident
    // slots (SMs x CTAs per SM): the best fill over 2..8 waves, fewer on ties
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)nsm * (per_sm > 0 ? per_sm : 1), chunks = ng / kX;
    double best = -1.0;
    nsplit = 1;
    for (int w = 2; w <= 8; ++w) {
      const long long ns = std::max<long long>(1, std::min<long long>(chunks, slots * w / ntiles));
      const long long units = ns * ntiles;
      const double fill = (double)units / (double)(slots * ((units + slots - 1) / slots));
      if (fill > best + 1e-3) {
        best = fill;
        nsplit = (int)ns;
      }
    }
  }
  if (nsplit > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)ntiles, (unsigned)nsplit);
  kern<<<grid, 256, smem, st>>>(astore, ng, delta, tiles, rows, cols, uniq, nsplit, nsingle, T, imag, spf,
                                t_field_stride);
  return cudaGetLastError();
}

cudaError_t launch_simt4(const float2* astore, long long ng, const float* delta, const Tile4* tiles, int ntiles,
                         const Row4* rows, const int* cols, const int* uniq, int complex_out, int tcg, int nsplit,
                         int nsingle, double* T, int nsm, cudaStream_t st, int nfld, long long t_field_stride) {
  if (ntiles <= 0) return cudaSuccess;
  if (ng % kX || complex_out < 0 || complex_out > 2 || nfld < 1 || (ng / nfld) % kX) return cudaErrorInvalidValue;
  const int imag = complex_out == 2 ? 1 : 0;  // real T holding Im(P a)
  if (complex_out == 1) {
    if (tcg == 4) return simt4_t<4, true>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
    if (tcg == 8) return simt4_t<8, true>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
    if (tcg == 16) return simt4_t<16, true>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
  } else {
    if (tcg == 4) return simt4_t<4, false>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
    if (tcg == 8) return simt4_t<8, false>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
    if (tcg == 16) return simt4_t<16, false>(astore, ng, delta, tiles, ntiles, rows, cols, uniq, nsplit, nsingle, T, nsm, imag, st, nfld, t_field_stride);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------- finalisation --
__global__ void couple_kernel(const double* __restrict__ T, int complex_t, const int* __restrict__ ptr,
                              const int* __restrict__ idx, const double* __restrict__ coef, int nout,
                              double* __restrict__ zeta, long long t_stride) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  // field blockIdx.y of a slab: its T and zeta follow the previous field's
  T += (long long)blockIdx.y * t_stride * (complex_t ? 2 : 1);
  zeta += (long long)blockIdx.y * nout * (complex_t ? 2 : 1);
  double re = 0.0, im = 0.0;
  for (int e = ptr[o]; e < ptr[o + 1]; ++e) {
    int i = idx[e];
    const bool cj = i < 0;
    if (cj) i = -i - 1;
    const double c = coef[e];
    if (complex_t) {
      re += c * T[2LL * i];
      im += c * (cj ? -T[2LL * i + 1] : T[2LL * i + 1]);
    } else {
      re += c * T[i];
    }
  }
  if (complex_t) {
    zeta[2LL * o] = re;
    zeta[2LL * o + 1] = im;
  } else {
    zeta[o] = re;
  }
}

cudaError_t launch_couple(const double* T, int complex_t, const int* ptr, const int* idx, const double* coef, int nout,
                          double* zeta, cudaStream_t st, int nfld, long long t_stride) {
  if (nout <= 0) return cudaSuccess;
  if (nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  couple_kernel<<<dim3((nout + 255) / 256, nfld), 256, 0, st>>>(T, complex_t, ptr, idx, coef, nout, zeta, t_stride);
  return cudaGetLastError();
}

__global__ void finish3_kernel(const double* __restrict__ S, int full, int lmax, int nb, double* __restrict__ zeta,
                               long long s_stride) {
  const int nl = lmax + 1;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nl * nb * nb) return;
  // field blockIdx.y of a slab
  S += (long long)blockIdx.y * s_stride;
  zeta += (long long)blockIdx.y * nl * nb * nb * (full ? 1 : 2);
  const int l = o / (nb * nb), b1 = (o / nb) % nb, b2 = o % nb;
  // S stored for b1 <= b2; S[b2][b1] = conj(S[b1][b2])
  const int lo = min(b1, b2), hi = max(b1, b2);
  const double cj = (b1 <= b2) ? 1.0 : -1.0;
  if (full) {
    double s = 0.0;
    for (int m = 0; m <= l; ++m) {
      const long long pi = (long long)l * (l + 1) / 2 + m;
      const double re = S[((pi * nb + lo) * nb + hi) * 2];
      s += (m == 0 ? 1.0 : 2.0) * re;
    }
    zeta[o] = ((l & 1) ? -1.0 : 1.0) / sqrt(2.0 * l + 1.0) * s;
  } else {
    const long long pi = l;
    zeta[2LL * o] = S[((pi * nb + lo) * nb + hi) * 2];
    zeta[2LL * o + 1] = cj * S[((pi * nb + lo) * nb + hi) * 2 + 1];
  }
}

cudaError_t launch_finish3(const double* S, int full, int lmax, int nb, double* zeta, cudaStream_t st, int nfld,
                           long long s_stride) {
  if (nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  const int n = (lmax + 1) * nb * nb;
  finish3_kernel<<<dim3((n + 255) / 256, nfld), 256, 0, st>>>(S, full, lmax, nb, zeta, s_stride);
  return cudaGetLastError();
}

__global__ void normalize_kernel(double* zeta, long long nouter, int nb, int order, int ncomp, const double* acc,
                                 double ng, const double* vbin) {
  const long long per = (order == 4 ? (long long)nb * nb * nb : (long long)nb * nb);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nouter * per) return;
  // field blockIdx.y of a slab: its outputs and N_gal
  zeta += (long long)blockIdx.y * nouter * per * ncomp;
  const double ngal = acc[2 * blockIdx.y + 1];
  const double nbar = ngal / ng;
  const long long w = i % per;
  double norm = ngal;
  if (order == 4) {
    norm *= nbar * vbin[w / (nb * nb)] * nbar * vbin[(w / nb) % nb] * nbar * vbin[w % nb];
  } else {
    norm *= nbar * vbin[w / nb] * nbar * vbin[w % nb];
  }
  for (int c = 0; c < ncomp; ++c) zeta[i * ncomp + c] /= norm;
}

cudaError_t launch_normalize(double* zeta, long long nouter, int nb, int order, int ncomp, const double* acc, double ng,
                             const double* vbin_dev, cudaStream_t st, int nfld) {
  const long long per = (order == 4 ? (long long)nb * nb * nb : (long long)nb * nb);
  const long long n = nouter * per;
  if (n <= 0) return cudaSuccess;
  if (nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  normalize_kernel<<<dim3((unsigned)((n + 255) / 256), nfld), 256, 0, st>>>(zeta, nouter, nb, order, ncomp, acc, ng,
                                                                            vbin_dev);
  return cudaGetLastError();
}

}  // namespace sbg
