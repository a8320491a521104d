// Shared-memory two-step (four-step) FFT axis passes for N = 8 .. 1024.
//
// The convolution coefficients of the method (Sec. 2.1, Eq. almconv; Algorithms
// 3-4) are inverse FFTs of delta-hat times a kernel spectrum.  A 3D (2D)
// transform is three (two) axis passes over HBM; each pass moves one line of N
// points per (thread group, line) through registers:
//
//   N = R1 * R2,  n = n1 + R1 n2,  k = k2 + R2 k1
//   step 1: R1 DFTs of length R2 over n2, then twiddle W_N^(n1 k2)
//   step 2: R2 DFTs of length R1 over n1 (through shared memory)
//
// Each line is owned by T = min(R1, R2) threads that hold N/T points each, so
// global loads and stores of step 1/2 are single coalesced sweeps (lines that
// are adjacent in memory are handled by adjacent lanes for the strided axes,
// points of one row by adjacent lanes for the contiguous axis).  The spectral
// product of the convolution (delta-hat x kernel spectrum) is fused into the
// first pass, the real->complex promotion of delta into the first forward pass.
#include "sbg_fft_core.cuh"

namespace sbg {


// Lines per CTA of a strided pass: the default, or (variants 1 and 2, chosen
// by the context's autotuner) half or twice it.
template <int N> constexpr int tl_strided_default() { return N >= 1024 ? 8 : (N >= 16 ? 16 : N); }
template <int N> constexpr int tl_strided(int variant) {
  return variant == 1 ? tl_strided_default<N>() / 2 : variant == 2 ? 2 * tl_strided_default<N>() : tl_strided_default<N>();
}

template <int N, bool CONTIG, int TLV = 0> struct Geo {
  static constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
  static constexpr int T = R1 < R2 ? R1 : R2;            // threads per line
  // lines per CTA; strided passes of N = 1024 take 8 lines (64 B runs) so that a
  // CTA stages 64 KB rather than 128 KB and two CTAs per SM overlap their loads
  // and stores (at N = 512, 16 lines measured faster); TLV selects a variant
  static constexpr int TL = CONTIG ? (N <= 32 ? 8 : 256 / T) : tl_strided<N>(TLV);
  static constexpr int THREADS = TL * T;
  static constexpr int R2S = CONTIG ? R2 + 1 : R2;       // padded row of Y (contiguous layout)
  static constexpr int LS = CONTIG ? R1 * R2S + 1 : 0;
  static constexpr int SMEM = (CONTIG ? TL * LS : TL * N) * 8;
  __device__ __forceinline__ static int sidx(int l, int n1, int k2) {
    return CONTIG ? l * LS + n1 * R2S + k2 : (n1 * R2 + k2) * TL + l;
  }
};

template <int N, bool CONTIG, int SIGN, int LOAD, int OUTB, int TLV, bool SLAB>
__global__ void __launch_bounds__(Geo<N, CONTIG, TLV>::THREADS)
fft_axis_kernel(FftPass p) {
  using G = Geo<N, CONTIG, TLV>;
  constexpr int R1 = G::R1, R2 = G::R2, T = G::T, TL = G::TL;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  const int j = CONTIG ? (t % T) : (t / TL);
  const int l = CONTIG ? (t / T) : (t % TL);
  // Passes with the spectral product run every array of a field in one CTA:
  // the field's delta-hat values of the CTA's lines are read from HBM once
  // (into a thread-private shared-memory slot) and reused for each array.
  // Other passes: line group blockIdx.x of batch blockIdx.y.
  constexpr bool kBins = LOAD == LOAD_MUL || LOAD == LOAD_MUL2;
  const int nbpf = kBins ? (SLAB ? p.nb_per_field : p.batch) : 1;
  unsigned tile = blockIdx.x;
  long long bf0 = 0;  // field of the CTA (kBins)
  if (kBins) {
    const unsigned ntile = (unsigned)(p.outer * (p.inner / TL));
    tile = blockIdx.x % ntile;
    bf0 = blockIdx.x / ntile;
  }
  float2* sdh = sm + G::SMEM / 8;  // kBins: delta-hat slots, R1 / T x R2 per thread
  long long base;    // element index of point n = 0 of this thread's line
  long long estride; // element stride along the line
  if (CONTIG) {
    base = ((long long)tile * TL + l) * N;
    estride = 1;
  } else {
    const long long tiles = p.inner / TL;
    const long long o = tile / tiles;
    const long long i0 = (tile % tiles) * TL;
    if (p.prune_mode) {
      // the whole CTA leaves together: the test depends on blockIdx only
      const long long x0 = p.prune_mode == 1 ? i0 % N : i0;
      bool zero = x0 > p.prune_r && x0 + TL - 1 < N - p.prune_r;
      if (p.prune_mode == 1) {
        const long long y = i0 / N;
        zero = zero || (y > p.prune_r && y < N - p.prune_r);
      }
      if (zero) return;
    }
    base = o * (long long)N * p.inner + i0 + l;
    estride = p.inner;
  }

  if (kBins) {
    // this thread's delta-hat values (the points it loads in step 1), once
    const long long soff = (SLAB ? bf0 : 0LL) * p.shared_stride;
#pragma unroll
    for (int q = 0; q < R1 / T; ++q)
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2)
        sdh[(q * R2 + n2) * G::THREADS + t] = __ldg(p.shared + soff + base + (long long)(j + T * q + R1 * n2) * estride);
  }
#pragma unroll 1
  for (int it = 0; it < nbpf; ++it) {
  const int bat = kBins ? (int)(bf0 * nbpf + it) : (int)blockIdx.y;
  const long long boff = (long long)bat * p.bstride;
  // batch index = field bf x nb_per_field + array bj of that field (a slab of
  // fields, SLAB variants); otherwise every batch is array bj of one field
  const int bj = SLAB ? bat % p.nb_per_field : bat;
  const long long bf = SLAB ? (long long)bat / p.nb_per_field : 0;
  const long long moff = (long long)bj * p.bstride;      // factor array of the batch
  const long long soff = bf * p.shared_stride;            // shared array of its field
  const long long fpts = bf * p.field_points;             // its first point in the blocked store
  if (it > 0) __syncthreads();  // the previous array's step 2 has read the exchange buffer
  // opaque per array: the compiler would otherwise keep every point's address
  // and twiddle in registers across the loop (over 160 per thread)
  const float2* twid = p.twiddle;
  long long lbase = base;
  if (kBins) asm volatile("" : "+l"(twid), "+l"(lbase));

  // ---- step 1: R1/T DFTs of length R2 per thread ----
#pragma unroll
  for (int q = 0; q < R1 / T; ++q) {
    const int n1 = j + T * q;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      const long long e = lbase + (long long)(n1 + R1 * n2) * estride;
      if (LOAD == LOAD_REAL) {
        v[n2] = make_float2(__ldg(reinterpret_cast<const float*>(p.in) + boff + e), 0.0f);
      } else if (LOAD == LOAD_MUL || LOAD == LOAD_MUL2) {
        const float2 dh = sdh[(q * R2 + n2) * G::THREADS + t];
        if (LOAD == LOAD_MUL) {
          v[n2] = cmul(dh, __ldg(p.mul + moff + e));
        } else {
          const long long ia = 2 * moff + e;
          float2 f = __ldg(p.mul + ia);
          if (2 * bj + 1 < p.npack) {
            const float2 g = __ldg(p.mul + ia + p.bstride);
            f.x -= g.y;
            f.y += g.x;
          }
          v[n2] = cmul(dh, f);
        }
      } else {
        v[n2] = __ldg(reinterpret_cast<const float2*>(p.in) + boff + e);
      }
    }
    Dft<R2, SIGN>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      float2 w = __ldg(twid + ((n1 * k2) & (N - 1)));
      if (SIGN < 0) w.y = -w.y;
      sm[G::sidx(l, n1, k2)] = (k2 == 0) ? v[k2] : cmul(v[k2], w);
    }
  }
  __syncthreads();

  // ---- step 2: R2/T DFTs of length R1 per thread ----
#pragma unroll
  for (int q = 0; q < R2 / T; ++q) {
    const int k2 = j + T * q;
    float2 u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) u[n1] = sm[G::sidx(l, n1, k2)];
    Dft<R1, SIGN>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const long long e = lbase + (long long)(k2 + R2 * k1) * estride;
      if (OUTB == 1) {
        float* o = reinterpret_cast<float*>(p.out) + blocked_re(fpts + e, p.single0 + bj, p.nsingle);
        o[0] = u[k1].x;
        o[32] = u[k1].y;
      } else if (OUTB == 2) {
        const int s = p.single0 + 2 * bj;
        float* o = reinterpret_cast<float*>(p.out) + blocked_re(fpts + e, s, p.nsingle);
        o[0] = u[k1].x;
        o[32] = 0.0f;
        if (2 * bj + 1 < p.npack) {
          o = reinterpret_cast<float*>(p.out) + blocked_re(fpts + e, s + 1, p.nsingle);
          o[0] = u[k1].y;
          o[32] = 0.0f;
        }
      } else {
        p.out[boff + e] = u[k1];
      }
    }
  }
  }  // arrays of the CTA
}

template <int N, bool CONTIG, int SIGN, int LOAD, int OUTB, int TLV, bool SLAB>
static cudaError_t launch_s(const FftPass& p, cudaStream_t st) {
  using G = Geo<N, CONTIG, TLV>;
  auto kern = fft_axis_kernel<N, CONTIG, SIGN, LOAD, OUTB, TLV, SLAB>;
  constexpr bool kBins = LOAD == LOAD_MUL || LOAD == LOAD_MUL2;
  constexpr int smem = kBins ? 2 * G::SMEM : G::SMEM;  // + the delta-hat slots
  {
    cudaError_t e = ensure_smem_attr<fft_axis_kernel<N, CONTIG, SIGN, LOAD, OUTB, TLV, SLAB>>(smem);
    if (e != cudaSuccess) return e;
  }
  // contiguous: outer rows grouped by TL; strided: outer * inner lines grouped by TL
  long long blocks = CONTIG ? p.outer / G::TL : (p.outer * (p.inner / G::TL));
  if (blocks <= 0 || blocks > 0x7fffffffLL || p.batch <= 0 || p.batch > 65535) return cudaErrorInvalidValue;
  if (p.nb_per_field < 0 || (p.nb_per_field && p.batch % p.nb_per_field)) return cudaErrorInvalidValue;
  if (CONTIG ? (p.outer % G::TL) : (p.inner % G::TL)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)blocks, (unsigned)p.batch);
  if constexpr (kBins) {
    // one CTA per (field, line group), looping over the field's arrays
    const long long nfld = SLAB ? p.batch / p.nb_per_field : 1;
    if (blocks * nfld > 0x7fffffffLL) return cudaErrorInvalidValue;
    grid = dim3((unsigned)(blocks * nfld), 1u);
  }
  kern<<<grid, G::THREADS, smem, st>>>(p);
  return cudaGetLastError();
}

// Strided passes of N >= 128 take the lines-per-CTA variant p.tl (0 default,
// 1 half, 2 twice; N = 1024: 0 and 1); the other passes have one variant.
// Passes that index by field (the product's factors, the blocked-store output)
// have a slab variant, taken when p.nb_per_field is set; single fields keep
// the plain index arithmetic (and its registers).
template <int N, bool CONTIG, int SIGN, int LOAD, int OUTB, int TLV>
static cudaError_t launch_v(const FftPass& p, cudaStream_t st) {
  if constexpr (LOAD == LOAD_MUL || LOAD == LOAD_MUL2 || OUTB != 0)
    if (p.nb_per_field) return launch_s<N, CONTIG, SIGN, LOAD, OUTB, TLV, true>(p, st);
  return launch_s<N, CONTIG, SIGN, LOAD, OUTB, TLV, false>(p, st);
}

template <int N, bool CONTIG, int SIGN, int LOAD, int OUTB = 0>
static cudaError_t launch_t(const FftPass& p, cudaStream_t st) {
  if constexpr (!CONTIG && N >= 128) {
    if (p.tl == 1) return launch_v<N, CONTIG, SIGN, LOAD, OUTB, 1>(p, st);
    // twice the lines at N = 1024 would stage 128 KB per CTA and spill registers;
    // product passes stage their delta-hat values as well (256 KB at N = 512)
    constexpr bool kBins = LOAD == LOAD_MUL || LOAD == LOAD_MUL2;
    if constexpr (N <= 512 && !(kBins && N >= 512))
      if (p.tl == 2) return launch_v<N, CONTIG, SIGN, LOAD, OUTB, 2>(p, st);
  }
  if (p.tl < 0 || p.tl > 2) return cudaErrorInvalidValue;
  return launch_v<N, CONTIG, SIGN, LOAD, OUTB, 0>(p, st);
}

template <int N>
static cudaError_t dispatch_n(const FftPass& p, cudaStream_t st) {
  const bool contig = (p.inner == 1);
  if (contig) {
    if (p.load != LOAD_COMPLEX) return cudaErrorInvalidValue;
    if (p.out_blocked) {
      if (p.sign < 0) return cudaErrorInvalidValue;
      if (p.out_blocked == 2) {
        if (p.npack < 1 || p.npack > 2 * p.batch) return cudaErrorInvalidValue;
        return launch_t<N, true, 1, LOAD_COMPLEX, 2>(p, st);
      }
      return launch_t<N, true, 1, LOAD_COMPLEX, 1>(p, st);
    }
    return p.sign < 0 ? launch_t<N, true, -1, LOAD_COMPLEX>(p, st) : launch_t<N, true, 1, LOAD_COMPLEX>(p, st);
  }
  if (p.out_blocked) return cudaErrorInvalidValue;
  if (p.sign < 0) {
    if (p.load == LOAD_REAL) return launch_t<N, false, -1, LOAD_REAL>(p, st);
    if (p.load == LOAD_COMPLEX) return launch_t<N, false, -1, LOAD_COMPLEX>(p, st);
    return cudaErrorInvalidValue;
  }
  if (p.load == LOAD_MUL) return launch_t<N, false, 1, LOAD_MUL>(p, st);
  if (p.load == LOAD_MUL2) {
    if (p.npack < 1 || p.npack > 2 * p.batch) return cudaErrorInvalidValue;
    return launch_t<N, false, 1, LOAD_MUL2>(p, st);
  }
  if (p.load == LOAD_COMPLEX) return launch_t<N, false, 1, LOAD_COMPLEX>(p, st);
  return cudaErrorInvalidValue;
}

cudaError_t fft_axis_pass(int n, const FftPass& p, cudaStream_t st) {
  switch (n) {
    case 8: return dispatch_n<8>(p, st);
    case 16: return dispatch_n<16>(p, st);
    case 32: return dispatch_n<32>(p, st);
    case 64: return dispatch_n<64>(p, st);
    case 128: return dispatch_n<128>(p, st);
    case 256: return dispatch_n<256>(p, st);
    case 512: return dispatch_n<512>(p, st);
    case 1024: return dispatch_n<1024>(p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbg
