// Projected 3PCF entry point that performs no device allocation.
//
// Some callers cannot allocate device memory during a measurement: code that
// runs inside a pre-sized memory pool or an allocator that must not be
// re-entered, and embedders whose device-memory policy forbids cudaMalloc
// after start-up.  sbg_projected3_noalloc runs the same kernels as the
// projected 3PCF of sbg_projected, with every intermediate buffer carved out of
// one file-scope __device__ array (kScratchBytes per device that loads this
// library, held until the process exits).  The caller passes the field and the
// output as device pointers.
#include <atomic>
#include <cmath>
#include <cstring>

#include "sarabande_gb300.h"
#include "sbg_kernels.cuh"

namespace {

constexpr int kMaxN = 256;
constexpr int kMaxBins = 10;
constexpr int kMaxM = 10;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
// layout of the scratch array (bytes), sized for the maxima above
constexpr size_t kOffAcc = 0;                                                // 8 doubles
constexpr size_t kOffE2 = kOffAcc + up(8 * 8);                               // nbins+1 doubles
constexpr size_t kOffTw = kOffE2 + up((kMaxBins + 1) * 8);                   // N float2
constexpr size_t kOffDelta = kOffTw + up((size_t)kMaxN * 8);                 // N^2 floats
constexpr size_t kOffDhat = kOffDelta + up((size_t)kMaxN * kMaxN * 4);       // N^2 float2
constexpr size_t kOffG = kOffDhat + up((size_t)kMaxN * kMaxN * 8);           // nbins N^2 float2
constexpr size_t kOffGroup = kOffG + up((size_t)kMaxBins * kMaxN * kMaxN * 8);
constexpr size_t kOffS = kOffGroup + up((size_t)kMaxBins * kMaxN * kMaxN * 8);
constexpr size_t kScratchBytes = kOffS + up((size_t)(kMaxM + 1) * kMaxBins * kMaxBins * 16);

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up (set-up) on the first call
// made with that device current.  In host code the name g_scratch is only a
// host-side stand-in, so kernels are always given this looked-up address.  The
// slots are atomic so that host threads making their first calls at once are
// safe (they store the same address).  A cudaDeviceReset unloads the module and
// may move the array: the cached address is not valid across a reset.
std::atomic<unsigned char*> g_addr[64];

sbg_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SBG_ERR_CUDA;
  unsigned char* a = g_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SBG_ERR_CUDA;
    }
    a = (unsigned char*)p;
    g_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return SBG_OK;
}

// The small host-computed tables of a call (snapped squared edges, twiddles),
// passed by value as a kernel parameter and written into the scratch array on
// the stream, so the call holds no host buffer that the GPU reads later.
struct HostTables {
  double e2[kMaxBins + 1];
  float2 tw[kMaxN];
  int nbins, n;
};

__global__ void tables_kernel(const HostTables t, double* e2d, float2* tw) {
  for (int i = threadIdx.x; i < t.n; i += blockDim.x) tw[i] = t.tw[i];
  if ((int)threadIdx.x <= t.nbins) e2d[threadIdx.x] = t.e2[threadIdx.x];
}

#define NA_CU(call)                         \
  do {                                      \
    if ((call) != cudaSuccess) {            \
      cudaGetLastError();                   \
      return SBG_ERR_CUDA;                  \
    }                                       \
  } while (0)

}  // namespace

extern "C" sbg_status sbg_projected3_noalloc(const void* field, sbg_dtype dtype, int64_t n, const double* edges,
                                             int nbins, int mmax, unsigned flags, double* zeta3, void* cuda_stream) {
  using namespace sbg;
  if (!field || !edges || !zeta3) return SBG_ERR_INVALID_ARG;
  if (dtype != SBG_F32 && dtype != SBG_F64) return SBG_ERR_INVALID_ARG;
  if (flags & ~(unsigned)SBG_SUBTRACT_MEAN) return SBG_ERR_INVALID_ARG;
  if (n < 8 || n > kMaxN || (n & (n - 1))) return SBG_ERR_UNSUPPORTED_SHAPE;
  if (nbins < 1 || nbins > kMaxBins || mmax < 0 || mmax > kMaxM) return SBG_ERR_INVALID_ARG;
  for (int i = 0; i <= nbins; ++i)
    if (!std::isfinite(edges[i])) return SBG_ERR_BIN_RANGE;
  if (edges[0] < 0) return SBG_ERR_BIN_RANGE;
  for (int i = 0; i < nbins; ++i)
    if (!(edges[i + 1] > edges[i])) return SBG_ERR_BIN_RANGE;
  if (!(edges[nbins] < 0.5 * (double)n)) return SBG_ERR_BIN_RANGE;

  unsigned char* s = nullptr;
  sbg_status st = scratch_for_current_device(&s);
  if (st != SBG_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int N = (int)n;
  const long long ng = (long long)N * N;
  double* acc = (double*)(s + kOffAcc);
  double* e2d = (double*)(s + kOffE2);
  float2* tw = (float2*)(s + kOffTw);
  float* delta = (float*)(s + kOffDelta);
  float2* dhat = (float2*)(s + kOffDhat);
  float2* G = (float2*)(s + kOffG);
  float2* grp = (float2*)(s + kOffGroup);
  double* S = (double*)(s + kOffS);

  // host tables: squared edges snapped to integers, twiddles
  HostTables ht{};
  ht.nbins = nbins;
  ht.n = N;
  for (int i = 0; i <= nbins; ++i) {
    double v = edges[i] * edges[i];
    const double r = std::nearbyint(v);
    if (std::fabs(v - r) <= 1e-9 * (v > 1.0 ? v : 1.0)) v = r;
    ht.e2[i] = v;
  }
  for (int j = 0; j < N; ++j) {
    const double a = 2.0 * 3.14159265358979323846 * j / N;
    ht.tw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  tables_kernel<<<1, 256, 0, stream>>>(ht, e2d, tw);
  NA_CU(cudaGetLastError());
  // the array keeps the previous call's contents: clear the accumulators
  NA_CU(cudaMemsetAsync(acc, 0, 8 * sizeof(double), stream));
  NA_CU(cudaMemsetAsync(S, 0, (size_t)(mmax + 1) * nbins * nbins * 16, stream));

  NA_CU(launch_sum(field, dtype == SBG_F64, ng, acc, stream));
  NA_CU(launch_convert(field, dtype == SBG_F64, ng, acc, (flags & SBG_SUBTRACT_MEAN) ? 1 : 0, delta, stream));
  FftPass p{};
  p.twiddle = tw;
  // delta-hat = FFT(delta): y pass (real input), x pass
  p.batch = 1; p.bstride = ng; p.sign = -1;
  p.in = delta; p.out = dhat; p.load = LOAD_REAL; p.outer = 1; p.inner = N;
  NA_CU(fft_axis_pass(N, p, stream));
  p.in = dhat; p.load = LOAD_COMPLEX; p.outer = N; p.inner = 1;
  NA_CU(fft_axis_pass(N, p, stream));
  for (int m = 0; m <= mmax; ++m) {
    // kernel spectra G^b_m = FFT_+(conj(e^{i m phi}) Theta_b) / N^2
    NA_CU(cudaMemsetAsync(G, 0, (size_t)nbins * ng * sizeof(float2), stream));
    NA_CU(launch_kgen2d(N, m, e2d, nbins, 1.0 / (double)ng, G, stream));
    FftPass q{};
    q.twiddle = tw; q.batch = nbins; q.bstride = ng; q.sign = +1;
    q.in = G; q.out = G; q.load = LOAD_COMPLEX; q.outer = 1; q.inner = N;
    NA_CU(fft_axis_pass(N, q, stream));
    q.outer = N; q.inner = 1;
    NA_CU(fft_axis_pass(N, q, stream));
    // c^b_m = IFFT(delta-hat G^b_m), product fused into the first pass
    FftPass c{};
    c.twiddle = tw; c.batch = nbins; c.bstride = ng; c.sign = +1;
    c.out = grp; c.mul = G; c.shared = dhat; c.load = LOAD_MUL; c.outer = 1; c.inner = N;
    NA_CU(fft_axis_pass(N, c, stream));
    c.in = grp; c.mul = nullptr; c.shared = nullptr; c.load = LOAD_COMPLEX; c.outer = N; c.inner = 1;
    NA_CU(fft_axis_pass(N, c, stream));
    NA_CU(launch_gram3(grp, ng, nbins, delta, S + (size_t)m * nbins * nbins * 2, 0, 0, stream));
  }
  NA_CU(launch_finish3(S, 0, mmax, nbins, zeta3, stream));
  return SBG_OK;
}
