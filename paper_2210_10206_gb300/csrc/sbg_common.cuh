// Shared device/host helpers of the GB300 SARABANDE library (internal header).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace sbg {

struct cplx { float x, y; };

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Launch-time knobs shared by the FFT launchers.
// LOAD_MUL2: batch j multiplies `shared` by mul_{2j} + i mul_{2j+1} (mul_{2j+1}
// taken as 0 past npack arrays), so that two transforms with real results share
// one complex transform
enum FftLoad { LOAD_COMPLEX = 0, LOAD_REAL = 1, LOAD_MUL = 2, LOAD_MUL2 = 3 };

// One axis pass of a batched 3D/2D complex FFT.  The array is viewed as
// [batch][outer][N][inner]; the pass transforms along the N axis.
struct FftPass {
  const void* in;        // float2 (or float for LOAD_REAL) base of batch 0
  float2* out;           // base of batch 0 (may alias `in`)
  const float2* mul;     // LOAD_MUL: per-batch factor array (batch stride = bstride)
  const float2* shared;  // LOAD_MUL: array common to every batch (e.g. delta-hat)
  const float2* twiddle; // N-entry table exp(sign 2 pi i j / N)
  long long outer, inner;
  long long bstride;     // elements between batches (in, out and mul)
  int batch;
  int sign;              // -1 forward, +1 inverse (unnormalised)
  int load;              // FftLoad
  // Contiguous (last) pass only: with out_blocked = 1, batch b of the output
  // goes to the blocked coefficient store as single s = single0 + b (see
  // blocked_re); with out_blocked = 2 (the packed batches of LOAD_MUL2), the
  // real part of batch b goes to single0 + 2b and the imaginary part to
  // single0 + 2b + 1 (if 2b + 1 < npack), each with imaginary part 0.
  int out_blocked;
  int npack;
  int nsingle;
  int single0;
  // Strided passes only: skip line groups that are known to be all zero (a
  // kernel whose support lies within minimum-image distance prune_r of the
  // origin on every axis; the skipped lines must already hold zeros).
  //   prune_mode 1: inner index = y * N + x (first pass of a 3D transform);
  //   prune_mode 2: inner index = x (second pass).
  int prune_mode;
  int prune_r;
  // A slab of fields (0: one field): batch b is array b % nb_per_field of
  // field b / nb_per_field; the factor array of LOAD_MUL / LOAD_MUL2 is taken
  // per array of a field (offset (b % nb_per_field) bstride), `shared` per
  // field (offset (b / nb_per_field) shared_stride), and a blocked-store
  // output puts field f's points at f field_points onwards.
  int nb_per_field;
  long long shared_stride;
  long long field_points;
  // Strided passes of N >= 128: lines per CTA, 0 the default, 1 half of it,
  // 2 twice it (chosen by measurement, see the context's autotuner).
  int tl;
};

// Blocked coefficient store (float view): for each 32-point K-block xb and
// single s, 64 floats [Re x0..x31][Im x0..x31] at ((xb * nsingle + s) * 64).
// One K-block of every single is one contiguous slab, and real and imaginary
// parts of neighbouring points are adjacent (packed f32x2 arithmetic).
__host__ __device__ __forceinline__ long long blocked_re(long long x, int s, int nsingle) {
  return ((x >> 5) * nsingle + s) * 64 + (x & 31);
}

// Streaming multiprocessors of the current device (queried once per device).
inline int device_sms() {
  static std::atomic<int> sms[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return 1;
  }
  if (dev >= 64) {
    int n = 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  int n = sms[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return 1;
    }
    sms[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// Opt kernel K in to `bytes` of dynamic shared memory on the current device.
// The attribute belongs to the device's context, so it is set once per device
// (and per kernel), not once per process.
template <auto K>
cudaError_t ensure_smem_attr(int bytes) {
  static std::atomic<unsigned long long> done{0};  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Host launcher (sbg_fft.cu).  Returns cudaSuccess or the launch error.
cudaError_t fft_axis_pass(int n, const FftPass& p, cudaStream_t st);

}  // namespace sbg
