// Building blocks of the library's FFT passes (internal header): radix-2/4/8/16/32
// DFTs in registers, the two-step split N = R1 x R2 of a line of N points, and
// the twiddle constants exp(2 pi i j / 32) written out as values of cos / sin.
#pragma once
#include "sbg_common.cuh"

namespace sbg {

__device__ constexpr float kC32[32] = {
    1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
    7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
    0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
    -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
    -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
    -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f,
    0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
    7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
__device__ constexpr float kS32[32] = {
    0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
    7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f,
    1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
    7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
    0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
    -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
    -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
    -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f};

// exp(SIGN * 2 pi i e / R) for compile-time R <= 32
template <int R, int SIGN>
__device__ __forceinline__ float2 wsmall(int e) {
  const int j = ((e % R) * (32 / R)) & 31;
  return make_float2(kC32[j], SIGN * kS32[j]);
}

template <int R, int SIGN> struct Dft;

template <int SIGN> struct Dft<1, SIGN> {
  __device__ __forceinline__ static void run(float2*) {}
};
template <int SIGN> struct Dft<2, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <int SIGN> struct Dft<4, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    // W = exp(SIGN i pi/2) = SIGN * i;  W * t3 = SIGN * (-t3.y, t3.x)
    float2 wt3 = make_float2(-SIGN * t3.y, SIGN * t3.x);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, wt3);
    v[3] = csub(t1, wt3);
  }
};

// R = A * B in registers: n = a + A b, k = kb + B ka.
template <int A, int B, int SIGN>
__device__ __forceinline__ void dft_four_step(float2* v) {
  constexpr int R = A * B;
#pragma unroll
  for (int a = 0; a < A; ++a) {
    float2 t[B];
#pragma unroll
    for (int b = 0; b < B; ++b) t[b] = v[a + A * b];
    Dft<B, SIGN>::run(t);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) v[a + A * kb] = (a * kb) ? cmul(t[kb], wsmall<R, SIGN>(a * kb)) : t[kb];
  }
  float2 out[R];
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
    float2 u[A];
#pragma unroll
    for (int a = 0; a < A; ++a) u[a] = v[a + A * kb];
    Dft<A, SIGN>::run(u);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) out[kb + B * ka] = u[ka];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = out[i];
}

template <int SIGN> struct Dft<8, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { dft_four_step<2, 4, SIGN>(v); }
};
template <int SIGN> struct Dft<16, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { dft_four_step<4, 4, SIGN>(v); }
};
template <int SIGN> struct Dft<32, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { dft_four_step<4, 8, SIGN>(v); }
};

template <int N> struct Plan;
template <> struct Plan<8>    { static constexpr int R1 = 4,  R2 = 2;  };
template <> struct Plan<16>   { static constexpr int R1 = 4,  R2 = 4;  };
template <> struct Plan<32>   { static constexpr int R1 = 8,  R2 = 4;  };
template <> struct Plan<64>   { static constexpr int R1 = 8,  R2 = 8;  };
template <> struct Plan<128>  { static constexpr int R1 = 16, R2 = 8;  };
template <> struct Plan<256>  { static constexpr int R1 = 16, R2 = 16; };
template <> struct Plan<512>  { static constexpr int R1 = 16, R2 = 32; };
template <> struct Plan<1024> { static constexpr int R1 = 32, R2 = 32; };

}  // namespace sbg
