// Tensor-core (tcgen05, sm_103a) delta-weighted Gram of one group of binned
// coefficients: the combination step of the 3PCF,
//     S^{b1 b2} = sum_x delta(x) a_b1(x) conj(a_b2(x)),  b1 <= b2,
// for the nb bins of one (l, m) (full 3PCF, Eq. alm_to_zeta_clean, Algorithm 5)
// or one m (projected 3PCF, Eq. proj_3pcf_coeff, Algorithm 7).
//
// As a real GEMM over the grid points: the R = 2 nb real rows
// u_{2b} = Re a_b, u_{2b+1} = Im a_b and their delta-weighted copies w = delta u
// give G = W U^T (R x R, symmetric), and
//     Re S^{b1 b2} = G[2b1][2b2] + G[2b1+1][2b2+1],
//     Im S^{b1 b2} = G[2b1+1][2b2] - G[2b1][2b2+1].
// Both operands are split into hi + lo parts (bf16 for SBG_PREC_BF16X3, tf32
// for SBG_PREC_TF32X3).  One MMA (M = 128, N = 4 nb rounded up to 16) per K
// step takes A = [W_hi; W_lo] (2R rows) against B = [U_hi | U_lo] (2R columns),
// so the four products W_hi U_hi, W_hi U_lo, W_lo U_hi and W_lo U_lo land in
// four quadrants of one TMEM accumulator and are summed when it is folded.  A
// and B are both formed on chip from the same coefficient values, so there is
// no operand image in HBM; per K-block (64 points for bf16, 32 for tf32: one
// 128-byte row per operand row) a CTA reads nb x 64 / 32 complex values and
// the delta values once.
//
// Roles of a CTA (one per SM, each on a contiguous range of K-blocks):
//   warp 0      loader: one thread issues the K-block's copies into a raw
//               stage, completing on the stage's mbarrier: one 2D TMA tile
//               (every bin's points of the K-block) from a group buffer in the
//               [bin][x] layout, or one bulk copy per 32-point block of the
//               blocked coefficient store, and one bulk copy of delta;
//   warp 1      MMA issuer: 4 tcgen05.mma (kind::f16 or kind::tf32, both
//               operands in shared memory) per K-block into one of two TMEM
//               accumulators (ranges of kFlush K-blocks alternate between them);
//   warps 2-9   producers, in 4 groups of 2 warps: group g forms the K-blocks
//               k = g (mod 4) of the CTA, the bf16 / tf32 hi and lo rows of W
//               and U (128-byte swizzled K-major tiles); it reads raw stage
//               k mod 6 into registers and frees it, then waits for operand
//               stage k mod 6, so four K-blocks are formed at once while the
//               MMAs of up to six drain;
//   warps 10-13 fold: per finished range, read the accumulator (one TMEM lane
//               quarter each), sum its quadrants in FP32 and add them to an FP64
//               accumulator in shared memory; at the end add this CTA's S^{b1 b2}
//               to the output with FP64 atomics.
// Every wait is bounded (wait_ns of %globaltimer); on expiry the CTA records an
// error code, drains the copies and MMAs it issued and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "sbg_kernels.cuh"
#include "sbg_tcgen05.cuh"

namespace sbg {

namespace {

template <bool TF>
struct GramCfg {
  static constexpr int kPts = TF ? 32 : 64;      // points per K-block (one 128-byte atom per row)
  static constexpr int kKSteps = 4;              // MMAs per K-block (K = 16 bf16 or 8 tf32)
  static constexpr uint32_t kFmt = TF ? 2u : 1u; // operand format in the instruction descriptor
  // K-blocks per TMEM accumulation range (8192 points for bf16; 256 for tf32,
  // whose 1e-5 target needs short FP32 accumulation chains in the tensor core)
  static constexpr int kFlush = TF ? 8 : 128;
};

constexpr int kGThreads = 448;
constexpr int kGLoadWarp = 0;
constexpr int kGMmaWarp = 1;
constexpr int kGProd0 = 2;
constexpr int kGProdWarps = 8;
constexpr int kGGroups = 4;                    // producer groups = operand stages
constexpr int kGGroupWarps = kGProdWarps / kGGroups;
constexpr int kGFold0 = 10;
constexpr int kGFoldThreads = 128;
constexpr int kGMaxNb = kGramTcMaxNb;
constexpr int kGMaxR = 2 * kGMaxNb;            // real rows per operand half
// K-block k goes through raw stage k % kGRaw and operand stage k % kGOps,
// formed by producer group k % kGGroups: a stage's next user is another group,
// so a group never waits for the MMAs of its own previous K-block
constexpr int kGRaw = 6;                       // raw stages
constexpr int kGOps = 6;                       // operand stages
// One operand tile holds 2R <= 80 rows of 128 bytes; A (M = 128) is followed by
// B, so the MMA's reads of A rows 80..127 fall on B rows (their products land
// in accumulator rows the fold never reads), and B rows past 2R (read when N
// is padded to 16) were zeroed at the start and are never written.
constexpr int kGTile = 2 * kGMaxR * 128;
// A raw stage holds every bin's points of a K-block (1024-byte aligned, as the
// 128-byte swizzle of the tiled copy needs); the stages' delta values follow
// all of them, 256 bytes each.
constexpr int kGRawBytes = kGMaxNb * 64 * 8;
constexpr int kGDeltaBytes = 256;
constexpr int kGScratch = 2 * kGMaxR * 2 * kGMaxR * 4;  // FP32 rows of one folded range [2R][2R]
constexpr int kGAcc = kGMaxR * kGMaxR * 8;               // FP64 G [R][R]
constexpr int kGMeta = 256;                    // barriers, TMEM address, fold flag
constexpr int kGSmem = kGOps * 2 * kGTile + kGRaw * (kGRawBytes + kGDeltaBytes) + kGScratch + kGAcc + kGMeta + 1024;
static_assert(kGTile % 1024 == 0 && kGRawBytes % 1024 == 0, "raw stages must stay 1024-byte aligned");
constexpr int kGTmemCols = 256;                // two accumulators of <= 128 columns

template <bool TF>
__device__ __forceinline__ void mma_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

// 16 bytes at chunk c of row r of a 128-byte-swizzled K-major tile
__device__ __forceinline__ void st_chunk(uint8_t* tile, int r, int c, uint4 v) {
  *(uint4*)(tile + r * 128 + ((c ^ (r & 7)) << 4)) = v;
}

// hi/lo words of 8 values: bf16 (4 words each) or tf32 (8 words each, as FP32 bit patterns)
template <bool TF>
struct Split8 {
  uint32_t hi[TF ? 8 : 4], lo[TF ? 8 : 4];
};

template <bool TF>
__device__ __forceinline__ Split8<TF> split8(const float (&v)[8]) {
  Split8<TF> s;
  if constexpr (TF) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float h = tf32_rna(v[e]);
      s.hi[e] = __float_as_uint(h);
      s.lo[e] = __float_as_uint(v[e] - h);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) split_pair(pk(v[2 * e], v[2 * e + 1]), s.hi[e], s.lo[e]);
  }
  return s;
}

// 8 consecutive points (chunk q of 8 within the K-block) of one operand row
template <bool TF>
__device__ __forceinline__ void store8(uint8_t* tile, int row, int q, const uint32_t (&w)[TF ? 8 : 4]) {
  if constexpr (TF) {
    st_chunk(tile, row, 2 * q, make_uint4(w[0], w[1], w[2], w[3]));
    st_chunk(tile, row, 2 * q + 1, make_uint4(w[4], w[5], w[6], w[7]));
  } else {
    st_chunk(tile, row, q, make_uint4(w[0], w[1], w[2], w[3]));
  }
}

// 3D TMA tile (box of the tensor map) at element coordinates (x, y, z) into
// shared memory, completing as transaction bytes on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}

template <bool TF>
__global__ void __launch_bounds__(kGThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ a, long long ng, int nb,
               const float* __restrict__ delta,
               double* __restrict__ S, int nsingle, int single0, int* err_flag, unsigned long long wait_ns,
               int stall, long long s_stride, int gnb, long long g_stride) {
  using C = GramCfg<TF>;
  constexpr int kPts = C::kPts, kFlush = C::kFlush;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ops = sm;                                   // kGOps x (A tile, B tile)
  uint8_t* raw = ops + kGOps * 2 * kGTile;             // kGRaw raw stages
  uint8_t* draw = raw + kGRaw * kGRawBytes;             // kGRaw x delta of the stage's points
  float* scratch = (float*)(draw + kGRaw * kGDeltaBytes); // [2R][2R] FP32
  double* gacc = (double*)((uint8_t*)scratch + kGScratch);  // [R][R] FP64
  uint64_t* bars = (uint64_t*)((uint8_t*)gacc + kGAcc);
  uint64_t* raw_full = bars;                 // kGRaw
  uint64_t* raw_empty = raw_full + kGRaw;    // kGRaw
  uint64_t* op_full = raw_empty + kGRaw;     // kGOps
  uint64_t* op_empty = op_full + kGOps;      // kGOps
  uint64_t* d_full = op_empty + kGOps;       // 2
  uint64_t* d_free = d_full + 2;             // 2
  uint64_t* mma_done = d_free + 2;           // 1
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* fold_go = (volatile int*)(tmem_slot + 1);  // the fold warps' shared decision per range
  volatile int* err = err_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = 2 * nb;                                // real rows of W and of U
  const int N = (2 * R + 15) & ~15;                    // MMA N: [U_hi | U_lo] padded
  // field f = blockIdx.y of a slab of fields: its points follow field f - 1's
  // in the blocked store and delta, its bins in the [field][bin][x] buffer
  // (rows f nb .. f nb + nb - 1 of the tensor map), its S after field f - 1's
  const int fld = blockIdx.y;
  S += (long long)fld * s_stride;
  const long long nkb_all = ng / kPts;
  const long long per = (nkb_all + gridDim.x - 1) / gridDim.x;
  const long long kb0 = blockIdx.x * per;
  const int nk = (int)max(0LL, min(nkb_all, kb0 + per) - kb0);
  const int nranges = (nk + kFlush - 1) / kFlush;

  // zero the operand tiles (rows past 2R and columns past N stay zero) and G
  for (int i = tid; i < kGOps * 2 * kGTile / 16; i += kGThreads) ((uint4*)ops)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < R * R; i += kGThreads) gacc[i] = 0.0;
  if (tid == 0) {
    for (int i = 0; i < kGRaw; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], kGGroupWarps);
    }
    for (int i = 0; i < kGOps; ++i) {
      mbar_init(&op_full[i], kGGroupWarps);
      mbar_init(&op_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&d_full[i], 1);
      mbar_init(&d_free[i], 1);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kGTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zeroed tiles visible to the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kGLoadWarp) {
    // ---------------------------------------------------------------- loader --
    if (lane == 0) {
      uint32_t issued[kGRaw] = {};
      const uint32_t bytes = (uint32_t)(nb * kPts * 8 + kPts * 4);
      for (int k = 0; k < nk; ++k) {
        const int rs = k % kGRaw;
        if (!mbar_wait(&raw_empty[rs], ((k / kGRaw) & 1) ^ 1, err, 51, wait_ns)) break;
        ++issued[rs];
        uint8_t* st = raw + rs * kGRawBytes;
        const long long x0 = (kb0 + k) * kPts;
        mbar_expect_tx(&raw_full[rs], bytes);
        if (nsingle) {
          // blocked store: one contiguous run of nb singles per 32-point block
          for (int j = 0; j < kPts / 32; ++j) {
            const long long xb = (((long long)fld * ng + x0) >> 5) + j;
            bulk_g2s(st + j * nb * 256, a + (xb * nsingle + single0) * 64, (uint32_t)nb * 256, &raw_full[rs]);
          }
        } else {
          // rows b = 0 .. nb-1, 128-byte lines x0 / 16 .. x0 / 16 + kPts / 16 - 1
          // (floats 2 x0 .. 2 x0 + 2 kPts - 1), each line's 16-byte chunks
          // swizzled by its line index within the stage
          tma_load_3d(st, &tmap, 0, (int)(x0 / 16), fld * nb, &raw_full[rs]);
        }
        bulk_g2s(draw + rs * kGDeltaBytes, delta + (long long)fld * ng + x0, (uint32_t)kPts * 4, &raw_full[rs]);
      }
      // every copy issued has landed before the CTA may exit (also after an error)
      for (int rs = 0; rs < kGRaw; ++rs)
        if (issued[rs]) mbar_drain(&raw_full[rs], (issued[rs] - 1) & 1, err, 52);
    }
  } else if (warp == kGMmaWarp) {
    // ------------------------------------------------------------------- MMA --
    // stall != 0 (a test of the timeout path): the issuer takes no work, so
    // every wait of the other roles runs out
    if (lane == 0 && !stall) {
      // FP32 accumulator, K-major A and B, M = 128
      const uint32_t idesc = (1u << 4) | (C::kFmt << 7) | (C::kFmt << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      bool ok = true;
      for (int k = 0; k < nk && ok; ++k) {
        const int os = k % kGOps;
        const int r = k / kFlush, buf = r & 1;
        if (k % kFlush == 0 && r >= 2 && !mbar_wait(&d_free[buf], ((r >> 1) - 1) & 1, err, 53, wait_ns)) break;
        if (!mbar_wait(&op_full[os], (k / kGOps) & 1, err, 54, wait_ns)) break;
        tc_fence_after();
        const uint64_t ad = sdesc(su32(ops + os * 2 * kGTile));
        const uint64_t bd = sdesc(su32(ops + os * 2 * kGTile + kGTile));
        const uint32_t d = tmem + (uint32_t)(buf * 128);
#pragma unroll
        for (int s = 0; s < C::kKSteps; ++s)  // K step s starts 32 bytes further in every row
          mma_ss<TF>(d, ad + 2 * s, bd + 2 * s, idesc, (k % kFlush == 0 && s == 0) ? 0u : 1u);
        mma_commit(&op_empty[os]);
        if (k % kFlush == kFlush - 1 || k == nk - 1) mma_commit(&d_full[buf]);
      }
      // every MMA issued has completed before TMEM is freed (also after an error)
      mma_commit(mma_done);
      mbar_drain(mma_done, 0, err, 55);
    }
  } else if (warp < kGFold0) {
    // ------------------------------------------------------------- producers --
    // A thread's items (bin b, 8-point chunk q) of a K-block are it = ptid +
    // 64 u; they share q, hence delta.  The raw stage is read into registers
    // and released before the wait for the operand stage, so the loader can
    // refill it while the previous MMAs drain.
    constexpr int kGU = (kGMaxNb * (kPts / 8) + kGGroupWarps * 32 - 1) / (kGGroupWarps * 32);
    const int grp = (warp - kGProd0) / kGGroupWarps;         // producer group
    const int ptid = tid - (kGProd0 + grp * kGGroupWarps) * 32;  // thread within the group
    const int items = nb * (kPts / 8);
    const int q = ptid % (kPts / 8);
    for (int k = grp; k < nk; k += kGGroups) {
      const int rs = k % kGRaw, os = k % kGOps;
      // Raw stage rs alternates between two groups (6 stages, 4 groups), and
      // copies into different stages may land out of order.  So before the
      // parity wait for K-block k's copy, wait until the stage's previous
      // K-block (k - kGRaw, the other group's) has been read and released:
      // its copy has then landed, and raw_full cannot be two phases behind.
      if (k >= kGRaw && !warp_wait(&raw_empty[rs], ((k / kGRaw) - 1) & 1, err, 59, wait_ns)) break;
      if (!warp_wait(&raw_full[rs], (k / kGRaw) & 1, err, 56, wait_ns)) break;
      const uint8_t* st = raw + rs * kGRawBytes;
      float re[kGU][8], im[kGU][8], dl[8];
      {
        const uint8_t* dp = draw + rs * kGDeltaBytes + q * 32;
        const float4 d0 = *(const float4*)dp;
        const float4 d1 = *(const float4*)(dp + 16);
        dl[0] = d0.x; dl[1] = d0.y; dl[2] = d0.z; dl[3] = d0.w; dl[4] = d1.x; dl[5] = d1.y; dl[6] = d1.z; dl[7] = d1.w;
      }
#pragma unroll
      for (int u = 0; u < kGU; ++u) {
        const int it = ptid + u * kGGroupWarps * 32;
        if (it >= items) break;
        const int b = it / (kPts / 8);
        if (nsingle) {
          const float* p = (const float*)(st + (q / 4) * nb * 256 + b * 256) + (q % 4) * 8;
          const float4 r0 = *(const float4*)p, r1 = *(const float4*)(p + 4);
          const float4 i0 = *(const float4*)(p + 32), i1 = *(const float4*)(p + 36);
          re[u][0] = r0.x; re[u][1] = r0.y; re[u][2] = r0.z; re[u][3] = r0.w;
          re[u][4] = r1.x; re[u][5] = r1.y; re[u][6] = r1.z; re[u][7] = r1.w;
          im[u][0] = i0.x; im[u][1] = i0.y; im[u][2] = i0.z; im[u][3] = i0.w;
          im[u][4] = i1.x; im[u][5] = i1.y; im[u][6] = i1.z; im[u][7] = i1.w;
        } else {
          // 64 bytes from byte (b kPts + 8 q) 8 of the unswizzled tile: line
          // L = that / 128, chunks 4 (q & 1) + e, stored at chunk ^ (L & 7);
          // the 8 threads of a quarter warp hit 8 distinct bank groups
          const int line = (b * kPts + q * 8) >> 4;
          const uint8_t* lp = st + line * 128;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float4 v = *(const float4*)(lp + ((((q & 1) * 4 + e) ^ (line & 7)) << 4));
            re[u][2 * e] = v.x; im[u][2 * e] = v.y; re[u][2 * e + 1] = v.z; im[u][2 * e + 1] = v.w;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&raw_empty[rs]);  // its values are in registers
      if (!warp_wait(&op_empty[os], ((k / kGOps) & 1) ^ 1, err, 57, wait_ns)) break;
      tc_fence_after();
      uint8_t* at = ops + os * 2 * kGTile;  // A = [W_hi; W_lo]
      uint8_t* bt = at + kGTile;            // B = [U_hi | U_lo] (rows of the MMA's N)
#pragma unroll
      for (int u = 0; u < kGU; ++u) {
        const int it = ptid + u * kGGroupWarps * 32;
        if (it >= items) break;
        const int b = it / (kPts / 8);
        float wr[8], wi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          wr[e] = dl[e] * re[u][e];
          wi[e] = dl[e] * im[u][e];
        }
        const Split8<TF> ur = split8<TF>(re[u]), ui = split8<TF>(im[u]), vr = split8<TF>(wr), vi = split8<TF>(wi);
        store8<TF>(bt, 2 * b, q, ur.hi);
        store8<TF>(bt, 2 * b + 1, q, ui.hi);
        store8<TF>(bt, R + 2 * b, q, ur.lo);
        store8<TF>(bt, R + 2 * b + 1, q, ui.lo);
        store8<TF>(at, 2 * b, q, vr.hi);
        store8<TF>(at, 2 * b + 1, q, vi.hi);
        store8<TF>(at, R + 2 * b, q, vr.lo);
        store8<TF>(at, R + 2 * b + 1, q, vi.lo);
      }
      // generic-proxy stores -> visible to the tensor core, then publish
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&op_full[os]);
    }
  } else {
    // ------------------------------------------------------------------ fold --
    const int ft = tid - kGFold0 * 32;           // 0..127
    const int quarter = warp & 3;                // TMEM lane quarter of this warp
    const int row = quarter * 32 + lane;         // accumulator row (TMEM lane) of this thread
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const int R2 = 2 * R;
    bool ok = true;
    for (int r = 0; r < nranges && ok; ++r) {
      const int buf = r & 1;
      // one thread waits and all four warps take its outcome, so that they
      // pass the same named barriers (a barrier has no time limit)
      if (ft == 0) *fold_go = mbar_wait(&d_full[buf], (r >> 1) & 1, err, 58, wait_ns) ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"n"(kGFoldThreads) : "memory");
      if (!*fold_go) {
        ok = false;
        break;
      }
      tc_fence_after();
      // rows of [W_hi; W_lo] x columns of [U_hi | U_lo], FP32, to shared memory
      for (int c0 = 0; c0 < R2; c0 += 8) {
        float v[8];
        tmem_ld8(tmem + lane_addr + (uint32_t)(buf * 128 + c0), v);
        if (row < R2) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (c0 + e < R2) scratch[row * R2 + c0 + e] = v[e];
        }
      }
      tc_fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(kGFoldThreads) : "memory");
      if (ft == 0) mbar_arrive(&d_free[buf]);  // the accumulator may take the next range
      // G[i][j] = W_hi U_hi + W_hi U_lo + W_lo U_hi + W_lo U_lo
      for (int e = ft; e < R * R; e += kGFoldThreads) {
        const int i = e / R, j = e % R;
        const float g = scratch[i * R2 + j] + scratch[i * R2 + R + j] + scratch[(R + i) * R2 + j] +
                        scratch[(R + i) * R2 + R + j];
        gacc[e] += (double)g;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kGFoldThreads) : "memory");
    }
    // this CTA's S^{b1 b2} (b1 <= b2) into the output; with groups of gnb bins
    // stacked into one launch, only pairs within a group, each group's S
    // g_stride doubles after the previous one's
    if (ok && nranges > 0) {
      for (int p = ft; p < nb * nb; p += kGFoldThreads) {
        const int b1 = p / nb, b2 = p % nb;
        if (b1 > b2 || b1 / gnb != b2 / gnb) continue;
        const double sre = gacc[(2 * b1) * R + 2 * b2] + gacc[(2 * b1 + 1) * R + 2 * b2 + 1];
        const double sim = gacc[(2 * b1 + 1) * R + 2 * b2] - gacc[(2 * b1) * R + 2 * b2 + 1];
        double* Sg = S + (long long)(b1 / gnb) * g_stride + ((long long)(b1 % gnb) * gnb + b2 % gnb) * 2;
        atomicAdd(&Sg[0], sre);
        atomicAdd(&Sg[1], sim);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kGMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols));
}

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> fn{nullptr};
  PFN_cuTensorMapEncodeTiled_v12000 f = fn.load();
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    f = (PFN_cuTensorMapEncodeTiled_v12000)p;
    fn.store(f);
  }
  return f;
}

template <bool TF>
cudaError_t launch_gram_tc_t(const float2* a, long long ng, int nb, const float* delta, double* S, int nsingle,
                             int single0, int* err, int nsm, unsigned long long wait_ns, int stall, int nfld,
                             long long s_stride, int gnb, long long g_stride, cudaStream_t st) {
  cudaError_t e = ensure_smem_attr<gram_tc_kernel<TF>>(kGSmem);
  if (e != cudaSuccess) return e;
  constexpr int kPts = GramCfg<TF>::kPts;
  const long long nkb = ng / kPts;
  // CTAs per field: the SMs shared out over the fields
  const int grid = (int)std::max<long long>(1, std::min<long long>((nsm + nfld - 1) / nfld, nkb));
  CUtensorMap map;
  std::memset(&map, 0, sizeof map);
  if (!nsingle) {
    // group buffer [nb][ng] float2 as a 3D float tensor: 128-byte lines of 32
    // floats, ng / 16 lines per row, rows = bins (stride 8 ng bytes); a box of
    // every row's 2 kPts / 32 lines per K-block, 128-byte swizzled
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc || ng / 16 >= (1LL << 31)) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {32, (cuuint64_t)(ng / 16), (cuuint64_t)nb * nfld};
    const cuuint64_t strides[2] = {128, (cuuint64_t)ng * 8};
    const cuuint32_t box[3] = {32, (cuuint32_t)(2 * kPts / 32), (cuuint32_t)nb};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)a, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  gram_tc_kernel<TF><<<dim3(grid, nfld), kGThreads, kGSmem, st>>>(map, (const float*)a, ng, nb, delta, S, nsingle,
                                                                   single0, err, wait_ns, stall, s_stride, gnb,
                                                                   g_stride);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_tc(const float2* a, long long ng, int nb, const float* delta, double* S, int nsingle,
                           int single0, int tf32, int* err, int nsm, unsigned long long wait_ns, int stall,
                           cudaStream_t st, int nfld, long long s_stride, int ngroups, long long g_stride) {
  if (nb < 1 || nb > kGMaxNb || ng % 64 || !err || nfld < 1 || nfld > 65535) return cudaErrorInvalidValue;
  if (ngroups < 1 || nb % ngroups || (ngroups > 1 && !nsingle)) return cudaErrorInvalidValue;
  const int gnb = nb / ngroups;
  if (tf32)
    return launch_gram_tc_t<true>(a, ng, nb, delta, S, nsingle, single0, err, nsm, wait_ns, stall, nfld, s_stride, gnb,
                                  g_stride, st);
  return launch_gram_tc_t<false>(a, ng, nb, delta, S, nsingle, single0, err, nsm, wait_ns, stall, nfld, s_stride, gnb,
                                 g_stride, st);
}

}  // namespace sbg
