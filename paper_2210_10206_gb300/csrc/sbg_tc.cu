// Tensor-core (tcgen05, sm_103a) split-BF16 contraction of the 4PCF.
//
// For one tile of 128 rows r (pairs of singles) and N columns c (singles):
//     D[r][c] = sum_x Re( P_r(x) * delta(x) a_c(x) ),   P_r = f1 f2
// (Eq. mu of Sec. 2.3 / Eq. proj_4pcf_coeff of Sec. 2.4 before the coupling
// contraction).  As a real GEMM over K = 64 per 32-point K-block:
// A[r] = (Re P, Im P), B[c] = (Re(delta a), -Im(delta a)) over the block's 32
// points (split BF16: Re and Im of points 8q..8q+7 in turn; split TF32: all
// Re, then all Im); 2D adds the column (Im(delta a), Re(delta a)) for Im.  Each operand is split into
// bf16 hi + lo and D += Ahi Bhi + Ahi Blo + Alo Bhi (three products summed in
// TMEM).  The row signs (-1)^m of a_{l,-m} are applied in the FP64
// coupling step, not here.
//
// B depends only on the column group (the columns shared by the tiles of one
// m3 block) and the K-block, so bimage_kernel writes it once per field as an
// image of the swizzled shared-memory tile; A depends on the row pair and is
// formed on chip.  Operand stage g (an A tile in TMEM plus a B tile in shared
// memory) belongs to producer group g, so every stage is filled by one group
// in order and no waiter can be two mbarrier phases ahead.  Roles of a
// persistent CTA (one per SM):
//   warps 0-15 producers, in 4 groups of 4 warps: group g takes the K-blocks
//              kb = g (mod 4) of every unit and writes their bf16 hi/lo A tile
//              (formed with packed f32x2 arithmetic from the FP32 singles in a
//              raw stage, one row per TMEM lane) straight into tensor memory.
//              Group 0 also folds each 256-K-block range's TMEM accumulator
//              into the outer TMEM accumulator (before it forms the first
//              K-block of the next range, which reuses the inner one) and, at
//              the end of a unit, adds it to T in FP64;
//   warp 16    MMA issuer: one thread issues 8 tcgen05.mma (M=128, K=16) per
//              K-block, Ahi [Bhi | Blo] (N = 2n) and Alo Bhi (N = n) per K step
//              (the cost of an MMA hardly grows with N up to 128, so fewer,
//              wider MMAs are faster), and commits to the mbarriers that free
//              the operand stage and publish the accumulator;
//   warps 17-18 loaders: per-thread 16-byte cp.async of each K-block's raw
//              FP32 row singles into two raw stages per producer group; each
//              thread's copies complete onto the stage's mbarrier (noinc);
//   warp 19    B loader: one bulk copy (cp.async.bulk) per K-block of the
//              tile's B image into the operand stage, once the MMAs that last
//              read that stage have completed.
// Work units (tile, x-split) are dealt round-robin to a cooperative grid of one
// CTA per SM; the loaders of all CTAs advance through x together (a CTA may run
// at most four 256-K-block epochs ahead of the slowest), so that the singles of
// the current x-window are read from HBM once and then served from L2.
// Every wait is bounded (wait_ns of %globaltimer, 1 s by default); on expiry
// the CTA records an error code, and before it frees TMEM and returns it drains
// what it has in flight: the B loader waits for its last bulk copy into each
// stage, the loaders for their cp.async copies and the MMA issuer for the
// completion of every MMA it issued (each drain with its own short bound, and
// whatever the error word says).
#include <algorithm>

#include "sbg_kernels.cuh"
#include "sbg_tcgen05.cuh"

namespace sbg {

namespace {

constexpr int kRS = 8;                // raw stages, split evenly over the producer groups
constexpr int kKX = 32;                // grid points per K-block (64 bf16 = one 128-B row)
constexpr int kProdWarps = 16;         // producer warps 0..15
constexpr int kMmaWarp = kProdWarps;   // warp 16
constexpr int kLoadWarps = 2;          // warps 17..18: raw A singles
constexpr int kLoad0 = kMmaWarp + 1;
constexpr int kLoaders = kLoadWarps * 32;
constexpr int kBWarp = kLoad0 + kLoadWarps;  // warp 19: B tiles
constexpr int kThreads = (kBWarp + 1) * 32;
// Per precision of the split products:
//   split BF16 (kind::f16): 4 producer groups of 4 warps, K = 16 per MMA, an A
//     tile of 64 TMEM columns (32 hi, 32 lo) and B rows of one 128-byte atom;
//   split TF32 (kind::tf32): 2 groups of 8 warps (two warps per TMEM lane
//     quarter, each forming half of the points), K = 8 per MMA, an A tile of
//     128 columns (64 hi, 64 lo) and B rows of two 128-byte atoms (K 0..31 and
//     32..63).
// Either way operand stage g belongs to group g, the A tiles fill TMEM columns
// [256, 512) and the B tiles 64 KB of shared memory.
template <bool TF>
struct Cfg {
  static constexpr int kGroups = TF ? 2 : 4;
  static constexpr int kWarps = 16 / kGroups;          // producer warps per group
  static constexpr int kParts = kWarps / 4;            // point ranges per TMEM lane quarter
  static constexpr int kOS = kGroups;                  // operand stages
  static constexpr int kRawPer = kRS / kGroups;        // raw stages per group
  static constexpr int kAtoms = TF ? 2 : 1;            // 128-byte swizzle atoms per B row (64 K values)
  static constexpr int kACols = 64 * kAtoms;           // TMEM columns of an A tile (hi then lo)
  static constexpr int kOpStage = 128 * 128 * kAtoms;  // B tile: n hi rows, then n lo rows (n <= 64)
  static constexpr int kKSteps = TF ? 8 : 4;           // MMA K steps per K-block
  static constexpr uint32_t kFmt = TF ? 2u : 1u;       // A/B format in the instruction descriptor
  // K-blocks per TMEM accumulation range before the fold into the outer
  // accumulator (FP32 with round-to-nearest on the CUDA cores).  The error of
  // the tensor core's accumulation grows with the range: measured on the 32^3
  // test field, split TF32 reaches 3.2e-5 of max|zeta| with 256-K-block ranges,
  // 7.6e-6 with 32 and 2.1e-6 with 8, at 240 / 250 / 282 ms per 256^3 field.
  // Split TF32 is the accurate option, so its ranges are 8 K-blocks; split BF16
  // keeps 256 (1.9e-5, its bf16 split dominates).
  static constexpr int kFlush = TF ? 8 : 256;
  // group 0 forms the first K-block of every range (it folds the previous one)
  static_assert(kFlush % kGroups == 0, "ranges must start on group 0's K-blocks");
};
// TMEM columns: the inner accumulator [0, 192) of the current range (columns
// [0, n) collect Ahi Bhi, [n, 2n) Ahi Blo, [2n, 3n) Alo Bhi, whose MMA writes
// up to column 2n + 64 <= 192 when n is rounded up to 16 there), the outer
// accumulator [192, 256), then the A stages in [256, 512) (per operand stage
// 64 columns for split BF16, 128 for split TF32).  Alo Bhi has columns of its
// own so that its MMAs do not wait for the Ahi MMAs before them: the two
// chains of dependent accumulations overlap in the tensor core.
constexpr int kTmemOuter = 192;
constexpr int kTmemA0 = 256;
constexpr int kTmemCols = 512;
// FP32 (re, im) row singles, 256 bytes each, padded to 272 bytes: chunk k of
// slot s then falls in bank quad (s + k) mod 8, so the eight rows a
// quarter-warp reads at once are conflict-free when their slots differ mod 8
constexpr int kRawRow = kKX * 8 + 16;
constexpr int kRawStage = kTcMaxRowSlots * kRawRow;
constexpr int kLag = 4;                // epochs a loader may run ahead of the slowest CTA
constexpr int kMeta = 512;             // barriers (2 kRS + 3 * 4 + 2) and the TMEM address
constexpr int kOpBytes = 4 * 128 * 128;  // B tiles of every operand stage (both precisions)
constexpr int kSmem = kOpBytes + kRS * kRawStage + kMeta + 1024;
struct Unit {
  int tile;
  long long x0;
  int nk;
};

// Unit u covers x-split u / ntiles of tile u % ntiles.
__device__ __forceinline__ Unit unit_of(long long u, int ntiles, int nsplit, long long ng) {
  Unit it;
  const int split = (int)(u / ntiles);
  it.tile = (int)(u % ntiles);
  const long long per = ((ng / kKX + nsplit - 1) / nsplit) * kKX;
  it.x0 = split * per;
  const long long x1 = min(ng, it.x0 + per);
  it.nk = it.x0 < x1 ? (int)((x1 - it.x0) / kKX) : 0;
  return it;
}

// n: B rows of each half of the tile's B image (its columns rounded up to 8);
// the Ahi MMA takes N = 2n (a multiple of 16), the Alo MMA N = n rounded up to
// 16 (its extra columns meet lo rows of B and are never read)
__device__ __forceinline__ int n_mma(const Tile4& t, int cplx) {
  const int nb = cplx ? 2 * t.ncols : t.ncols;
  return (nb + 7) & ~7;
}

// Bounded wait for a global progress counter written by other CTAs.
__device__ __forceinline__ bool wait_count(const int* c, int target, volatile int* err, int code,
                                           unsigned long long limit) {
  if (*(volatile const int*)c >= target) return true;
  const unsigned long long t0 = gtime();
  while (*(volatile const int*)c < target) {
    if (*err) return false;
    if (gtime() - t0 > limit) {
      atomicCAS((int*)err, 0, code);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}


__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
// arrive on `bar` once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

template <bool TF>
__global__ void __launch_bounds__(kThreads, 1)
tc4_kernel(const float* __restrict__ astore, const uint8_t* __restrict__ bimg, const BGroup* __restrict__ bgroups,
           long long img_stride, long long ng, const Tile4* __restrict__ tiles, int ntiles,
           const Row4* __restrict__ rows, const int* __restrict__ slots, int nsingle, int cplx, int nsplit,
           double* __restrict__ T, int* cnt, int* err_flag, unsigned long long wait_ns, int stall,
           int splits_per_field, long long t_field_stride) {
  using C = Cfg<TF>;
  constexpr int kGroups = C::kGroups, kOS = C::kOS, kOpStage = C::kOpStage, kRawPer = C::kRawPer;
  constexpr int kFlush = C::kFlush;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* op_base = sm;
  uint8_t* raw_base = sm + kOpBytes;
  uint64_t* bars = (uint64_t*)(raw_base + kRS * kRawStage);
  uint64_t* raw_full = bars;
  uint64_t* raw_empty = bars + kRS;
  uint64_t* op_full = bars + 2 * kRS;
  uint64_t* op_empty = bars + 2 * kRS + kOS;
  uint64_t* b_full = bars + 2 * kRS + 2 * kOS;    // B tile landed (transaction bytes)
  uint64_t* acc_full = b_full + kOS;              // a range's MMAs are complete
  uint64_t* mma_done = acc_full + 1;              // every MMA of this CTA is complete (drain)
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* err = err_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long nunits = (long long)ntiles * nsplit;
  const long long nrounds = (nunits + gridDim.x - 1) / gridDim.x;
  const long long nk_unit = ((ng / kKX) + nsplit - 1) / nsplit;
  const int epochs = (int)((nk_unit + kTcEpoch - 1) / kTcEpoch);

  if (tid == 0) {
    for (int i = 0; i < kRS; ++i) {
      mbar_init(&raw_full[i], kLoaders);              // one cp.async completion per loader thread
      mbar_init(&raw_empty[i], C::kWarps);            // one arrival per warp of the owning group
    }
    for (int i = 0; i < kOS; ++i) {
      mbar_init(&op_full[i], C::kWarps);
      mbar_init(&op_empty[i], 1);                     // tcgen05.commit
    }
    for (int i = 0; i < kOS; ++i) mbar_init(&b_full[i], 1);  // expect_tx arrival + bytes
    mbar_init(acc_full, 1);
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;  // base of the 512 allocated columns

  if (warp == kBWarp) {
    // ------------------------------------------------------------ B tiles --
    // One bulk copy per K-block of the tile's pre-swizzled B image (2n rows of
    // 128 bytes) into operand stage kb % 4, once the MMAs of K-block kb - 4 have
    // released it.
    if (lane == 0) {
      uint32_t issued[kOS] = {};
      bool ok = true;
      for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const Unit it = unit_of(u, ntiles, nsplit, ng);
        const Tile4 tl = tiles[it.tile];
        const BGroup bg = bgroups[tl.bgroup];
        const uint32_t bytes = (uint32_t)bg.n * 256 * C::kAtoms;
        for (int kb = 0; kb < it.nk; ++kb) {
          const int os = kb % kOS;
          if (!mbar_wait(&op_empty[os], (issued[os] & 1) ^ 1, err, 41, wait_ns)) {
            ok = false;
            break;
          }
          ++issued[os];
          mbar_expect_tx(&b_full[os], bytes);
          bulk_g2s(op_base + os * kOpStage, bimg + ((it.x0 >> 5) + kb) * img_stride + bg.off * C::kAtoms, bytes,
                   &b_full[os]);
        }
      }
      // every copy issued has landed before the CTA may exit (also after an error)
      for (int os = 0; os < kOS; ++os)
        if (issued[os]) mbar_drain(&b_full[os], (issued[os] - 1) & 1, err, 42);
    }
  } else if (warp >= kLoad0) {
    // ------------------------------------------------------------ loaders --
    const int li = tid - kLoad0 * 32;  // 0 .. kLoaders - 1
    const int ck = li & 15;            // 16-byte chunk within a 256-byte row
    const int rq = li >> 4;            // slots rq, rq + kLoaders / 16, ...
    constexpr int kSlotStep = kLoaders / 16;
    constexpr int kSlotIter = (kTcMaxRowSlots + kSlotStep - 1) / kSlotStep;
    uint32_t gcount[kGroups] = {};  // K-blocks loaded so far for each producer group
    bool ok = true;
    for (long long rd = 0; rd < nrounds && ok; ++rd) {
      const long long u = rd * gridDim.x + blockIdx.x;
      Unit it{0, 0, 0};
      Tile4 tl{};
      int asi[kSlotIter];
      if (u < nunits) {
        it = unit_of(u, ntiles, nsplit, ng);
        tl = tiles[it.tile];
      }
#pragma unroll
      for (int k = 0; k < kSlotIter; ++k) {
        const int sl = rq + kSlotStep * k;
        asi[k] = sl < tl.nuniq ? slots[tl.uniq0 + sl] : -1;
      }
      for (int e = 0; e < epochs && ok; ++e) {
        const long long ce = rd * epochs + e;  // global epoch index
        if (ce >= kLag) {
          int good = 1;
          if (lane == 0) good = wait_count(&cnt[ce - kLag], (int)gridDim.x * kLoadWarps, err, 13, wait_ns);
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
        }
        const int kb1 = min(it.nk, (e + 1) * kTcEpoch);
        for (int kb = e * kTcEpoch; kb < kb1; ++kb) {
          const int gg = kb % kGroups;
          const uint32_t n = gcount[gg]++;
          const int rs = kRawPer * gg + (int)(n % kRawPer);
          if (!warp_wait(&raw_empty[rs], ((n / kRawPer) & 1) ^ 1, err, 11, wait_ns)) {
            ok = false;
            break;
          }
          uint8_t* st = raw_base + rs * kRawStage;
          const long long xb = (it.x0 >> 5) + kb;  // K-block index in the blocked stores
#pragma unroll
          for (int k = 0; k < kSlotIter; ++k) {
            const int sl = rq + kSlotStep * k;
            if (asi[k] >= 0)
              cp_async16(st + sl * kRawRow + ck * 16, astore + (xb * nsingle + asi[k]) * 64 + ck * 4, 16);
          }
          cp_async_arrive(&raw_full[rs]);
        }
        __syncwarp();
        if (lane == 0) atomicAdd(&cnt[ce], 1);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA --
    // stall != 0 (a test of the timeout path): the issuer takes no work, so
    // every wait of the other roles runs out
    if (lane == 0 && !stall) {
      uint32_t uses[kOS] = {};
      bool ok = true;
      for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const Unit it = unit_of(u, ntiles, nsplit, ng);
        const Tile4 tl = tiles[it.tile];
        const int N = n_mma(tl, cplx), Nlo = (N + 15) & ~15;
        // BF16 inputs, FP32 accumulator, K-major A and B, M = 128; N = n
        // rounded up to 16 for Alo Bhi and N = 2n for Ahi [Bhi | Blo]
        const uint32_t idesc = (1u << 4) | (C::kFmt << 7) | (C::kFmt << 10) | ((uint32_t)(Nlo >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        const uint32_t idesc2 = (idesc & ~(0x3Fu << 17)) | ((uint32_t)((2 * N) >> 3) << 17);
        for (int kb = 0; kb < it.nk; ++kb) {
          const int os = kb % kOS;
          if (!mbar_wait(&op_full[os], uses[os] & 1, err, 21, wait_ns)) {  // A formed and (checked by a producer) B landed
            ok = false;
            break;
          }
          ++uses[os];
          tc_fence_after();
          // B descriptor of the stage; K step k starts 32 bytes further (+2 in
          // the descriptor's 16-byte address field, which cannot carry out)
          // (an atom of 2n rows x 128 B holds 32 K values, of 4 K steps for TF32)
          const uint64_t bd = sdesc(su32(op_base + os * kOpStage));
          const uint32_t a_hi = tmem + kTmemA0 + C::kACols * os, a_lo = a_hi + C::kACols / 2;
          const uint32_t acc0 = (kb % kFlush) == 0 ? 0u : 1u;
          // two MMAs per K step: Ahi meets Bhi and Blo in one (N = 2n) into
          // columns [0, 2n), Alo meets Bhi into [2n, 3n); a K step is 8 TMEM
          // columns of A in both precisions
#pragma unroll
          for (int k = 0; k < C::kKSteps; ++k) {
            const uint64_t bk = bd + 2 * (k & 3) + (uint64_t)((k >> 2) * 2 * N * 128 / 16);
            mma_ts<TF>(tmem, a_hi + 8 * k, bk, idesc2, k == 0 ? acc0 : 1u);
            mma_ts<TF>(tmem + 2 * N, a_lo + 8 * k, bk, idesc, k == 0 ? acc0 : 1u);
          }
          mma_commit(&op_empty[os]);
          if ((kb + 1) % kFlush == 0 || kb + 1 == it.nk) mma_commit(acc_full);
        }
      }
      // every MMA issued has completed before TMEM is freed (also after an error)
      mma_commit(mma_done);
      mbar_drain(mma_done, 0, err, 22);
    }
  } else {
    // ---------------------------------------------------------- producers --
    const int quarter = warp & 3;        // TMEM lane quarter = rows 32 quarter .. +31
    const int grp = warp / C::kWarps;    // producer group: K-blocks kb = grp (mod kGroups), stage grp
    const int part = (warp % C::kWarps) >> 2;  // which 32 / kParts points of the K-block this warp forms
    const int row = quarter * 32 + lane; // the A row (TMEM lane) this thread writes
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const int os = grp;
    uint32_t uses = 0;                   // K-blocks this group has produced so far
    uint32_t R = 0;                      // ranges of earlier units (group 0 bookkeeping)
    bool ok = true;
    for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const Unit it = unit_of(u, ntiles, nsplit, ng);
      const Tile4 tl = tiles[it.tile];
      const int N = n_mma(tl, cplx);
      const int nranges = (it.nk + kFlush - 1) / kFlush;
      // a slab of fields: the x-splits of a field are consecutive, its T follows the previous field's
      double* Tu = T + (splits_per_field ? (long long)(u / ntiles) / splits_per_field * t_field_stride : 0LL);
      const bool aval = row < tl.nrows;
      // a padding row repeats row 0: its accumulator row is never read out
      const Row4 rw = rows[tl.row0 + (aval ? row : 0)];
      const float s1 = (rw.flags & 1) ? -1.f : 1.f, s2 = (rw.flags & 2) ? -1.f : 1.f;
      const uint64_t as1 = pk(s1, s1), as2 = pk(s2, s2), ans2 = pk(-s2, -s2);
      const int r1 = rw.u1 * kRawRow, r2 = rw.u2 * kRawRow;  // the two singles in a raw stage
      int flushed = 0;                              // ranges of this unit already folded (group 0)
      // fold range i of this unit: inner accumulator -> outer (or -> T for the last range)
      auto fold = [&](int i) -> bool {
        const uint32_t Rg = R + i;
        if (!warp_wait(acc_full, Rg & 1, err, 33, wait_ns)) return false;
        tc_fence_after();
        const bool last = i + 1 == nranges;
        const uint32_t inner = tmem + lane_addr;
        const uint32_t outer = tmem + lane_addr + kTmemOuter;
        for (int c0 = 0; c0 < N; c0 += 8) {
          float in[8], lo[8], out[8];
          float lo2[8];
          tmem_ld8(inner + c0, in);
          tmem_ld8(inner + N + c0, lo);
          tmem_ld8(inner + 2 * N + c0, lo2);
#pragma unroll
          for (int e = 0; e < 8; ++e) in[e] += lo[e] + lo2[e];
          if (i == 0) {
#pragma unroll
            for (int e = 0; e < 8; ++e) out[e] = in[e];
          } else {
            tmem_ld8(outer + c0, out);
#pragma unroll
            for (int e = 0; e < 8; ++e) out[e] += in[e];
          }
          if (!last) {
            tmem_st8(outer + c0, out);
          } else if (aval) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int c = c0 + e;
              if (cplx) {
                if ((c >> 1) < tl.ncols)
                  atomicAdd(&Tu[(tl.tout + (long long)row * tl.ncols + (c >> 1)) * 2 + (c & 1)], (double)out[e]);
              } else if (c < tl.ncols) {
                atomicAdd(&Tu[tl.tout + (long long)row * tl.ncols + c], (double)out[e]);
              }
            }
          }
        }
        tc_fence_before();
        return true;
      };
      for (int kb = grp; kb < it.nk && ok; kb += kGroups) {
        // group 0 produces the first K-block of every range: fold the previous
        // range first, whose inner accumulator this range overwrites (the warps
        // of part 0 fold; the MMA waits for every warp of the group anyway)
        if (grp == 0 && part == 0 && kb % kFlush == 0 && kb / kFlush >= 1) {
          if (!fold(kb / kFlush - 1)) {
            ok = false;
            break;
          }
          flushed = kb / kFlush;
        }
        const int rs = kRawPer * grp + (int)(uses % kRawPer);
        if (!warp_wait(&raw_full[rs], (uses / kRawPer) & 1, err, 31, wait_ns) ||
            !warp_wait(&op_empty[os], (uses & 1) ^ 1, err, 32, wait_ns)) {
          ok = false;
          break;
        }
        ++uses;
        tc_fence_after();
        const uint8_t* raw = raw_base + rs * kRawStage;
        // ---- A: the 32 pair products of this thread's row, to TMEM ----
        const uint32_t acol = tmem + lane_addr + kTmemA0 + C::kACols * os;
#pragma unroll 1
        for (int cq = part * (4 / C::kParts); cq < (part + 1) * (4 / C::kParts); ++cq) {  // points 8 cq .. +7
          const float4* p1 = (const float4*)(raw + r1 + 32 * cq);  // Re at +0, Im at +128 bytes
          const float4* p2 = (const float4*)(raw + r2 + 32 * cq);
          const float4 ra0 = p1[0], ra1 = p1[1], ia0 = p1[8], ia1 = p1[9];
          const float4 rb0 = p2[0], rb1 = p2[1], ib0 = p2[8], ib1 = p2[9];
          const float fr1[8] = {ra0.x, ra0.y, ra0.z, ra0.w, ra1.x, ra1.y, ra1.z, ra1.w};
          const float fi1[8] = {ia0.x, ia0.y, ia0.z, ia0.w, ia1.x, ia1.y, ia1.z, ia1.w};
          const float fr2[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
          const float fi2[8] = {ib0.x, ib0.y, ib0.z, ib0.w, ib1.x, ib1.y, ib1.z, ib1.w};
          uint64_t prs[4], pis[4];
#pragma unroll
          for (int p2 = 0; p2 < 4; ++p2) {
            const uint64_t ar = pk(fr1[2 * p2], fr1[2 * p2 + 1]);
            const uint64_t ai = mul2(pk(fi1[2 * p2], fi1[2 * p2 + 1]), as1);
            const uint64_t br = pk(fr2[2 * p2], fr2[2 * p2 + 1]);
            const uint64_t bi0 = pk(fi2[2 * p2], fi2[2 * p2 + 1]);
            const uint64_t bi = mul2(bi0, as2), nbi = mul2(bi0, ans2);
            prs[p2] = fma2(ar, br, mul2(ai, nbi));   // ar br - ai bi
            pis[p2] = fma2(ar, bi, mul2(ai, br));    // ar bi + ai br
          }
          if constexpr (TF) {
            // A K order: Re x0..x31 then Im x0..x31, one tf32 per column; hi in
            // columns [0, 64), lo = value - hi in [64, 128)
            float hr[8], lr[8], hi[8], li[8];
#pragma unroll
            for (int p2 = 0; p2 < 4; ++p2) {
              float r0, r1, i0, i1;
              upk(prs[p2], r0, r1);
              upk(pis[p2], i0, i1);
              hr[2 * p2] = tf32_rna(r0); hr[2 * p2 + 1] = tf32_rna(r1);
              hi[2 * p2] = tf32_rna(i0); hi[2 * p2 + 1] = tf32_rna(i1);
              upk(sub2(prs[p2], pk(hr[2 * p2], hr[2 * p2 + 1])), lr[2 * p2], lr[2 * p2 + 1]);
              upk(sub2(pis[p2], pk(hi[2 * p2], hi[2 * p2 + 1])), li[2 * p2], li[2 * p2 + 1]);
            }
            tmem_st8_nw(acol + 8 * cq, hr);        // hi, real parts
            tmem_st8_nw(acol + 32 + 8 * cq, hi);   // hi, imaginary parts
            tmem_st8_nw(acol + 64 + 8 * cq, lr);   // lo, real parts
            tmem_st8_nw(acol + 96 + 8 * cq, li);   // lo, imaginary parts
          } else {
            // A K order: per 8 points (Re x0..x7, Im x0..x7), two bf16 per
            // column: hi in columns [8 cq, 8 cq + 8), lo 32 columns further,
            // one 8-column store each (half the store instructions of four
            // 4-column stores, which contend less with the MMAs' reads)
            uint32_t h[8], lw[8];
#pragma unroll
            for (int p2 = 0; p2 < 4; ++p2) {
              split_pair(prs[p2], h[p2], lw[p2]);
              split_pair(pis[p2], h[4 + p2], lw[4 + p2]);
            }
            tmem_st8u_nw(acol + 8 * cq, h);
            tmem_st8u_nw(acol + 32 + 8 * cq, lw);
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        // the first warp of the group also sees this K-block's B tile land, so
        // the MMA issuer waits on op_full alone (the copy of the stage's next
        // K-block needs this op_full first, so the parity cannot run ahead)
        if (warp % C::kWarps == 0 && !warp_wait(&b_full[os], (uses - 1) & 1, err, 34, wait_ns)) {
          ok = false;
          break;
        }
        // publish the A tile to the MMA issuer, release the raw stage
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&op_full[os]);
          mbar_arrive(&raw_empty[rs]);
        }
      }
      // group 0: fold the ranges not folded yet, the last one into T
      if (grp == 0 && part == 0 && ok) {
        for (int i = flushed; i < nranges && ok; ++i)
          if (!fold(i)) ok = false;
      }
      R += nranges;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// B image of every K-block: for each column group (the columns shared by the
// tiles of one m3 block), 2n rows of 64 values in the 128-byte-swizzled K-major
// layout the MMA reads, rows [0, n) the hi parts and rows [n, 2n) the lo parts
// of the B rows (3D column c: (Re v, -Im v) of single cols[col0 + c]; 2D column
// c: (Re v, -Im v) for even c and (Im v, Re v) for odd c of single
// cols[col0 + c / 2]; v = delta * a; zero past the group's columns).  BF16: one
// 128-byte atom per row; TF32: two atoms (K 0..31, then K 32..63), each 2n rows.
// One thread writes one 16-byte chunk of a hi row and of its lo row.
template <bool TF>
__global__ void bimage_kernel(const float* __restrict__ astore, const float* __restrict__ delta, long long nkb,
                              int nsingle, int cplx, const BGroup* __restrict__ groups, const int* __restrict__ cols,
                              int chunks_per_kb, long long img_stride, uint8_t* __restrict__ bimg) {
  constexpr int kAtoms = Cfg<TF>::kAtoms;
  constexpr int kPer = TF ? 4 : 8;  // values per 16-byte chunk
  const long long total = nkb * chunks_per_kb;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const long long xb = w / chunks_per_kb;
    int r = (int)(w - xb * chunks_per_kb);
    int g = 0;
    while (r >= groups[g].n * 8 * kAtoms) {
      r -= groups[g].n * 8 * kAtoms;
      ++g;
    }
    const BGroup bg = groups[g];
    const int c = r / (8 * kAtoms), j = r % (8 * kAtoms);
    const int atom = j >> 3, jj = j & 7;
    // the chunk's 8 (BF16) or 4 (TF32) K values: points p0.. of the real
    // (second = 0) or imaginary (second = 1) form.  BF16 K order: per 8 points
    // (Re, then Im), as the producers lay out A; TF32: Re x0..x31, Im x0..x31.
    const int second = TF ? atom : (jj & 1);
    const int p0 = TF ? 4 * jj : 8 * (jj >> 1);
    // columns of the (Im v, Re v) form: the odd ones of a complex group, and
    // every one of an imaginary-only group (cplx = 2)
    const bool imcol = cplx == 2 || (cplx == 1 && (c & 1));
    const int cs = cplx == 1 ? (c >> 1) : c;
    uint4 hi = make_uint4(0, 0, 0, 0), lo = make_uint4(0, 0, 0, 0);
    if (cs < bg.ncols) {
      const float* a = astore + (xb * nsingle + cols[bg.col0 + cs]) * 64;
      const float* ap = a + ((imcol ? !second : second) ? 32 : 0) + p0;
      const float* dp = delta + xb * 32 + p0;
      // component: Re v for (even, first half) and (odd, second half); Im v otherwise,
      // negated for (even, second half)
      const float sg = (!imcol && second) ? -1.f : 1.f;
      if constexpr (TF) {
        const float4 a0 = *(const float4*)ap, d0 = *(const float4*)dp;
        const float v[4] = {sg * (d0.x * a0.x), sg * (d0.y * a0.y), sg * (d0.z * a0.z), sg * (d0.w * a0.w)};
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          h[e] = tf32_rna(v[e]);
          l[e] = v[e] - h[e];
        }
        hi = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
        lo = make_uint4(__float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]), __float_as_uint(l[3]));
      } else {
        const float4 a0 = ((const float4*)ap)[0], a1 = ((const float4*)ap)[1];
        const float4 d0 = ((const float4*)dp)[0], d1 = ((const float4*)dp)[1];
        uint32_t h[4], l[4];
        split_pair(pk(sg * (d0.x * a0.x), sg * (d0.y * a0.y)), h[0], l[0]);
        split_pair(pk(sg * (d0.z * a0.z), sg * (d0.w * a0.w)), h[1], l[1]);
        split_pair(pk(sg * (d1.x * a1.x), sg * (d1.y * a1.y)), h[2], l[2]);
        split_pair(pk(sg * (d1.z * a1.z), sg * (d1.w * a1.w)), h[3], l[3]);
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
      }
      (void)kPer;
    }
    uint8_t* img = bimg + xb * img_stride + bg.off * kAtoms + atom * (2 * bg.n * 128);
    const int pos = (jj ^ (c & 7)) << 4;  // rows c and n + c share c & 7 (n is a multiple of 8)
    *(uint4*)(img + c * 128 + pos) = hi;
    *(uint4*)(img + (bg.n + c) * 128 + pos) = lo;
  }
}

template <bool TF>
cudaError_t launch_tc4_t(const float2* astore, void* bimg, const BGroup* bgroups, int chunks_per_kb,
                         long long img_stride, const float* delta, long long ng, const Tile4* tiles, int ntiles,
                         const Row4* rows, const int* cols, const int* slots, int nsingle, int complex_out,
                         int nsplit, double* T, int* cnt, int* err, int nsm, cudaStream_t st, cudaEvent_t ev_begin,
                         cudaEvent_t ev_end, unsigned long long wait_ns, int stall, int splits_per_field,
                         long long t_field_stride) {
  constexpr int kAtoms = Cfg<TF>::kAtoms;
  const long long stride = img_stride * kAtoms;  // the tables give BF16 image offsets
  // B images of every K-block, once per field
  {
    const long long nkb = ng / kKX;
    const int cpk = chunks_per_kb * kAtoms;
    long long blocks = (nkb * cpk + 255) / 256;
    if (blocks > (long long)nsm * 32) blocks = (long long)nsm * 32;
    bimage_kernel<TF><<<(unsigned)blocks, 256, 0, st>>>((const float*)astore, delta, nkb, nsingle, complex_out,
                                                        bgroups, cols, cpk, stride, (uint8_t*)bimg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = ensure_smem_attr<tc4_kernel<TF>>(kSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc4_kernel<TF>, kThreads, kSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const float* af = (const float*)astore;
  const uint8_t* bi = (const uint8_t*)bimg;
  const int ccols = complex_out == 1 ? 1 : 0;  // two B columns and complex T per single
  const int grid = nsm;  // every CTA takes part in every round so that the progress counters fill up
  void* args[] = {(void*)&af,    (void*)&bi,      (void*)&bgroups, (void*)&stride,     (void*)&ng,
                  (void*)&tiles, (void*)&ntiles,  (void*)&rows,    (void*)&slots,      (void*)&nsingle,
                  (void*)&ccols, (void*)&nsplit, (void*)&T,  (void*)&cnt,        (void*)&err,
                  (void*)&wait_ns, (void*)&stall, (void*)&splits_per_field, (void*)&t_field_stride};
  if (ev_begin && (e = cudaEventRecord(ev_begin, st)) != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel((const void*)tc4_kernel<TF>, dim3(grid), dim3(kThreads), args, kSmem, st);
  if (e != cudaSuccess) return e;
  if (ev_end && (e = cudaEventRecord(ev_end, st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc4(const float2* astore, void* bimg, const BGroup* bgroups, int nbgroups, int chunks_per_kb,
                       long long img_stride, const float* delta, long long ng, const Tile4* tiles, int ntiles,
                       const Row4* rows, const int* cols, const int* slots, int nsingle, int complex_out,
                       int nsplit, double* T, int* cnt, int* err, int nsm, cudaStream_t st, cudaEvent_t ev_begin,
                       cudaEvent_t ev_end, int tf32, unsigned long long wait_ns, int stall, int splits_per_field,
                       long long t_field_stride) {
  if (splits_per_field < 0 || (splits_per_field && nsplit % splits_per_field)) return cudaErrorInvalidValue;
  if (ntiles <= 0) return cudaSuccess;
  if (ng % kKX || nbgroups <= 0 || chunks_per_kb <= 0 || img_stride % 1024) return cudaErrorInvalidValue;
  if (tf32)
    return launch_tc4_t<true>(astore, bimg, bgroups, chunks_per_kb, img_stride, delta, ng, tiles, ntiles, rows, cols,
                              slots, nsingle, complex_out, nsplit, T, cnt, err, nsm, st, ev_begin, ev_end, wait_ns,
                              stall, splits_per_field, t_field_stride);
  return launch_tc4_t<false>(astore, bimg, bgroups, chunks_per_kb, img_stride, delta, ng, tiles, ntiles, rows, cols,
                             slots, nsingle, complex_out, nsplit, T, cnt, err, nsm, st, ev_begin, ev_end, wait_ns,
                             stall, splits_per_field, t_field_stride);
}

}  // namespace sbg
