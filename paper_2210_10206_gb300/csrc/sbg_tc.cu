// Tensor-core (tcgen05, sm_103a) split-BF16 contraction of the 4PCF.
//
// For one tile of 128 rows r (pairs of singles) and N columns c (singles):
//     D[r][c] = sum_x Re( P_r(x) * delta(x) a_c(x) ),   P_r = sign f1 f2
// (Eq. mu of Sec. 2.3 / Eq. proj_4pcf_coeff of Sec. 2.4 before the coupling
// contraction).  As a real GEMM over K = 2 x-points: A[r][2x, 2x+1] = (Re P, Im P)
// and B[c][2x, 2x+1] = (Re(delta a), -Im(delta a)); 2D adds the column
// (Im(delta a), Re(delta a)) for Im.  Each operand is split into bf16 hi + lo
// and D += Ahi Bhi + Ahi Blo + Alo Bhi (three MMAs into one TMEM accumulator).
//
// Roles of a persistent CTA (one per SM):
//   warp 9     loader: cp.async.bulk of the raw FP32 inputs of each 32-point
//              K-block (delta and the tile's staged singles, which lie in a few
//              contiguous runs of the blocked coefficient store) into a 4-deep
//              ring, completion on mbarriers (expect_tx);
//   warps 0-7  producers: form the swizzled (SW128, K-major) bf16 hi/lo A and B
//              tiles of a K-block in a 2-deep ring; every 64 K-blocks they also
//              fold the TMEM accumulator into a second TMEM accumulator
//              (FP32 partial sums over at most 2048 points), and at the end of a
//              work item add it to T in FP64;
//   warp 8     MMA issuer: one thread issues 12 tcgen05.mma (M=128, K=16) per
//              K-block and commits to the mbarriers that free the operand stage
//              and publish the accumulator.
// Work units (tile, x-split) are dealt round-robin to a cooperative grid of one
// CTA per SM; the loaders of all CTAs advance through x together (a CTA may run
// at most two 256-K-block epochs ahead of the slowest), so that the singles of
// the current x-window are read from HBM once and then served from L2.
// Every wait is bounded (1 s of %globaltimer); on expiry the CTA records an
// error code, drains its own copies, frees TMEM and returns.
#include <algorithm>

#include "sbg_kernels.cuh"

namespace sbg {

namespace {

constexpr int kRS = 4;                 // raw stages
constexpr int kOS = 2;                 // operand stages
constexpr int kFlush = 64;             // K-blocks per inner accumulation range
constexpr int kKX = 32;                // grid points per K-block (64 bf16 = one 128-B row)
constexpr int kProd = 256;             // producer threads (warps 0..7)
constexpr int kThreads = kProd + 64;   // + MMA warp + loader warp
constexpr int kATile = 128 * 128;      // bytes of one 128-row bf16 K-block tile
constexpr int kBTile = 64 * 128;       // bytes of one <=64-row tile
constexpr int kOpStage = 2 * kATile + 2 * kBTile;
constexpr int kRawD = kKX * 4;
constexpr int kRawStage = kRawD + kTcMaxSlots * kKX * 8;
constexpr int kLag = 2;                // epochs a loader may run ahead of the slowest CTA
constexpr int kMeta = 256 + 3 * kTcMaxSlots * 4;  // barriers + run table
constexpr int kSmem = kOS * kOpStage + kRS * kRawStage + kMeta + 1024;
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false if this or another thread of the grid gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* err, int code) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  while (!mbar_try(b, parity)) {
    if (*err) return false;
    if (gtime() - t0 > kWaitNs) {
      atomicCAS((int*)err, 0, code);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// split (re, im) into bf16x2 hi and lo words (re in the low half)
__device__ __forceinline__ void split2(float re, float im, uint32_t& hi, uint32_t& lo) {
  hi = bf16x2_rn(re, im);
  const float hr = __uint_as_float(hi << 16), hi_ = __uint_as_float(hi & 0xffff0000u);
  lo = bf16x2_rn(re - hr, im - hi_);
}

__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  // K-major, 128-byte swizzle, 8-row groups 1024 B apart (SBO), version 1
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

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

__device__ __forceinline__ int n_mma(const Tile4& t, int cplx) {
  const int nb = cplx ? 2 * t.ncols : t.ncols;
  return (nb + 15) & ~15;
}

// Bounded wait for a global progress counter written by other CTAs.
__device__ __forceinline__ bool wait_count(const int* c, int target, volatile int* err, int code) {
  if (*(volatile const int*)c >= target) return true;
  const unsigned long long t0 = gtime();
  while (*(volatile const int*)c < target) {
    if (*err) return false;
    if (gtime() - t0 > kWaitNs) {
      atomicCAS((int*)err, 0, code);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
tc4_kernel(const float2* __restrict__ astore, long long ng, const float* __restrict__ delta,
           const Tile4* __restrict__ tiles, int ntiles, const Row4* __restrict__ rows,
           const int* __restrict__ colslot, const int* __restrict__ slots, int nsingle, int cplx, int nsplit,
           double* __restrict__ T, int* cnt, int* err_flag) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* op_base = sm;
  uint8_t* raw_base = sm + kOS * kOpStage;
  uint64_t* bars = (uint64_t*)(raw_base + kRS * kRawStage);
  uint64_t* raw_full = bars;
  uint64_t* raw_empty = bars + kRS;
  uint64_t* op_full = bars + 2 * kRS;
  uint64_t* op_empty = bars + 2 * kRS + kOS;
  uint64_t* acc_full = bars + 2 * kRS + 2 * kOS;
  uint32_t* tmem_slot = (uint32_t*)(acc_full + 1);
  int* run_start = (int*)(bars + 32);            // loader-private run table
  int* run_len = run_start + kTcMaxSlots;
  int* run_slot = run_len + kTcMaxSlots;
  volatile int* err = err_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long nunits = (long long)ntiles * nsplit;
  const long long nrounds = (nunits + gridDim.x - 1) / gridDim.x;
  const long long nk_unit = ((ng / kKX) + nsplit - 1) / nsplit;
  const int epochs = (int)((nk_unit + kTcEpoch - 1) / kTcEpoch);

  if (tid == 0) {
    for (int i = 0; i < kRS; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], kProd);
    }
    for (int i = 0; i < kOS; ++i) {
      mbar_init(&op_full[i], kProd);
      mbar_init(&op_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;  // inner accumulator at column 0, outer at column 64

  if (warp == 9) {
    // ------------------------------------------------------------- loader --
    uint32_t g = 0;
    bool ok = true;
    for (long long rd = 0; rd < nrounds && ok; ++rd) {
      const long long u = rd * gridDim.x + blockIdx.x;
      Unit it{0, 0, 0};
      Tile4 tl{};
      int nruns = 0;
      if (u < nunits) {
        it = unit_of(u, ntiles, nsplit, ng);
        tl = tiles[it.tile];
        if (lane == 0) {
          // runs of consecutive store indices in the tile's (sorted) slot list
          for (int k = 0; k < tl.nuniq; ++k) {
            const int v = slots[tl.uniq0 + k];
            if (nruns > 0 && v == run_start[nruns - 1] + run_len[nruns - 1]) {
              ++run_len[nruns - 1];
            } else {
              run_start[nruns] = v;
              run_len[nruns] = 1;
              run_slot[nruns] = k;
              ++nruns;
            }
          }
        }
        nruns = __shfl_sync(0xffffffffu, nruns, 0);
        __syncwarp();
      }
      const uint32_t bytes = kRawD + (uint32_t)tl.nuniq * kKX * 8;
      for (int e = 0; e < epochs && ok; ++e) {
        const long long ce = rd * epochs + e;  // global epoch index
        if (ce >= kLag) {
          int good = 1;
          if (lane == 0) good = wait_count(&cnt[ce - kLag], (int)gridDim.x, err, 13);
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
        }
        const int kb1 = min(it.nk, (e + 1) * kTcEpoch);
        for (int kb = e * kTcEpoch; kb < kb1; ++kb, ++g) {
          const int rs = g % kRS;
          const uint32_t ph = (g / kRS) & 1;
          int good = 1;
          if (lane == 0) good = mbar_wait(&raw_empty[rs], ph ^ 1, err, 11);
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
          uint8_t* st = raw_base + rs * kRawStage;
          if (lane == 0) mbar_expect_tx(&raw_full[rs], bytes);
          __syncwarp();
          const long long x = it.x0 + (long long)kb * kKX;
          const long long slab = (x >> 5) * (long long)nsingle;  // start of this K-block in the blocked store
          for (int r = lane; r <= nruns; r += 32) {
            if (r == nruns) {
              bulk_g2s(st, delta + x, kRawD, &raw_full[rs]);
            } else {
              bulk_g2s(st + kRawD + run_slot[r] * kKX * 8, astore + (slab + run_start[r]) * kKX,
                       (uint32_t)run_len[r] * kKX * 8, &raw_full[rs]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) atomicAdd(&cnt[ce], 1);
      }
    }
    // drain: wait (bounded) for every issued stage's copies to land
    if (lane == 0) {
      const uint32_t first = g > kRS ? g - kRS : 0;
      for (uint32_t h = first; h < g; ++h) mbar_wait(&raw_full[h % kRS], (h / kRS) & 1, err, 12);
    }
  } else if (warp == 8) {
    // ---------------------------------------------------------------- MMA --
    if (lane == 0) {
      uint32_t q = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const Unit it = unit_of(u, ntiles, nsplit, ng);
        const Tile4 tl = tiles[it.tile];
        const int N = n_mma(tl, cplx);
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        for (int kb = 0; kb < it.nk; ++kb, ++q) {
          const int os = q % kOS;
          if (!mbar_wait(&op_full[os], (q / kOS) & 1, err, 21)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = su32(op_base + os * kOpStage);
          const uint32_t a_hi = base, a_lo = base + kATile, b_hi = base + 2 * kATile, b_lo = b_hi + kBTile;
          const bool first = (kb % kFlush) == 0;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const uint32_t a = p == 2 ? a_lo : a_hi;
            const uint32_t b = p == 1 ? b_lo : b_hi;
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_bf16(tmem, sdesc(a + 32 * k), sdesc(b + 32 * k), idesc, (first && p == 0 && k == 0) ? 0u : 1u);
          }
          mma_commit(&op_empty[os]);
          if ((kb + 1) % kFlush == 0 || kb + 1 == it.nk) mma_commit(acc_full);
        }
      }
    }
  } else {
    // ---------------------------------------------------------- producers --
    const int j = tid & 7;       // 16-byte chunk = 4 grid points
    const int rb = tid >> 3;     // 0..31
    const int quarter = warp & 3, half = warp >> 2;
    uint32_t g = 0, q = 0, f = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const Unit it = unit_of(u, ntiles, nsplit, ng);
      const Tile4 tl = tiles[it.tile];
      const int N = n_mma(tl, cplx);
      int cslot[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int c = rb + 32 * k;
        const int cs = cplx ? (c >> 1) : c;
        cslot[k] = (c < N && cs < tl.ncols) ? colslot[tl.colslot0 + cs] : 0;
      }
      Row4 rw[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = rb + 32 * k;
        if (r < tl.nrows) rw[k] = rows[tl.row0 + r];
        else rw[k] = Row4{0, 0, 0, 0.f};
      }
      bool first_flush = true;
      for (int kb = 0; kb < it.nk; ++kb, ++g, ++q) {
        const int rs = g % kRS, os = q % kOS;
        if (!mbar_wait(&raw_full[rs], (g / kRS) & 1, err, 31) || !mbar_wait(&op_empty[os], ((q / kOS) & 1) ^ 1, err, 32)) {
          ok = false;
          break;
        }
        const uint8_t* raw = raw_base + rs * kRawStage;
        const float* D = (const float*)raw;
        const float4* U4 = (const float4*)(raw + kRawD);
        uint8_t* op = op_base + os * kOpStage;
        // ---- A: 4 rows x 4 points per thread ----
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = rb + 32 * k;
          uint4 hv = make_uint4(0, 0, 0, 0), lv = make_uint4(0, 0, 0, 0);
          if (r < tl.nrows) {
            const float4 p0 = U4[rw[k].u1 * 16 + 2 * j], p1 = U4[rw[k].u1 * 16 + 2 * j + 1];
            const float4 q0 = U4[rw[k].u2 * 16 + 2 * j], q1 = U4[rw[k].u2 * 16 + 2 * j + 1];
            float2 f1[4] = {{p0.x, p0.y}, {p0.z, p0.w}, {p1.x, p1.y}, {p1.z, p1.w}};
            float2 f2[4] = {{q0.x, q0.y}, {q0.z, q0.w}, {q1.x, q1.y}, {q1.z, q1.w}};
            const float s1 = (rw[k].flags & 1) ? -1.f : 1.f, s2 = (rw[k].flags & 2) ? -1.f : 1.f;
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float ar = f1[e].x, ai = s1 * f1[e].y, br = f2[e].x, bi = s2 * f2[e].y;
              const float pr = rw[k].sign * (ar * br - ai * bi);
              const float pi = rw[k].sign * (ar * bi + ai * br);
              split2(pr, pi, h[e], l[e]);
            }
            hv = make_uint4(h[0], h[1], h[2], h[3]);
            lv = make_uint4(l[0], l[1], l[2], l[3]);
          }
          *(uint4*)(op + swz(r, j)) = hv;
          *(uint4*)(op + kATile + swz(r, j)) = lv;
        }
        // ---- B: rows c of delta * a_col, 4 points per thread ----
        {
          const float4 d4 = ((const float4*)D)[j];
          const float dd[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int c = rb + 32 * k;
            if (c >= N) continue;
            const int cs = cplx ? (c >> 1) : c;
            const int part = cplx ? (c & 1) : 0;
            uint4 hv = make_uint4(0, 0, 0, 0), lv = make_uint4(0, 0, 0, 0);
            if (cs < tl.ncols) {
              const float4 c0 = U4[cslot[k] * 16 + 2 * j], c1 = U4[cslot[k] * 16 + 2 * j + 1];
              const float2 av[4] = {{c0.x, c0.y}, {c0.z, c0.w}, {c1.x, c1.y}, {c1.z, c1.w}};
              uint32_t h[4], l[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float vr = dd[e] * av[e].x, vi = dd[e] * av[e].y;
                if (part == 0) split2(vr, -vi, h[e], l[e]);
                else split2(vi, vr, h[e], l[e]);
              }
              hv = make_uint4(h[0], h[1], h[2], h[3]);
              lv = make_uint4(l[0], l[1], l[2], l[3]);
            }
            *(uint4*)(op + 2 * kATile + swz(c, j)) = hv;
            *(uint4*)(op + 2 * kATile + kBTile + swz(c, j)) = lv;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&op_full[os]);
        mbar_arrive(&raw_empty[rs]);
        // ---- fold the inner accumulator every kFlush K-blocks ----
        const bool last = kb + 1 == it.nk;
        if ((kb + 1) % kFlush == 0 || last) {
          if (!mbar_wait(acc_full, f & 1, err, 33)) {
            ok = false;
            break;
          }
          ++f;
          tc_fence_after();
          const int hc = N >> 1;  // columns of this thread's half
          const int row = quarter * 32 + lane;
          const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
          for (int c0 = 0; c0 < hc; c0 += 8) {
            const int col = half * hc + c0;
            float in[8], out[8];
            tmem_ld8(tmem + lane_addr + col, in);
            if (first_flush) {
#pragma unroll
              for (int e = 0; e < 8; ++e) out[e] = in[e];
            } else {
              tmem_ld8(tmem + lane_addr + 64 + col, out);
#pragma unroll
              for (int e = 0; e < 8; ++e) out[e] += in[e];
            }
            if (!last) {
              tmem_st8(tmem + lane_addr + 64 + col, out);
            } else if (row < tl.nrows) {
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int c = col + e;
                if (cplx) {
                  if ((c >> 1) < tl.ncols)
                    atomicAdd(&T[(tl.tout + (long long)row * tl.ncols + (c >> 1)) * 2 + (c & 1)], (double)out[e]);
                } else if (c < tl.ncols) {
                  atomicAdd(&T[tl.tout + (long long)row * tl.ncols + c], (double)out[e]);
                }
              }
            }
          }
          first_flush = false;
          tc_fence_before();
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

cudaError_t launch_tc4(const float2* astore, long long ng, const float* delta, const Tile4* tiles, int ntiles,
                       const Row4* rows, const int* colslot, const int* slots, int nsingle, int complex_out,
                       int nsplit, double* T, int* cnt, int* err, int nsm, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (ng % kKX) return cudaErrorInvalidValue;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc4_kernel, kThreads, kSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // every CTA takes part in every round so that the progress counters fill up
  const int grid = nsm;
  void* args[] = {(void*)&astore, (void*)&ng,     (void*)&delta, (void*)&tiles, (void*)&ntiles,
                  (void*)&rows,   (void*)&colslot, (void*)&slots, (void*)&nsingle, (void*)&complex_out,
                  (void*)&nsplit, (void*)&T,      (void*)&cnt,   (void*)&err};
  e = cudaLaunchCooperativeKernel((const void*)tc4_kernel, dim3(grid), dim3(kThreads), args, kSmem, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sbg
