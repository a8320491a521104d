// Internal declarations of the non-FFT kernels (launchers live in sbg_kernels.cu).
#pragma once
#include "sbg_common.cuh"

namespace sbg {

// ---- preprocessing (Sec. 4.1 mean subtraction; Eq. num_gals) ----
// acc[0] += sum(x); then out = float(x - mean) and acc[1] += sum(x - mean + 1).
// A slab of nfld fields of n values each (field f at in + f n, out + f n) uses
// acc[2f] and acc[2f + 1].
cudaError_t launch_sum(const void* in, int is_f64, long long n, double* acc, cudaStream_t st, int nfld = 1);
cudaError_t launch_convert(const void* in, int is_f64, long long n, const double* acc, int subtract,
                           float* out, cudaStream_t st, int nfld = 1);

// ---- kernel generation (Algorithms 1-2) ----
// 3D: out[b][cell] = conj(Y_lm(r_hat)) Theta_b(|r|) * scale for b < nb (buffer pre-zeroed).
cudaError_t launch_kgen3d(int n, int l, int m, double norm_lm, const double* e2_dev, int nb, double scale,
                          float2* out, cudaStream_t st);
// 2D: out[b][cell] = conj(((x+iy)/rho)^m) Theta_b(rho) * scale.
cudaError_t launch_kgen2d(int n, int m, const double* e2_dev, int nb, double scale, float2* out,
                          cudaStream_t st);

// ---- 3PCF Gram (Eq. alm_to_zeta_clean / proj_3pcf_coeff, Algorithms 5 and 7) ----
// S[b1][b2] += sum_x delta(x) a_b1(x) conj(a_b2(x)) for b1 <= b2, complex double.
// nsingle > 0: `a` is the blocked coefficient store and bin b is single single0 + b;
// nsingle = 0: `a` is [nb][ng].
// A slab of nfld fields of ng points: field f's bins follow field f - 1's in
// the [field][bin][x] buffer (nsingle = 0) or its points follow in the blocked
// store; delta + f ng; S + f s_stride (doubles).
cudaError_t launch_gram3(const float2* a, long long ng, int nb, const float* delta, double* S, int nsingle,
                         int single0, cudaStream_t st, int nfld = 1, long long s_stride = 0);

// ---- 4PCF pair x single contraction tables (Algorithms 6 and 8) ----
struct Tile4 {
  int row0, nrows;     // rows of the global row table
  int col0, ncols;     // cols of the global col table
  int uniq0, nuniq;    // staged singles (store indices); tensor-core tiles: sorted slot list
  int bgroup;          // tensor-core tiles: the B image (column group) of the tile
  int pad;
  long long tout;      // offset (in outputs) of this tile's [nrows][ncols] block of T
};
struct Row4 {
  int u1, u2;          // local (tile) indices of the two singles
  int flags;           // bit0: conj first, bit1: conj second
  float sign;          // +-1 from a_{l,-m} = (-1)^m conj(a_{lm}) (3D)
};

// T[tile][r][c] (+)= sum_x delta * f1 * f2 * a_col: its real part
// (complex_out 0), complex value (1, two doubles per entry) or imaginary part
// (2).  nsplit <= 0: x-splits per tile chosen to fill whole waves of nsm SMs.
// A slab of nfld fields (ng = nfld x the points of one field): each field is
// split alike and adds into T + f t_field_stride (doubles).
cudaError_t launch_simt4(const float2* astore, long long ng, const float* delta, const Tile4* tiles,
                         int ntiles, const Row4* rows, const int* cols, const int* uniq, int complex_out,
                         int tcg, int nsplit, int nsingle, double* T, int nsm, cudaStream_t st, int nfld = 1,
                         long long t_field_stride = 0);

// Tensor-core (tcgen05) split-BF16 version of the same contraction (sbg_tc.cu).
// Tiles of <= 128 rows whose row singles (<= kTcMaxRowSlots, in the slot order
// given by `slots`, -1 for an unused slot) are staged per K-block.  The tiles
// of one column group share their columns (<= 64 B rows: 3D one per column,
// 2D two); per K-block the group's B operand is an image of n hi rows then n
// lo rows of 128 bytes (n = B rows rounded up to 16) at byte `off` of the
// K-block's img_stride-byte slab of `bimg` (nkb * img_stride bytes, written by
// the launcher).  tf32 != 0 selects split TF32 products: every image, offset
// and stride is twice as large (bimg must hold 2 * nkb * img_stride bytes).
// *err is set (never cleared) if a bounded wait inside the kernel expired:
// every wait gives up after wait_ns of the GPU's global timer.  stall != 0
// withholds the kernel's MMA issuer, so that the other roles' waits run out (a
// host-side test of the timeout path; nothing is computed).
constexpr int kTcMaxRowSlots = 56;  // row singles staged per K-block
constexpr int kSimtMaxUniq = 64;    // row singles staged per chunk by the FP32 SIMT kernel
constexpr int kTcEpoch = 256;       // K-blocks between progress checkpoints of the lag limiter
struct BGroup {
  int col0, ncols;     // columns (global col table)
  int n;               // B rows of each half (hi, lo) of the image (multiple of 8, <= 64)
  int pad;
  long long off;       // byte offset of the image in a K-block's slab
};
// A slab of fields (splits_per_field > 0): the points of the fields follow each
// other, each field is splits_per_field consecutive x-splits, and field f adds
// into T + f t_field_stride (doubles).
// Units (tile, x-split) are spread over a cooperative grid of one CTA per SM;
// cnt holds one progress counter per (round, epoch), zeroed by the caller.
// chunks_per_kb = 8 * sum of the groups' n.  complex_out as for launch_simt4:
// 1 takes two B columns per single, 2 one column of the form (Im v, Re v).
cudaError_t launch_tc4(const float2* astore, void* bimg, const BGroup* bgroups, int nbgroups, int chunks_per_kb,
                       long long img_stride, const float* delta, long long ng, const Tile4* tiles, int ntiles,
                       const Row4* rows, const int* cols, const int* slots, int nsingle, int complex_out,
                       int nsplit, double* T, int* cnt, int* err, int nsm, cudaStream_t st,
                       cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr, int tf32 = 0,
                       unsigned long long wait_ns = 1000000000ull, int stall = 0, int splits_per_field = 0,
                       long long t_field_stride = 0);

// Tensor-core (tcgen05) version of launch_gram3 (sbg_gram_tc.cu): the same
// S[b1][b2] (b1 <= b2, complex double, accumulated) from split-BF16 (tf32 = 0)
// or split-TF32 (tf32 = 1) products with FP32 accumulation in tensor memory
// over ranges of points and FP64 across ranges and CTAs.  nb <= 20, ng a
// multiple of 64.  *err is set (never cleared) if a bounded wait (wait_ns of
// the GPU's global timer) expired; stall != 0 withholds its MMA issuer (a
// host-side test of the timeout path).
// Slabs of nfld fields as for launch_gram3.  With ngroups > 1 (blocked store
// only) the nb singles from single0 are ngroups adjacent groups of nb / ngroups
// bins: only pairs within one group are kept, group k's S at S + k * g_stride.
constexpr int kGramTcMaxNb = 20;
cudaError_t launch_gram_tc(const float2* a, long long ng, int nb, const float* delta, double* S, int nsingle,
                           int single0, int tf32, int* err, int nsm, unsigned long long wait_ns, int stall,
                           cudaStream_t st, int nfld = 1, long long s_stride = 0, int ngroups = 1,
                           long long g_stride = 0);

// ---- kernel generation fused with the FFT (sbg_fft_fused.cu) ----
// One (l, m) group of nb bins of a 3D grid of side n whose kernel spectra are
// not cached: pass A generates conj(Y_lm) Theta_b * norm_scale on the `lines`
// (z n + y rows whose y^2 + z^2 <= e2nb) and transforms them along x into kbuf
// ([nb][n^3]); pass B transforms the planes |z| <= R along y in place; pass C
// transforms every column along z, multiplies by dhat and transforms back
// along z into out ([nb or (npack + 1) / 2][n^3]).  The inverse y and x passes
// follow (fft_axis_pass).
struct FusedGroup {
  int l, m, nb;
  double norm_scale;     // sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) / N_g
  const double* e2;      // device, nb + 1 snapped squared edges
  double e2nb;           // e2[nb] on the host
  const int* lines;      // device
  int nlines, R;         // R = max |z| of the support
  int npack;             // > 0: real arrays packed two per transform
  const float2* tw;
  float2* kbuf;
  const float2* dhat;
  float2* out;
};
cudaError_t launch_fused_group(int n, const FusedGroup& g, cudaStream_t st);

// ---- finalisation ----
// zeta[o] = sum_{e in [ptr[o], ptr[o+1])} coef[e] * T[idx[e]] (idx < 0: conj of T[-idx-1]).
// A slab of nfld fields: field f reads T + f t_stride (entries) and writes zeta + f nout.
cudaError_t launch_couple(const double* T, int complex_t, const int* ptr, const int* idx, const double* coef,
                          int nout, double* zeta, cudaStream_t st, int nfld = 1, long long t_stride = 0);
// 3PCF from Grams: full: zeta[l][b1][b2] = (-1)^l/sqrt(2l+1) (Re S_l0 + 2 sum_{m>0} Re S_lm);
// projected: zeta[m][b1][b2] = S_m (complex).  S is [npair][nb][nb][2] with b1 <= b2 filled.
// A slab of nfld fields: field f reads S + f s_stride (doubles) and writes its own zeta block.
cudaError_t launch_finish3(const double* S, int full, int lmax, int nb, double* zeta, cudaStream_t st, int nfld = 1,
                           long long s_stride = 0);
// zeta[i] /= N_gal * prod nbar V_b over the bin indices of output i (Eq. for the normalisation
// coefficient, Sec. 2.5).  order = 3 or 4; outputs laid out [..][b1][b2]([b3])[ncomp].
// A slab of nfld fields: field f's outputs follow field f - 1's, its N_gal is acc[2f + 1].
cudaError_t launch_normalize(double* zeta, long long nouter, int nb, int order, int ncomp, const double* acc,
                             double ng, const double* vbin_dev, cudaStream_t st, int nfld = 1);

}  // namespace sbg
