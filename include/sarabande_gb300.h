/*
 * sarabande_gb300.h -- C ABI of the GB300 (sm_103a) implementation of the hot
 * path of SARABANDE (Sunseri et al. 2022, arXiv 2210.10206): FFT-based 3- and
 * 4-point correlation functions of a periodic gridded density field.
 *
 * The pipeline behind every measurement call is the paper's (Sec. 3, Fig.
 * workflow): binned angular kernels (Algorithms 1-2) -> convolution
 * coefficients a^b_lm(x) / c^b_m(x) by FFT (Algorithms 3-4, Eq. almconv) ->
 * delta-weighted combination (Algorithms 5-8).  All work runs in CUDA kernels
 * of this library on one GPU.
 *
 * Conventions shared by every call:
 *  - Grid: periodic, C order, cell units (box side N, cell volume 1, Sec. 4.3).
 *    3D index (i, j, k) <-> (z, y, x); 2D (i, j) <-> (y, x).  phi = atan2(y, x),
 *    theta from +z; Y_lm orthonormal with the Condon-Shortley phase.
 *  - Bins: bin b holds the integer minimum-image offsets r with
 *    e_b^2 < |r|^2 <= e_{b+1}^2 (Algorithm 1 mask).  e^2 is computed in double
 *    and snapped to the nearest integer when within 1e-9 relative of it.
 *  - Coefficients are correlations a(x) = sum_r K(r) delta(x + r) (footnote to
 *    Eq. almconv), masks are 0/1 (no 1/V_b), outputs are sums over all grid
 *    points (Algorithms 5-8).  The full 3PCF carries (-1)^l / sqrt(2l+1)
 *    (Eq. alm_to_zeta_clean); the projected 3PCF has no 1/(2 pi)^2.
 *  - Ownership: the caller owns every pointer it passes.  The library never
 *    keeps a caller pointer after a call returns and never writes `field`.
 *  - Synchronicity: measurement calls return after the results are in the
 *    caller's host arrays.  Results are always float64 host arrays.
 *  - Threads: one context per host thread.
 *  - Errors: every call returns sbg_status; on error the output contents are
 *    unspecified and sbg_last_error() holds a one-line reason.
 */
#ifndef SARABANDE_GB300_H
#define SARABANDE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbg_context sbg_context;

typedef enum {
  SBG_OK = 0,
  SBG_ERR_INVALID_ARG = -1,       /* NULL pointer, bad count, bad flag or enum value */
  SBG_ERR_UNSUPPORTED_SHAPE = -2, /* side not a power of two in range, or not cubic/square */
  SBG_ERR_BIN_RANGE = -3,         /* edges not increasing, edges[0] < 0, or edges[nbins] >= N/2 */
  SBG_ERR_EMPTY_BIN = -4,         /* a bin holds no cell and SBG_NORMALIZED was asked for */
  SBG_ERR_OUT_OF_MEMORY = -5,     /* device allocation failed or exceeds the context budget */
  SBG_ERR_CUDA = -6,              /* a CUDA runtime call failed */
  SBG_ERR_TIMEOUT = -7,           /* a bounded device wait gave up */
  SBG_ERR_INTERNAL = -8
} sbg_status;

typedef enum { SBG_F32 = 0, SBG_F64 = 1 } sbg_dtype;

/* Arithmetic of the combination steps: the delta-weighted Gram of the 3PCF
 * (Algorithms 5, 7) and the pair x single contraction of the 4PCF (Algorithms
 * 6, 8).  FFTs are FP32, final sums and couplings FP64.
 * FP32: SIMT FP32 products and accumulation.
 * BF16X3: tcgen05 tensor cores, each operand split into bf16 hi + lo, products
 *         hi*hi + hi*lo + lo*hi (the 3PCF Gram also adds lo*lo), FP32
 *         accumulation in TMEM over ranges of points, FP64 across ranges.
 * TF32X3: the same with tf32 hi + lo (hi rounded to 10 mantissa bits, lo the
 *         exact remainder): more accurate, about twice the MMA work.
 * Value 2 is not used: a six-product bf16 split is not built, because the
 * three-product split already meets its 1e-4 target with margin and split
 * TF32 serves the 1e-5 target. */
typedef enum { SBG_PREC_FP32 = 0, SBG_PREC_BF16X3 = 1, SBG_PREC_TF32X3 = 3 } sbg_precision;

enum {
  SBG_3PCF = 1u,            /* NPCF = 3 (Sec. 3.3 `NPCF`)                          */
  SBG_4PCF = 2u,            /* NPCF = 4                                            */
  SBG_NORMALIZED = 4u,      /* divide by N_gal prod nbar V_bin (Sec. 2.5)          */
  SBG_SUBTRACT_MEAN = 8u,   /* delta <- delta - mean(delta) first (Sec. 4.1)       */
  SBG_FIELD_ON_DEVICE = 16u /* `field` is a device pointer of the context's device */
};

/* Create a context on CUDA device `cuda_device`.  hbm_budget_bytes caps the
 * device memory the context may hold (0: no cap beyond what is free).  The
 * context owns its buffers and cached plans until sbg_destroy. */
sbg_status sbg_create(int cuda_device, size_t hbm_budget_bytes, sbg_context** out);

/* Release every resource of `ctx`; NULL is accepted and ignored. */
void sbg_destroy(sbg_context* ctx);

/* Run subsequent work on `cuda_stream` (a cudaStream_t of the context's device,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL selects the context's
 * own stream.  The caller keeps the stream alive while the context uses it. */
sbg_status sbg_set_stream(sbg_context* ctx, void* cuda_stream);

/* Bound on every wait inside the tensor-core combination kernels of ctx
 * (SBG_PREC_BF16X3 and SBG_PREC_TF32X3), in nanoseconds of the GPU's global timer; the default is
 * 1e9 (1 s).  The kernel's roles hand work to each other through barriers in
 * shared memory; when a wait runs out, every role of the kernel stops, drains the
 * copies and tensor-core operations it has already issued (each drain bounded
 * too) and exits, and the measurement call returns SBG_ERR_TIMEOUT.  The context
 * stays usable.
 * test_stall = 1 withholds the kernels' MMA issuers in the following calls, so
 * that the other roles' waits run out: a way to exercise the timeout path from
 * the host without faulting the GPU (those calls compute nothing and return
 * SBG_ERR_TIMEOUT).  test_stall = 0 restores normal operation.
 * Errors: SBG_ERR_INVALID_ARG for a NULL ctx, wait_ns = 0 or test_stall not 0/1. */
sbg_status sbg_set_wait_limit(sbg_context* ctx, unsigned long long wait_ns, int test_stall);

/* Static string naming a status code. */
const char* sbg_status_string(sbg_status s);

/* Reason for the last failure on `ctx` (owned by ctx, valid until its next call). */
const char* sbg_last_error(const sbg_context* ctx);

/* Number of even-parity Lambda = (l1, l2, l3) with every l <= lmax, the loop
 * set of Algorithm 6 (23 at lmax 3, 42 at lmax 4).  lmax in 0..10. */
sbg_status sbg_lambda_count(int lmax, int* n_lambda);

/* The same list as 3 ints per entry (l1, l2, l3) in the order of the first
 * axis of zeta4: l1 then l2 ascending, l3 from |l1-l2| to min(l1+l2, lmax). */
sbg_status sbg_lambda_list(int lmax, int* l123);

/* Full (3D) 3PCF and 4PCF of one periodic field (Secs. 2.1 and 2.3;
 * Algorithms 1, 3, 5, 6).
 *   field   : [n0][n1][n2] of `dtype`, host pointer unless SBG_FIELD_ON_DEVICE.
 *   shape   : n0 = n1 = n2 = N, a power of two in 8..512.
 *   edges   : nbins + 1 strictly increasing doubles, edges[0] >= 0,
 *             edges[nbins] < N/2; 1 <= nbins <= 20.
 *   lmax3   : 0..10, used when flags has SBG_3PCF.
 *   lmax4   : 0..5, used when flags has SBG_4PCF.
 *   zeta3   : out, [lmax3+1][nbins][nbins] real
 *             zeta_l^{b1 b2} = (-1)^l/sqrt(2l+1) sum_x delta sum_m a^{b1}_lm a^{b2 *}_lm.
 *   zeta4   : out, [n_lambda(lmax4)][nbins][nbins][nbins] real, Lambda order of
 *             sbg_lambda_list; zeta = Re sum_x delta sum_M C^Lambda_M a a a with
 *             C^Lambda_M = (-1)^(l1+l2+l3) (3j), m3 = -(m1+m2) (Eq. mu, Sec. 2.3).
 *             Every bin triple is written, diagonals included.
 * Either output may be NULL when its flag is not set. */
sbg_status sbg_full(sbg_context* ctx, const void* field, sbg_dtype dtype, const int64_t shape[3],
                    const double* edges, int nbins, int lmax3, int lmax4, sbg_precision prec,
                    unsigned flags, double* zeta3, double* zeta4);

/* Unique bin combinations in the 1D bin index of the paper's coefficient plots
 * (Sec. 4.3, caption of Fig. normalization_projected; the bin loops of
 * Algorithm 6): nested loops with b1 ascending from 0, b2 from b1 + 1 and, for
 * the 4PCF, b3 from b2 + 1, so that no two bins of a combination coincide; the
 * 1D index of a combination is its position in this list.  Host only.
 *   order   : 3 (bin pairs of the 3PCF) or 4 (bin triples of the 4PCF)
 *   n_index : out, nbins (nbins - 1) / 2 or nbins (nbins - 1) (nbins - 2) / 6
 *   bins    : out, [n_index][order - 1] ints, or NULL to query n_index only
 * Errors: SBG_ERR_INVALID_ARG for nbins outside 1..20 or another order. */
sbg_status sbg_unique_bins(int nbins, int order, int* n_index, int* bins);

/* The unique coefficients of a dense output in that 1D order: zeta holds
 * nouter blocks of [nbins]^(order - 1) entries of ncomp doubles (1: real, 2:
 * re, im), e.g. zeta3 of sbg_full (nouter = lmax3 + 1, order 3, ncomp 1) or
 * zeta4 of sbg_projected (nouter = (2 mmax + 1)^2, order 4, ncomp 2); out
 * receives [nouter][n_index][ncomp].  Host only; both pointers are host memory
 * owned by the caller.  Errors: SBG_ERR_INVALID_ARG for a NULL pointer or
 * arguments outside the ranges above. */
sbg_status sbg_unique_gather(const double* zeta, long long nouter, int nbins, int order, int ncomp, double* out);

/* Zero, in place, the coefficients whose bin combination has two coincident
 * bins: b1 = b2 for order 3; b1 = b2, b2 = b3 or b1 = b3 for order 4.  These
 * hold the grid estimator's self-overlap terms, which the paper's application
 * figure ignores by showing those diagonals as zero (Sec. 4, caption of
 * Fig. Full_path).  Every other entry is left as it is.
 *   zeta    : host pointer, nouter blocks of [nbins]^(order - 1) entries of
 *             ncomp doubles (1: real, 2: re, im), the layout of sbg_unique_gather;
 *             owned by the caller, modified in place.
 * Host only.  Errors: SBG_ERR_INVALID_ARG for a NULL pointer, nouter < 0,
 * nbins outside 1..20, order not 3 or 4, or ncomp not 1 or 2 (zeta untouched). */
sbg_status sbg_zero_overlap(double* zeta, long long nouter, int nbins, int order, int ncomp);

/* Number of odd-parity Lambda (l1 + l2 + l3 odd, triangle rule, each l <=
 * lmax) for lmax in 0..10: 1 at lmax 1, 4 at lmax 2, 23 at lmax 4. */
sbg_status sbg_lambda_odd_count(int lmax, int* n_lambda);

/* The odd-parity list as 3 ints per entry, in the loop order of Algorithm 6
 * (as sbg_lambda_list): the first axis of zeta4_odd of sbg_full_odd. */
sbg_status sbg_lambda_odd_list(int lmax, int* l123);

/* Odd-parity full (3D) 4PCF (Eq. mu, Sec. 2.3, with E(Lambda) = -1: the Lambda
 * that Algorithm 6 skips).  For a real field the sum over M of an odd Lambda is
 * imaginary (the terms M and -M are each other's negated conjugates), so each
 * coefficient is returned as its imaginary part:
 *   zeta4_odd : out, [n_odd(lmax4)][nbins][nbins][nbins] real, Lambda order of
 *               sbg_lambda_odd_list; zeta = Im sum_x delta sum_M E(Lambda)
 *               C^Lambda_M a a a, every bin triple.
 * field, dtype, shape, edges, nbins and prec as for sbg_full; lmax4 in 1..5;
 * flags: SBG_SUBTRACT_MEAN, SBG_NORMALIZED, SBG_FIELD_ON_DEVICE (the 4PCF is
 * implied).  A mirror image of the field flips the sign of every coefficient.
 * Errors as for sbg_full. */
sbg_status sbg_full_odd(sbg_context* ctx, const void* field, sbg_dtype dtype, const int64_t shape[3],
                        const double* edges, int nbins, int lmax4, sbg_precision prec, unsigned flags,
                        double* zeta4_odd);

/* Projected (2D) 3PCF and 4PCF of one periodic field (Secs. 2.2 and 2.4;
 * Algorithms 2, 4, 7, 8).
 *   shape   : n0 = n1 = N, a power of two in 8..1024; nbins 1..20; mmax 0..10.
 *   zeta3   : out, [mmax+1][nbins][nbins][2] (re, im),
 *             zeta_m^{b1 b2} = sum_x delta c^{b1}_m c^{b2 *}_m.
 *   zeta4   : out, [2mmax+1][2mmax+1][nbins][nbins][nbins][2], index m + mmax,
 *             zeta_{m1 m2}^{b1 b2 b3} = sum_x delta c^{b1}_{m1} c^{b2}_{m2} c^{b3}_{-(m1+m2)}
 *             with c_{-m} = conj(c_m); entries with |m1 + m2| > mmax are 0. */
sbg_status sbg_projected(sbg_context* ctx, const void* field, sbg_dtype dtype, const int64_t shape[2],
                         const double* edges, int nbins, int mmax, sbg_precision prec, unsigned flags,
                         double* zeta3, double* zeta4);

/* One projected field of a batch: its own shape, edges and output arrays
 * (layouts as in sbg_projected). */
typedef struct {
  const void* field;
  sbg_dtype dtype;
  int64_t shape[2];
  const double* edges;
  double* zeta3;
  double* zeta4;
} sbg_field2d;

/* Many projected fields of uneven sizes (e.g. simulation snapshots) measured in
 * one call with shared nbins, mmax, precision and flags (the paper measures
 * one field per run; each field here is computed as in sbg_projected, Secs.
 * 2.2 and 2.4).  Each entry's field and edges are read as
 * for sbg_projected; its zeta3 / zeta4 receive that field's outputs.  Fields
 * are queued back to back on the context's stream: field i + 1 is queued
 * before field i's results are copied to the caller, so all outputs are valid
 * only when the call returns.  sbg_last_timings then reports the stages summed
 * over the fields.  Errors: as sbg_projected, with the field's index in
 * sbg_last_error; SBG_ERR_TIMEOUT if any field's tensor-core kernel gave up
 * waiting.  Output contents are unspecified after an error. */
sbg_status sbg_projected_batch(sbg_context* ctx, const sbg_field2d* fields, int nfields, int nbins, int mmax,
                               sbg_precision prec, unsigned flags);

/* Projected 3PCF and 4PCF of every 2D slice of a 3D cube (Sec. 4 takes the
 * projected statistics of one slice of a simulation cube), through the batch path
 * of sbg_projected_batch: slice i is cube[i], the contiguous shape[1] x
 * shape[2] block (take slices along another axis by transposing first).
 *   cube   : [n0][n1][n2] of `dtype`, host pointer unless SBG_FIELD_ON_DEVICE;
 *            n1 = n2, a power of two in 8..1024; n0 in 1..65536.
 *   edges, nbins, mmax, prec, flags : as for sbg_projected, shared by every slice.
 *   zeta3  : out (SBG_3PCF), [n0] blocks of sbg_projected's zeta3.
 *   zeta4  : out (SBG_4PCF), [n0] blocks of sbg_projected's zeta4.
 * Errors as for sbg_projected_batch (the message names the slice). */
sbg_status sbg_projected_slices(sbg_context* ctx, const void* cube, sbg_dtype dtype, const int64_t shape[3],
                                const double* edges, int nbins, int mmax, sbg_precision prec, unsigned flags,
                                double* zeta3, double* zeta4);

/* The launch choices the context's autotuner has made so far, one
 * "key=choice" line each.  The first call of a geometry measures, with CUDA
 * events on the context's stream, the candidates of each choice and keeps the
 * fastest for the life of the context:
 *   fft/N/sign/load/axis : lines per CTA of a strided FFT pass (0 the default,
 *                          1 half of it, 2 twice it);
 *   tc4/..., tc4slab/... : x-splits per tile (per field of a slab) of the
 *                          tensor-core 4PCF contraction, among the three that
 *                          fill the SMs' waves best.
 * text: out, up to len bytes including a NUL (may be NULL); *needed (may be
 * NULL) receives the length of the whole report plus one.
 * Errors: SBG_ERR_INVALID_ARG for a NULL ctx. */
sbg_status sbg_autotune_report(const sbg_context* ctx, char* text, size_t len, size_t* needed);

/* Turn the autotuner of ctx on (enable = 1, the default) or off (0: every
 * launch takes its default shape, and the choices made so far are dropped).
 * Errors: SBG_ERR_INVALID_ARG for a NULL ctx or enable not 0 / 1. */
sbg_status sbg_set_autotune(sbg_context* ctx, int enable);

/* Device times (ms, CUDA events) of the stages of the last measurement call:
 * [0] upload+preprocess, [1] forward FFT of delta, [2] kernel spectra (plan),
 * [3] convolutions (inverse FFTs), [4] 3PCF Gram, [5] 4PCF combination,
 * [6] finalisation + download; [7] (not a time) the number of kernels the call
 * launched.  *n_stages is set to the count written (8); ms_per_stage must hold 8. */
sbg_status sbg_last_timings(const sbg_context* ctx, double* ms_per_stage, int* n_stages);

/* Device time (ms, CUDA events on the context's stream) of the 4PCF
 * contraction kernel alone in the last measurement call: the tensor-core
 * kernel for SBG_PREC_BF16X3 / TF32X3, the SIMT launches for SBG_PREC_FP32 (the sum
 * over the pair products of Eq. mu, Sec. 2.3 / Eq. proj_4pcf_coeff, Sec. 2.4,
 * before the coupling step).  It is
 * part of stage [5] of sbg_last_timings; the rest of that stage is the B
 * operand split and the coupling.  *ms is 0 when the call computed no 4PCF.
 * Errors: SBG_ERR_INVALID_ARG for a null pointer. */
sbg_status sbg_last_contraction_ms(const sbg_context* ctx, double* ms);

/* Tile plan of the 4PCF combination, on the host only (no context, no GPU,
 * no device memory).  It builds the tables that sbg_full (dim 3, order lmax =
 * lmax4) or sbg_projected (dim 2, lmax = mmax) uses for nbins bins at
 * precision prec (odd = 1: the odd-parity tables of sbg_full_odd, dim 3
 * only), and so checks that every output term of Algorithm 6 (full,
 * Eq. mu, Sec. 2.3) or Algorithm 8 (projected, Eq. proj_4pcf_coeff, Sec. 2.4)
 * finds its entry among the computed pair x single products.  Outputs (each
 * may be NULL):
 *   ntiles   : tiles of the contraction kernel (tensor-core tiles hold 128
 *              pair rows);
 *   nrows    : pair rows formed;
 *   covering : which pair rows the tiles use: 0 = the structured rows (tensor
 *              core: every pair within one half of the bins; FP32: pairs
 *              b1 <= b2 against columns b3 >= b2), 1 = a greedy cover of the
 *              needed triples; the plan keeps the one with fewer tiles (tensor
 *              core) or fewer pair x column entries (FP32).
 * Errors: SBG_ERR_INVALID_ARG for dim not 2 or 3, nbins outside 1..20, lmax
 * outside 0..5 (3D) or 0..10 (2D), an unknown precision, or odd not 0 / 1 (1
 * only with dim 3); SBG_ERR_INTERNAL
 * if a term finds no entry (a defect of the plan). */
sbg_status sbg_plan4_info(int dim, int nbins, int lmax, sbg_precision prec, int odd, int* ntiles, int* nrows,
                          int* covering);

/* Projected 3PCF that allocates no device memory (the paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * during a measurement, e.g. code running inside a pre-sized memory pool or an
 * allocator that must not be re-entered).  It computes exactly the zeta3 of
 * sbg_projected (SBG_3PCF) with the same kernels, but every intermediate buffer
 * lives in one static device array of the library (about 11 MB, held on every
 * device that loads the library until the process exits).
 *   field  : device pointer, [n][n] of `dtype` (n a power of two, 8..256).
 *   edges  : host pointer, nbins + 1 increasing doubles, edges[nbins] < n/2,
 *            nbins 1..10; mmax 0..10.
 *   flags  : 0 or SBG_SUBTRACT_MEAN.
 *   zeta3  : device pointer, [mmax+1][nbins][nbins][2] (re, im).
 *   stream : cudaStream_t to run on (NULL: legacy default stream).
 * Work is queued on `stream`; zeta3 is valid once the stream has completed.
 * Sizes beyond the maxima return SBG_ERR_UNSUPPORTED_SHAPE (n) or
 * SBG_ERR_INVALID_ARG (nbins, mmax, flags).  The first call made with a device
 * current looks up the array's device address for that device (set-up, once
 * per device); make that first call before any stream capture.  The looked-up
 * address is kept for the life of the process and is not valid across a
 * cudaDeviceReset.  All calls share the one array, which keeps the previous
 * call's contents (each call clears what must start at zero): calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. */
sbg_status sbg_projected3_noalloc(const void* field, sbg_dtype dtype, int64_t n, const double* edges, int nbins,
                                  int mmax, unsigned flags, double* zeta3, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SARABANDE_GB300_H */
