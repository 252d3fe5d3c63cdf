/*
 * cwt.h — C ABI of the GB300 (sm_103a) FFT-based continuous wavelet transform.
 *
 * The library computes the FFTCWT of Wang & He, "Comparisons between fast
 * algorithms for the continuous wavelet transform and applications in
 * cosmology: the 1D case" (RASTI 2023, arXiv:2302.03909), Sec. 3.1:
 *
 *   F(m)   = sum_n f(n) e^{+2 pi i m n / M}                       (Eq. 8, up to L/M)
 *   W(s,n) = sqrt(dx / w~_s) / M * sum_m F(m) psi_hat(2 pi m~ / (M w~_s)) e^{-2 pi i m n / M}
 *                                                                  (Eqs. 9-10)
 *
 * for n < N, one row per scale, where m~ is the signed frequency in
 * (-M/2, M/2] and psi_hat is the analytic Fourier transform of the mother
 * wavelet (Table 2).  M = N for the periodic boundary; for the zero boundary
 * (Sec. 4.1) the signal is zero-extended to M >= 2N and the first N outputs are
 * kept.  The global wavelet power spectrum is Eq. 42:
 *   P(s) = (1/N) sum_{n<N} |W(s,n)|^2.
 *
 * Conventions shared by every entry point:
 *   - Functions return a cwt_status; nothing throws across the ABI.  Arguments
 *     are checked on the host before any launch.
 *   - "device pointer" means memory of the CUDA device that was current when
 *     the plan was created (cudaMalloc, torch tensors, ...).  The caller owns
 *     every pointer it passes; the plan owns its own workspace and tables.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device entry points are asynchronous on that stream.  A plan's
 *     workspace is shared by its calls, so one plan must not run on two
 *     streams at the same time.
 *   - The device for every call must be the one current at plan creation
 *     (CWT_ERR_INVALID_ARG otherwise).
 */
#ifndef CWT_GB300_H
#define CWT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cwt_plan cwt_plan; /* opaque; created and destroyed by the library */
typedef struct cwt_batch cwt_batch; /* opaque; see cwt_batch_create */

typedef enum {
    CWT_OK = 0,
    CWT_ERR_INVALID_ARG = 1,  /* bad size, pointer, alignment, scale or option */
    CWT_ERR_UNSUPPORTED = 2,  /* valid request outside what this build handles */
    CWT_ERR_OOM = 3,          /* device or host allocation failed */
    CWT_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
    CWT_ERR_TIMEOUT = 5,      /* reserved: a bounded device wait gave up */
    CWT_ERR_INTERNAL = 6
} cwt_status;

/* Mother wavelets of Table 2. */
typedef enum {
    CWT_WAVELET_GDW = 0,     /* Gaussian-derived ("Mexican-hat type"):
                                psi(x) = C_N (2 - x^2) e^{-x^2/4},
                                psi_hat(k) = 8 sqrt(pi) C_N k^2 e^{-k^2}, C_N = (18 pi)^{-1/4} */
    CWT_WAVELET_MORLET = 1,  /* psi(x) = C_N (e^{-i w0 x} - e^{-w0^2/2}) e^{-x^2/2},
                                psi_hat(k) = sqrt(2 pi) C_N (e^{-(k-w0)^2/2} - e^{-(k^2+w0^2)/2}),
                                C_N = pi^{-1/4} (1 - 2 e^{-3 w0^2/4} + e^{-w0^2})^{-1/2};
                                Table 2 prints w0 = 4, the default here is w0 = 6 */
    CWT_WAVELET_CBSW = 2,    /* cubic B-spline wavelet: psi_hat(k) = 64 C_N sin^6(k/2) / k^4,
                                C_N = sqrt(30/31) */
    CWT_WAVELET_CWGDW = 3    /* cosine-weighted GDW: psi_hat(k) = sqrt(2 pi) C_N k (k cosh k - sinh k)
                                e^{-k^2/2}, C_N = sqrt(8 / (1 + 5e)) / pi^{1/4} */
} cwt_wavelet;

typedef enum {
    CWT_BOUNDARY_PERIODIC = 0, /* the N-periodic FFTCWT.  N a power of two: M = N.  Otherwise, for
                                  the GDW and the Morlet, the same result through zero-padded
                                  transforms of the periodically extended signal; rows where that does
                                  not apply (the CBSW and CW-GDW, scales whose spectrum is not
                                  negligible (1e-7) at the Nyquist frequency) through Bluestein's chirp
                                  transform on power-of-two FFTs of length >= 2N - 1 (at most 2^25) */
    CWT_BOUNDARY_ZERO = 1      /* zero padding to M = next power of two >= 2N (Eq. 40 context).  With
                                  fft_len 0, the same result with less padding where a scale's wavelet
                                  is short: N a power of two, a periodic N-point transform plus an edge
                                  correction; otherwise (GDW and Morlet) zero-padded transforms of
                                  length M' >= N + E + 1, E the dilated wavelet's support */
} cwt_boundary;

typedef enum {
    CWT_SCALE_DILATION = 0,  /* scales[] are dilations s in samples: w~ = 1 / s */
    CWT_SCALE_W_TILDE = 1    /* scales[] are the paper's dimensionless w~ = w dx (Eq. 4) */
} cwt_scale_unit;

typedef enum { CWT_INPUT_F32 = 0, CWT_INPUT_F64 = 1 } cwt_input_dtype;

/* Arithmetic of the inverse transforms' 1024-point DFT stages (the second pass
 * of the wide-band scales, Eq. 9 for M >= 2^14 up to 2^23).  FP32: CUDA-core
 * FFT stages in FP32.  The other forms run each 1024-point DFT as two
 * 32-point DFT-matrix products on the tensor cores (warp-level MMA) with FP32
 * accumulation, FP32 twiddles between them, and these operands:
 *   FP16   - FP16 operands; each 1024-sample column is scaled by a power of two
 *            into FP16's range (about 3e-4 relative error per stage);
 *   BF16   - BF16 operands (about 2e-3 relative error per stage);
 *   FP16X3 - hi + lo FP16 pairs with three products per block (hi*hi, lo*hi,
 *            hi*lo), about 2^-22 per stage (columns scaled as for FP16);
 *   BF16X3 - hi + lo BF16 pairs, three products per block, about 2^-16.
 * Every other kernel (forward transform, band kernels, first pass, power)
 * stays FP32.  The spectrum product and the FP64-generated tables are the
 * same for every form. */
typedef enum {
    CWT_PRECISION_FP32 = 0,
    CWT_PRECISION_FP16 = 1,
    CWT_PRECISION_BF16 = 2,
    CWT_PRECISION_FP16X3 = 3,
    CWT_PRECISION_BF16X3 = 4
} cwt_precision;

/* Plan options.  Fill with cwt_plan_opts_default() and change fields. */
typedef struct {
    double omega0;       /* Morlet centre wavenumber (default 6) */
    double dx;           /* sampling interval; W scales with sqrt(dx) (Eq. 4). Default 1 */
    int32_t scale_unit;  /* cwt_scale_unit (default CWT_SCALE_DILATION) */
    int32_t input_dtype; /* cwt_input_dtype of the signal (default CWT_INPUT_F32); f64 is
                            converted to f32 on load */
    int64_t fft_len;     /* 0: default M.  Zero boundary: any power of two >= N (e.g. the
                            paper's padding N + 2 Nint(chi / w~_min), rounded up). */
    double eps_trunc;    /* spectral bins where |psi_hat| < eps_trunc * max|psi_hat| are
                            skipped (default 1e-10; 0 keeps every bin) */
    int32_t min_ctas;    /* launch shape: the W-writing launches take up to 8 tiles per CTA while
                            keeping at least this many CTAs (0: 304, two per SM; at most 2^20) */
    int32_t tune;        /* 1: at creation, time plans with min_ctas in {152, 304, 608} and
                            wide_batch_bytes in {32, 128, 256} MiB ({64, 128, 256} with
                            wide2_kernel = 1 or a reduced precision, {16, 32} with
                            wide2_kernel = 2), then band_depth in {4, 8, 16, 2, 1} (a nonzero value given for any of
                            them is kept) on this device and keep the fastest.  Needs temporary device
                            memory of the output's size and runs the transform a few times.  If the
                            environment variable CWT_TUNE_CACHE names a file, a choice stored there for
                            the same device and plan inputs is used without timing, and new choices are
                            appended to it (one line each).  0: no tuning */
    int64_t wide_batch_bytes; /* launch shape: intermediate of one wide-scale launch, one per stream
                            (0: 128 MiB, 32 MiB with the Stockham pass 2; at most 2^36) */
    int32_t precision;   /* cwt_precision of the 1024-point DFT stages (default CWT_PRECISION_FP32) */
    int32_t band_depth;  /* stage fusion: bands of up to band_depth * 1024 bins (1, 2, 4, 8 or 16) are computed in
                            one pass, the band kernel's first DFT stage filled by a Horner sum of band_depth
                            terms; wider bands take the two-pass path.  0: 4 (or tuned) */
    int32_t wide2_kernel; /* pass 2 of the wide scales (1024-point DFTs over Y's columns) in FP32:
                            1: the tile pipeline (tiles of 8 columns copied by TMA, one warp per
                            column with two register radix-32 stages, separate store warps);
                            2: the CTA Stockham kernel (one column per 32 threads, Y read by the
                            DFT threads).  0: chosen per plan, 1 for transform lengths
                            M >= 2^21, 2 below.  The reduced precisions always take the tile
                            pipeline (tensor-core stages) */
    int32_t scratch;     /* cwt_scratch_mode: where the per-call buffers live (default
                            CWT_SCRATCH_PLAN).  CWT_SCRATCH_CALLER plans keep only their constant
                            tables and run with cwt_exec_scratch; they cannot be tuned */
} cwt_plan_opts;

/* Per-call buffers of a plan (the spectrum and its transposed copy, the wide
 * scales' intermediate, power partial sums, the periodic extension, the edge
 * corrections' partial sums, the Bluestein form's work arrays).
 *   CWT_SCRATCH_PLAN   - allocated with the plan, one set per plan;
 *   CWT_SCRATCH_CALLER - supplied by the caller on every call
 *                        (cwt_exec_scratch), so that plans of many shapes can
 *                        share one buffer per stream (a request server keeps
 *                        one per slot).  Sub-plans of one plan run one after
 *                        another and share offsets inside it. */
typedef enum {
    CWT_SCRATCH_PLAN = 0,
    CWT_SCRATCH_CALLER = 1
} cwt_scratch_mode;

void cwt_plan_opts_default(cwt_plan_opts* opts);

/* Plan the transform of N-sample signals at n_scales scales (Sec. 3.1).
 * scales: host array of n_scales finite values > 0 (copied).  Precomputes the
 * band of each scale, FP64-generated twiddle tables (stored FP32) and the
 * workspace on the current device.  *plan is NULL on failure. */
cwt_status cwt_plan_create(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales,
                           int32_t wavelet, int32_t boundary);
cwt_status cwt_plan_create_ex(cwt_plan** plan, int64_t N, const double* scales,
                              int32_t n_scales, int32_t wavelet, int32_t boundary,
                              const cwt_plan_opts* opts);
/* The options a plan was made with, min_ctas and wide_batch_bytes as used
 * (after defaults and tuning). */
cwt_status cwt_plan_get_opts(const cwt_plan* plan, cwt_plan_opts* opts);
/* Frees the plan and its device memory (synchronises the device first).  NULL is OK. */
cwt_status cwt_plan_destroy(cwt_plan* plan);

/* M (the largest transform length for a plan whose N is not a power of two),
 * the plan's device workspace in bytes (for a CWT_SCRATCH_CALLER plan its
 * tables only; see cwt_plan_scratch_bytes), and whether W is complex
 * (1: interleaved complex64, Morlet; 0: float32, the real wavelets).  Any out-pointer may be NULL. */
cwt_status cwt_plan_info(const cwt_plan* plan, int64_t* fft_len, size_t* workspace_bytes,
                         int32_t* out_is_complex);

/* W = CWT of one signal (Eqs. 8-10).
 * signal_dev: N contiguous f32 (or f64 with CWT_INPUT_F64), device, >= 4 (8) B aligned.
 * W_dev: [n_scales][N] row-major, device; f32 for the real wavelets (GDW, CBSW,
 *        CW-GDW), interleaved complex64 (re, im) for the Morlet; 4 B or 8 B aligned.
 * Row s holds scale scales[s]. */
cwt_status cwt_exec(cwt_plan* plan, const void* signal_dev, void* W_dev, void* stream);

/* cwt_exec plus the global wavelet power spectrum (Eq. 42) computed from the
 * FP32 results before they are stored: spectrum_dev[s] = (1/N) sum_n |W(s,n)|^2,
 * float64, device, n_scales entries.  Partial sums are reduced in a fixed order,
 * so repeated calls give bit-identical spectra. */
cwt_status cwt_exec_with_power(cwt_plan* plan, const void* signal_dev, void* W_dev,
                               double* spectrum_dev, void* stream);

/* Bytes of caller-supplied scratch a CWT_SCRATCH_CALLER plan needs per call
 * (0 for a CWT_SCRATCH_PLAN plan). */
cwt_status cwt_plan_scratch_bytes(const cwt_plan* plan, size_t* bytes);

/* cwt_exec_with_power for a CWT_SCRATCH_CALLER plan: the call's per-call
 * buffers are carved from scratch_dev (device, 256 B aligned, at least
 * cwt_plan_scratch_bytes bytes).  The scratch must not be used by anything
 * else until the call's work on `stream` has finished; the plan keeps no
 * pointer into it past the call.  spectrum_dev may be NULL.  Errors:
 * CWT_ERR_INVALID_ARG for a plan with its own scratch, a NULL, misaligned or
 * short scratch, or bad buffers.  CWT_SCRATCH_CALLER plans take no other
 * transform call (cwt_exec, cwt_exec_with_power, cwt_exec_host and
 * cwt_batch_create return CWT_ERR_INVALID_ARG); cwt_wavelet_power,
 * cwt_env_power and cwt_icwt work as for any plan. */
cwt_status cwt_exec_scratch(cwt_plan* plan, const void* signal_dev, void* W_dev, double* spectrum_dev,
                            void* scratch_dev, size_t scratch_bytes, void* stream);

/* Eq. 42 from a W array already in device memory (layout as cwt_exec writes it):
 * one read of W, fixed-order reduction, float64 output (device). */
cwt_status cwt_wavelet_power(cwt_plan* plan, const void* W_dev, double* spectrum_dev,
                             void* stream);

/* Environment-dependent wavelet power spectrum (Sec. 5, Eqs. 41 and 43) with the
 * paper's two environments, delta > 0 (overdense) and delta < 0 (underdense):
 *   p_pos[s] = <|W(s,n)|^2> over the positions n with delta(n) > 0,
 *   p_neg[s] = <|W(s,n)|^2> over the positions n with delta(n) < 0,
 *   frac[0] = N_pos / N, frac[1] = N_neg / N,
 * so that P(s) = frac[0] p_pos[s] + frac[1] p_neg[s] when no delta(n) is 0
 * (Eq. 43).  delta_dev: N samples of the environment field (the dtype of the
 * plan's input; usually the transformed density field itself).  All pointers
 * are device memory; outputs are float64 (p_pos, p_neg: n_scales values; an
 * environment with no position gets 0).  Fixed-order reductions: repeated calls
 * give bit-identical results.  Allocates its partial sums on the first call. */
cwt_status cwt_env_power(cwt_plan* plan, const void* W_dev, const void* delta_dev, double* p_pos_dev,
                         double* p_neg_dev, double* frac_dev, void* stream);

/* Inverse CWT over the plan's scales (Sec. 2, Eq. 6 for the real even
 * wavelets, Eq. 5 for the Morlet):
 *   f(n) - mean(f) ~= (1/K_psi) int_0^inf W(w, n) / sqrt(w) dw
 * (real part doubled for the Morlet), with the integral taken by the
 * trapezoid rule in ln w over the plan's scales (w = w~ / dx) and K_psi the
 * wavelet's admissibility constant (Table 2; for the Morlet computed by
 * quadrature at the plan's omega0).  The mean, which the CWT removes, is not
 * restored.  The reconstruction is as good as the scale grid covers the
 * signal's band.  f_out_dev: N float32, device.  Needs n_scales >= 2. */
cwt_status cwt_icwt(cwt_plan* plan, const void* W_dev, float* f_out_dev, void* stream);

/* Host-buffer form of cwt_exec_with_power: copies the signal from host memory,
 * runs the transform in plan-owned device buffers (allocated on first use) and
 * copies W and, if spectrum_host is not NULL, the spectrum back.  Each group of
 * W rows is copied as soon as the launch that finishes it is done, on a
 * plan-owned second stream, so the copies overlap the rest of the transform.
 * Pinned host memory gives the fastest copies (pageable memory works but does
 * not overlap).  Returns after the results are on the host. */
cwt_status cwt_exec_host(cwt_plan* plan, const void* signal_host, void* W_host,
                         double* spectrum_host, void* stream);

/* The paper's scale grid (Sec. 3.1): w~ = w~_min 2^{i + j/n_subs} with
 * w~_min = c_w pi / N and i < N_levs = Nint(log2 N), written as w~ values in
 * ascending order.  c_w = 2/sqrt(5) (GDW), 0.466094761079290 (CBSW), 0.428218886729052
 * (CW-GDW) or 2 / (w0 + sqrt(w0^2 + 2)) (Morlet).
 * *n_out receives N_levs * n_subs; w_tilde_out may be NULL to query the count. */
cwt_status cwt_scales_paper_grid(int64_t N, int32_t wavelet, double omega0, int32_t n_subs,
                                 double* w_tilde_out, int32_t* n_out);

/* Kernel classes for the timing hook below. */
typedef enum {
    CWT_KCLASS_FORWARD = 0, /* forward transform of the signal (Eq. 8) */
    CWT_KCLASS_BAND = 1,    /* single-pass band kernels: spectrum product (Eq. 10), inverse DFT
                               (Eq. 9), crop, store and power partials */
    CWT_KCLASS_WIDE1 = 2,   /* first pass of wide-band scales (spectrum product + A-point DFTs) */
    CWT_KCLASS_WIDE2 = 3,   /* second pass of wide-band scales (B-point DFTs, crop, store) */
    CWT_KCLASS_POWER = 4,   /* power-spectrum reductions (Eq. 42) */
    CWT_KCLASS_COUNT = 5
} cwt_kernel_class;

/* Timing hook.  enable = 1 makes the following device calls of this plan
 * record a CUDA event pair around every kernel launch, on the stream the
 * launch is made on (launches of independent work still overlap on the side
 * streams); enable = 2 also puts every launch on the call's stream, one after
 * another, so that each event pair times one kernel running alone; 0 turns
 * the hook off.  Any call resets the totals.  Costs one event record per
 * launch boundary.  Other values: CWT_ERR_INVALID_ARG. */
cwt_status cwt_plan_set_timing(cwt_plan* plan, int32_t enable);

/* Totals since cwt_plan_set_timing for one cwt_kernel_class: summed launch
 * durations in ms, the number of launches, and the algorithmic bytes those
 * launches must move (signal read and spectrum write for the forward pass;
 * the W rows written and the spectrum band read for the inverse passes).
 * Waits for the recorded events.  Any out-pointer may be NULL. */
cwt_status cwt_plan_get_timing(cwt_plan* plan, int32_t kernel_class, double* total_ms, int64_t* launches,
                               double* algorithmic_bytes);

/* Power spectrum without any allocation.
 *
 * Same result and layout as cwt_wavelet_power (one row of W per scale; f32
 * rows if is_complex == 0, interleaved complex64 rows otherwise;
 * spectrum_dev[s] = (1/N) sum_n |W(s,n)|^2 in float64), but it needs no plan
 * and calls no cudaMalloc, cudaFree or allocating library routine.  It is for
 * callers that cannot allocate device memory at the point of the call: a
 * process whose device memory is all reserved by another allocator (a
 * framework's caching allocator or a serving worker that has budgeted every
 * byte), or a latency-critical loop that must not pay for the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this
 * is a deployment convenience.
 *
 * Scratch: the partial sums live in one fixed device array inside the library,
 * CWT_NOALLOC_MAX_PARTIALS doubles (512 KiB), held on every device that loads
 * the library until the process exits.  Each row is split into chunks of
 * CWT_NOALLOC_CHUNK samples, so a call needs n_scales * ceil(N /
 * CWT_NOALLOC_CHUNK) partial sums; larger requests are rejected with
 * CWT_ERR_UNSUPPORTED before any launch (e.g. N = 2^22 allows up to 512 scales,
 * N = 2^24 up to 128).  Every call overwrites the partial sums it reads, so no
 * clearing is needed, but all calls share the one array: calls whose kernels
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture on the device.  W_dev and spectrum_dev must be device memory
 * (cudaMalloc, torch tensors) of the current device, checked with
 * cudaPointerGetAttributes; 4 B (f32) / 8 B (complex64, spectrum) aligned;
 * N >= 1, n_scales >= 1, otherwise CWT_ERR_INVALID_ARG.  Asynchronous on
 * `stream`. */
#define CWT_NOALLOC_MAX_PARTIALS 65536
#define CWT_NOALLOC_CHUNK 32768
cwt_status cwt_wavelet_power_noalloc(const void* W_dev, int64_t N, int32_t n_scales, int32_t is_complex,
                                     double* spectrum_dev, void* stream);

/* Batches of many transforms (signals of uneven lengths, each with its own
 * plan) run as a few grouped launches instead of one launch sequence per plan.
 *
 * cwt_batch_create binds plans[i] to its own device buffers signals_dev[i],
 * W_dev[i] and spectra_dev[i] (as cwt_exec_with_power takes them; spectra_dev
 * may be NULL, or hold NULL entries, for no power spectrum).  It records every
 * plan's launch sequence with the dependency level of each launch (its depth
 * in the plan's stream and event order) and merges, over all plans, the
 * launches of one kernel at one level into one grid: a per-CTA table gives
 * each CTA its plan's kernel argument and its block coordinates in the launch
 * it came from.  The CTAs compute exactly what the plan's own launches would,
 * so cwt_batch_exec writes, bit for bit, the results of calling
 * cwt_exec_with_power on each plan.  The result is the FFTCWT of Eqs. 8-10
 * and the power of Eq. 42 for every signal; the grouping is this library's
 * scheduling and has no counterpart in the paper.
 *
 * Every plan may appear once (its workspace is its own); timing must be off;
 * all plans belong to the current device.  n_streams (1..8) is the number of
 * streams a level's grouped launches are spread over.  The batch holds device
 * tables of about 4 bytes per CTA plus the launch arguments; the plans and
 * buffers stay owned by the caller and must outlive the batch, and a plan must
 * not run elsewhere while its batch runs.  Plans made for a batch do best
 * with min_ctas = 1 (fewest, largest CTAs: the batch supplies the parallelism
 * that a single plan's launches otherwise need).
 *
 * cwt_batch_exec runs the levels in order on `stream` (asynchronous; the
 * groups of a level fork to the batch's own streams and join back).
 * cwt_batch_info reports the number of levels, grouped launches and CTAs, and
 * the number of plan launches they replace; any out-pointer may be NULL.
 * Errors: CWT_ERR_INVALID_ARG for bad arguments (a NULL or repeated plan, a
 * bad buffer, n < 1, n_streams outside 1..8, another device), CWT_ERR_OOM or
 * CWT_ERR_CUDA if the tables cannot be made. */
cwt_status cwt_batch_create(cwt_batch** batch, cwt_plan* const* plans, const void* const* signals_dev,
                            void* const* W_dev, double* const* spectra_dev, int32_t n, int32_t n_streams);
cwt_status cwt_batch_exec(cwt_batch* batch, void* stream);
cwt_status cwt_batch_info(const cwt_batch* batch, int32_t* n_levels, int32_t* n_launches, int64_t* n_ctas,
                          int64_t* n_plan_launches);
cwt_status cwt_batch_destroy(cwt_batch* batch);

/* Static description of a status code. */
const char* cwt_status_string(cwt_status status);

/* Text of the last error a plan recorded (never NULL). */
const char* cwt_plan_last_error(const cwt_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* CWT_GB300_H */
