/*
 * fc2.h -- C ABI of libfc2, a GB300 (sm_103a) implementation of the Fast
 * chi-squared (Fchi2) periodogram of D. M. Palmer, "A Fast Chi-squared
 * Technique For Period Search of Irregularly Sampled Data" (arXiv 0901.1913).
 *
 * Model (Sec. 1, Eq. "eqtrunc"): for trial frequency f and H' harmonics,
 *     Phi(t) = A_0 + sum_{h=1..H'} A_{2h-1} sin(2 pi h f t) + A_{2h} cos(2 pi h f t).
 * Output (Sec. 2, Eqs. "eqchigen", "eqchix"; Sec. 3c):
 *     Delta chi^2_{H'}(f) = chi2_0 - min_A sum_i (Phi(t_i) - x_i)^2 / sigma_i^2,
 *     chi2_0 = sum_i (x_i - xbar)^2 / sigma_i^2,  xbar = weighted mean (Sec. 3b),
 * for every H' = 1..H at every trial frequency f_j = f_min + j * df,
 * j = 0..N-1 (evaluated in double exactly as written).
 *
 * Path (Sec. 2 "The function p(t) ... P and Q can be efficiently computed by
 * the application of the FFT", Sec. 3b-3e): the weights w_i = sigma_i^-2 and
 * the weighted data w_i (x_i - xbar) are spread onto uniform oversampled
 * grids, one per needed multiple k f (Q at k = 1..2H, P at k = 1..H), FFTs of
 * those grids give the trigonometric sums P(k f_j), Q(k f_j) (Eq. "eqPQ"), and
 * each frequency's (2H+1)-square normal equations (Eqs. "eqalphafirst" ..
 * "eqalpha" and the beta equations) are solved by one bordered Cholesky
 * factorisation that yields all H' at once.
 *
 * Conventions for every call:
 *   - Return value is an fc2_status; no call throws or aborts across the ABI.
 *   - Arrays are plain C arrays of the stated element type and length.  A
 *     pointer is a device pointer when the matching *_on_device option is set,
 *     otherwise a host pointer (pageable or pinned).
 *   - The library copies or borrows inputs as stated per call; output buffers
 *     always belong to the caller.
 *   - A plan is used from one host thread at a time and runs on one CUDA
 *     stream (opt->cuda_stream, or a stream the plan creates).
 *   - Device-side checks never trap: a kernel that finds a problem writes a
 *     status word that the calling function reads and returns.
 */
#ifndef FC2_H
#define FC2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FC2_MAX_H 16

typedef struct fc2_plan_s* fc2_plan;

typedef enum {
    FC2_OK = 0,
    FC2_ERR_INVALID_ARG = 1,   /* argument out of range, NULL, non-finite input, sigma <= 0 */
    FC2_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    FC2_ERR_OOM = 3,           /* device allocation failed or the plan exceeds device memory */
    FC2_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    FC2_ERR_UNSUPPORTED = 5,   /* valid request the library does not implement */
    FC2_ERR_NUMERIC = 6        /* non-finite intermediate (e.g. overflow in the solve) */
} fc2_status;

typedef enum {
    FC2_PREC_FP64 = 0,         /* grids, FFTs and solves in double */
    FC2_PREC_MIXED = 1         /* double phase reduction and moments; float grids and FFTs
                                  with compensated spreading; float Cholesky with a double
                                  re-solve of ill-conditioned bins and an exact double
                                  fix-up of near-singular (aliased) bins */
} fc2_precision;

typedef struct {
    fc2_precision prec;        /* default FC2_PREC_FP64 */
    int kernel_width;          /* spreading-kernel width in grid cells; 0 = default for prec */
    int top_k;                 /* number of peak records fc2_execute returns; 0 = 8 */
    double alias_tau;          /* rank-drop threshold on the Cholesky relative pivot
                                  d_l / alpha_ll; 0 = default (1e-9 FP64) */
    void* cuda_stream;         /* cudaStream_t to run on; NULL = plan-owned stream */
    int device;                /* CUDA device ordinal */
    int inputs_on_device;      /* t, x, sigma are device pointers (borrowed, not copied) */
    int outputs_on_device;     /* dchi2 (and d_dx, d_dsigma) are device pointers */
    int autotune;              /* fc2_plan_create: 1 = time the candidate transform plans
                                  (radix per pass, kernel family) on the plan's own
                                  buffers when it is created and keep the fastest; the
                                  choice is cached per device, size and precision for
                                  the process. 0 or -1 = the fixed balanced plan.
                                  fc2_execute_batched: 0 (default) = the launch
                                  configuration (transform plan and family, spreading
                                  tile, assembly block, exact-sum work item) from the
                                  tuning table, keyed by device, N, grid length,
                                  oversampling, precision, kernel width, largest H of
                                  the chunk and shared sampling; on a miss the chunk's
                                  candidates are timed on the chunk itself (a second or
                                  so for a full chunk) and the fastest is kept for the
                                  process and appended to the cache file
                                  $FC2_TUNE_CACHE (unset: ~/.cache/fc2-gb300/
                                  batch_tune.txt or under $XDG_CACHE_HOME; "" or "off":
                                  no file), which later processes read.  1 = tune
                                  anew; -1 = the fixed default configuration.  A
                                  transform family requested (fft_kernel != 0) also
                                  fixes the configuration.  Every configuration meets
                                  the same error bounds; float rounding depends on the
                                  choice.  Values outside -1..1 are
                                  FC2_ERR_INVALID_ARG */
    int fft_kernel;            /* kernel family of the float transform passes when autotune
                                  is 0: 0 = library default (= 1), 1 = two register stages
                                  of radix R/64 and 64 for radix 2^10..2^12 passes and
                                  family 3's kernel for 2^8 and 2^9, 2 = radix-16 stages in
                                  shared memory, 3 = radix-16 stages fed by bulk
                                  asynchronous copies (radix 2^8..2^12 passes), 4 = two
                                  register stages of radix 32 and 32 with 512 threads
                                  (2^10 passes; family 3's kernel for the others), 5 = the
                                  same for 2^9 (16 x 32) and 2^10 passes.  Passes a family
                                  does not cover use family 2.  FP64 ignores it; values
                                  outside 0..5 are FC2_ERR_INVALID_ARG */
    int gridding;              /* 0 = spreading kernel of width kernel_width with its
                                  Fourier transform divided out, one transform per
                                  harmonic multiple (default; meets 1e-4 chi2_0).
                                  1 = the paper's gridding (Sec. 3b): weights and
                                  weighted data binned into the lower cell
                                  floor((t - T0) / dt) of one zero-padded array
                                  (Kronecker delta, no correction), T0 = min t,
                                  dt = 1 / (M df), one transform of length M (the
                                  smallest power of two above 4 H (f_min/df + N - 1),
                                  oversample ignored), harmonics read at k fhat
                                  (Sec. 3c).  Delta chi^2 then equals the exact value
                                  for times moved to their cell's lower edge: the
                                  paper's gridding error is kept, not bounded.  Needs
                                  f_min a whole number of df steps; no exact fix-up
                                  (flagged bins keep the double re-solve of the
                                  gridded sums); peak records still come from direct
                                  sums at their bins.  Not available in
                                  fc2_execute_batched (FC2_ERR_UNSUPPORTED) */
    int detrend;               /* degree D (0..3) of the polynomial removed from x before
                                  the search: "detrend the data with a polynomial fit"
                                  (Sec. 4).  The weighted (sigma^-2) least-squares
                                  polynomial of degree D in t is subtracted at plan
                                  creation; chi2_0, Delta chi^2 and the records then
                                  describe the residuals (A_0 is their mean, the trend
                                  is not added back).  0 = none (the weighted mean is
                                  always removed, Sec. 3b).  FC2_ERR_INVALID_ARG outside
                                  0..3 or when the samples cannot fix the polynomial;
                                  fc2_backward and fc2_execute_batched return
                                  FC2_ERR_UNSUPPORTED for D > 0 */
    int shared_sampling;       /* fc2_execute_batched only: 1 = every curve was sampled at
                                  the same times with errors proportional to one set
                                  (sigma_c = r_c sigma), as for many sources measured
                                  together in one field (Sec. 4).  Their normalised
                                  weights agree, so the weights' transforms (Q, Eq.
                                  eqPQ) are computed once per chunk of curves and every
                                  curve only adds its H transforms of the weighted
                                  data (P): 3H C transforms become 2H + H C.  All
                                  curves need the same n, H, f_min, df and N and the
                                  same times (checked on the device, FC2_ERR_INVALID_ARG
                                  otherwise).  0 = independent curves */
    int fft_group;             /* when autotune is 0: the number of grids taken through all
                                  transform passes before the next grids start (with one
                                  or two, the data between passes largely stay in L2);
                                  0 = library default (all grids pass by pass); values
                                  below 0 are FC2_ERR_INVALID_ARG */
    int trend_fit;             /* with detrend = D > 0: 0 = subtract the trend first (above);
                                  1 = fit the trend together with the harmonics (Sec. 4's
                                  polynomial detrending as one least-squares model): the null
                                  model is the weighted least-squares polynomial of degree D
                                  in u = (t - t_c) / s (t_c, s the centre and half-width of
                                  the span), and Delta chi^2_{H'} = chi^2(polynomial) -
                                  chi^2(polynomial + H' harmonics), all coefficients fitted
                                  jointly.  Needs the D H extra transforms
                                  sum w u^p e^{2 pi i k f t} (p = 1..D, k = 1..H); the
                                  per-bin system is (2H + 1 + D)-square, its polynomial
                                  block eliminated once.  chi2_0 (fc2_execute) is the
                                  polynomial's chi^2; in records A[0] is the polynomial's
                                  value at t_c plus xbar and A[2H'+1 .. 2H'+D] its higher
                                  coefficients in u.  Single-curve plans only; no paper
                                  gridding; fc2_backward returns FC2_ERR_UNSUPPORTED.
                                  Values other than 0 and 1 are FC2_ERR_INVALID_ARG */
} fc2_options;

/* One selected frequency: bin index, frequency, Delta chi^2 and the
 * coefficients A[0..2H'] of Eq. "eqcoeffs" in the basis order of Eq. "eqtrunc"
 * (absolute time frame, xbar added to A_0 as Sec. 3b directs; entries past
 * 2H' are zero). */
typedef struct {
    int64_t j;
    double f;
    double dchi2;
    int32_t H;                 /* number of harmonics of this record's model */
    int32_t flags;             /* bit 0: bin needed the exact double fix-up */
    double A[2 * FC2_MAX_H + 1];
} fc2_best;

/* Fill *opt with defaults. */
void fc2_options_default(fc2_options* opt);

/*
 * fc2_plan_create -- bind one light curve and one frequency search.
 *   t, x, sigma [n]: sample times, values and standard errors (Sec. 2).
 *     n >= 1; all finite; sigma > 0.  Any order of t.
 *   H: highest harmonic, 1 <= H <= FC2_MAX_H.
 *   f_min >= 0, df > 0, N >= 2: trial frequencies f_j = f_min + j df.
 *   oversample: grid oversampling sigma_g >= 2; the grid length is the
 *     smallest power of two >= oversample * N.
 * Inputs are copied to plan-owned device memory unless inputs_on_device, in
 * which case the device arrays are borrowed and must stay valid and unchanged
 * for the plan's lifetime.  Creation sorts by time if needed, computes the
 * moments of Sec. 3b/3c, and allocates every buffer fc2_execute needs.
 * Errors: FC2_ERR_INVALID_ARG (ranges, NULL, non-finite or sigma <= 0 found
 * on the device), FC2_ERR_OOM, FC2_ERR_CUDA.  *out is NULL on error.
 */
fc2_status fc2_plan_create(const double* t, const double* x, const double* sigma,
                           int64_t n, int H, double f_min, double df, int64_t N,
                           int oversample, const fc2_options* opt, fc2_plan* out);

/*
 * fc2_execute -- run the periodogram.
 *   dchi2 [H][N] (row H'-1 holds Delta chi^2_{H'}), may be NULL.
 *   best [H]: best[H'-1] = argmax_j Delta chi^2_{H'} (ties -> lowest j; Sec. 3e
 *     "The value of f with the largest value of Delta chi^2 ... provides the
 *     best fit"), with the H'-harmonic coefficients.  May be NULL.
 *   peaks [top_k]: local maxima of Delta chi^2_H (value > left neighbour,
 *     >= right neighbour; edges one-sided) in decreasing value, ties by j
 *     (the multiple candidates of Sec. 3e).  Unused records have j = -1.
 *     May be NULL.
 *   chi2_0: scalar, may be NULL.
 * Synchronous: returns after the outputs are written.
 */
fc2_status fc2_execute(fc2_plan p, double* dchi2, fc2_best* best, fc2_best* peaks,
                       double* chi2_0);

/*
 * fc2_execute_batched -- many independent light curves (the "many sources"
 * case of Sec. 4) in one call.
 *   C curves; offsets [C+1] (host): curve c owns samples offsets[c] ..
 *   offsets[c+1]-1 of t, x, sigma (host, or device when inputs_on_device).
 *   H [C], f_min [C], df [C], N [C] (host): per-curve search.
 *   dchi2: packed float output; curve c's [H_c][N_c] block starts at
 *     sum_{c' < c} H_c' N_c'.  Host or device per outputs_on_device.  May be NULL.
 *   peaks [C][top_k] (host): per-curve peak records as fc2_execute.  May be NULL.
 * Validation as fc2_plan_create for each curve.
 */
fc2_status fc2_execute_batched(int64_t C, const int64_t* offsets,
                               const double* t, const double* x, const double* sigma,
                               const int* H, const double* f_min, const double* df,
                               const int64_t* N, int oversample, const fc2_options* opt,
                               float* dchi2, fc2_best* peaks);

/*
 * fc2_backward -- exact (ungridded) gradients and Newton refinement at peaks,
 * the local refinement "using the ungridded data" of Sec. 3e.
 *   K >= 1 peaks at bins peak_j [K] (host, 0 <= j < N).  For each k, with
 *   f = f_min + peak_j[k] df and the H-harmonic model (H <= 8):
 *     d_df[k]          = g_k * dDelta/df,
 *     d_dx[k * n + i]  = g_k * dDelta/dx_i,
 *     d_dsigma[k*n + i] = g_k * dDelta/dsigma_i   (i in the caller's sample order),
 *   with g_k = grad_out[k] (NULL = all ones) and Delta = Delta chi^2_H computed
 *   by direct double sums over the samples (envelope theorem: xbar and the
 *   coefficients are minimisers and need no derivative).
 *   f_refined[k]: maximiser of the exact Delta chi^2_H(f) within one df of the
 *   bin by safeguarded Newton steps (exact second derivative), stopping when
 *   the step is below 1e-10 /d; dchi2_refined[k] its value.
 *   Any output may be NULL; each output pointer may be host or device memory
 *   (detected from the pointer).  Synchronous.
 */
fc2_status fc2_backward(fc2_plan p, int K, const int64_t* peak_j, const double* grad_out,
                        double* f_refined, double* dchi2_refined, double* d_df,
                        double* d_dx, double* d_dsigma);

/*
 * fc2_backward_batched -- fc2_backward for K peaks of each of C curves laid out
 * as in fc2_execute_batched.  peak_j [C][K], grad_out [C][K] (NULL = ones),
 * f_refined / dchi2_refined / d_df [C][K]; d_dx and d_dsigma hold, for curve c
 * and peak r, n_c values starting at K * (offsets[c] - offsets[0]) + r * n_c.
 * t, x, sigma follow opt->inputs_on_device; outputs may be host or device.
 */
fc2_status fc2_backward_batched(int64_t C, const int64_t* offsets,
                                const double* t, const double* x, const double* sigma,
                                const int* H, const double* f_min, const double* df,
                                const int64_t* N, int K, const int64_t* peak_j,
                                const double* grad_out, const fc2_options* opt,
                                double* f_refined, double* dchi2_refined, double* d_df,
                                double* d_dx, double* d_dsigma);

/*
 * fc2_significance -- significance of the trial frequencies of the last
 * fc2_execute of p (Sec. 3d).
 *   The paper ranks frequencies by p(f) = fhat * P_{2H', >= Delta chi^2}, the
 *   chi^2 survival function with 2H' degrees of freedom at Delta chi^2_{H'}(f)
 *   times the trial count so far, fhat = f / df (taken as at least 1).
 *   log_p [H][N]: ln p(f_j) for every H' and j (row-major as dchi2), host or
 *     device memory (detected), or NULL.  ln p = ln fhat - Delta chi^2 / 2 +
 *     ln sum_{i < H'} (Delta chi^2 / 2)^i / i!, with the last two terms in float
 *     (absolute error ~1e-5, far below the error of Delta chi^2 itself).
 *   j_min [H], log_p_min [H] (host): per H' the bin with the smallest ln p
 *     (ties to the lowest j) and that value.  May be NULL.
 *   adj_scale [H] (host): s_{H'} = (n - 2H' - 1) / (chi2_0 - Delta chi^2_best),
 *     so that the adjusted Delta chi^2_adj = s_{H'} Delta chi^2 (Sec. 3d, the
 *     best fit's residual chi^2 per degree of freedom as the denominator;
 *     with a jointly fitted trend of degree D the degrees of freedom are
 *     n - 2H' - 1 - D and chi2_0 is the trend's chi^2); 0 when there are no
 *     degrees of freedom left or the best fit leaves no residual.  May be NULL.
 * Returns FC2_ERR_INVALID_ARG if p is NULL or has not completed an execute.
 * Synchronous; runs on the plan's stream.
 */
fc2_status fc2_significance(fc2_plan p, double* log_p, int64_t* j_min, double* log_p_min,
                            double* adj_scale);

/* Release a plan and its device memory.  NULL is ignored. */
void fc2_plan_destroy(fc2_plan p);

/* Static description of a status code. */
const char* fc2_status_string(fc2_status s);

/*
 * fc2_trim_device_memory -- return to the system the device memory the
 * library keeps for reuse on `device`.
 *
 * Plans and batched calls take device memory from a stream-ordered pool the
 * library owns (one per device); memory they release stays in that pool so the
 * next plan does not have to map it again.  Plans of the same geometry also
 * share deconvolution tables (kept by the library, at most 8 per process).
 * No counterpart in the paper.  Waits for all work on the device, drops the
 * device's cached tables, then trims the pool to zero bytes.
 * Returns FC2_OK (also when the library never allocated on `device`) or
 * FC2_ERR_CUDA.  Must not be called while plans on that device are in use
 * from other threads.
 */
fc2_status fc2_trim_device_memory(int device);

/*
 * fc2_dchi2_exact_noalloc -- exact (ungridded, double) Delta chi^2_{H'} for
 * H' = 1..H at trial bins j (f = f_min + j df), computed straight from the
 * samples, without allocating any device memory.  The paper has no
 * counterpart; this is an interface for callers that cannot allocate when
 * they need the answer: code whose device memory is fully reserved by another
 * allocator (a framework's caching pool, a fixed arena), or a latency-critical
 * loop that must not take the synchronisation an allocation can imply.
 *   t, x, sigma [n], bins [nb] (int64), dchi2 [H][nb]: DEVICE pointers, owned
 *   by the caller.  cuda_stream: cudaStream_t (NULL = legacy default stream).
 *   Limits (the fixed scratch size): 1 <= n <= 4,194,304; 1 <= H <= 8;
 *   1 <= nb <= 128.  Larger requests return FC2_ERR_INVALID_ARG.
 * Scratch: one file-scope device array of about 3.2 MB that every device that
 * loads the library holds until the process exits.  The first call on a device
 * looks up its device address (cudaGetSymbolAddress) with that device current,
 * and so does the first call after a cudaDeviceReset of that device; make
 * those calls before any stream capture.  All calls on a device share
 * the array, so calls whose work overlaps on the GPU race; order them on one
 * stream.  Synchronous: returns after dchi2 is written.  Non-finite inputs or
 * sigma <= 0 give FC2_ERR_INVALID_ARG (detected on the device).
 */
fc2_status fc2_dchi2_exact_noalloc(const double* t, const double* x, const double* sigma,
                                   int64_t n, int H, double f_min, double df,
                                   const int64_t* bins, int64_t nb, double* dchi2,
                                   void* cuda_stream);

/* Host-only helpers (no GPU needed), exposed for testing the host logic. */

/* Grid length the library uses for (N, oversample): smallest power of two >=
 * oversample * N, or 0 if out of range. */
int64_t fc2_grid_size(int64_t N, int oversample);

/* Default spreading-kernel width for a precision and oversampling. */
int fc2_default_width(fc2_precision prec, int oversample);

/* Fourier transform phihat(xi) = integral phi(z) cos(2 pi xi z) dz of the
 * spreading kernel of width w cells used for grids oversampled by
 * `oversample`, at nxi points (host, double).  Returns FC2_OK or
 * FC2_ERR_INVALID_ARG. */
fc2_status fc2_kernel_ft(int w, int oversample, const double* xi, int64_t nxi, double* out);

/* Spreading kernel phi(z) at nz points (host, double). */
fc2_status fc2_kernel_eval(int w, int oversample, const double* z, int64_t nz, double* out);

#ifdef __cplusplus
}
#endif
#endif /* FC2_H */
