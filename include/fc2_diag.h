/*
 * fc2_diag.h -- diagnostic and measurement entry points of libfc2.
 *
 * These calls expose the internal state of the last execute of a plan (or of
 * the last batched execute of the process) for tests and benchmarks: how many
 * bins each precision tier of the exact fix-up handled, the intermediate
 * trigonometric sums, per-stage timings.  They are not needed to compute a
 * periodogram and their layout may change with the implementation.
 *
 * The exact fix-up (Sec. 3e: bins whose gridded normal equations are too
 * ill-conditioned for the interpolated sums are recomputed from sums over the
 * samples, Eq. "eqPQ" evaluated directly) runs in three precision tiers:
 *   tier 1  float sine / cosine of the exact integer phases, compensated
 *           float sums;
 *   tier 2  double-float phasors and sums (about 48 significant bits);
 *   tier 3  double phasors and sums (the last tier of the FP64 path);
 *   tier 4  double-float phasors evaluated directly for every harmonic
 *           multiple from its exact integer phase, double-float products,
 *           sums exact in 64-bit fixed point (the last tier of the mixed
 *           path; on the float and integer pipes).
 * Each tier checks its own result (error estimate from the coefficient norm
 * and the smallest relative pivot of the bordered Cholesky factorisation) and
 * passes the bins it cannot vouch for to the next; the last tier keeps what it
 * finds.
 *
 * Conventions are those of fc2.h: plain C arrays, host pointers unless
 * stated, fc2_status returns, nothing throws across the ABI.  Calls that read
 * device state synchronise the plan's stream.
 */
#ifndef FC2_DIAG_H
#define FC2_DIAG_H

#include <stdint.h>

#include "fc2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bins the last fc2_execute of p sent to the exact fix-up; -1 if p is NULL. */
int64_t fc2_debug_flag_count(fc2_plan p);

/* Counts of the last fc2_execute of p into out7[0..6]: [0] bins re-solved in
 * double from the float spectra (mixed precision), [1] bins recomputed from
 * exact sums, [2] of those, bins that went through tier 2, [3] bins that went
 * through tier 3, [4..6] bins first routed to tiers 1, 2, 3.  No-op on NULL. */
void fc2_debug_counts(fc2_plan p, int64_t* out7);

/* The deconvolved trigonometric sums of the last execute (Eq. "eqPQ"):
 * re/im [3H][N] each, rows Q(f_j), Q(2 f_j) .. Q(2H f_j), then P(f_j) ..
 * P(H f_j), as double (float spectra are widened).  Caller-owned buffers of
 * 3 H N doubles.  Returns FC2_ERR_INVALID_ARG on NULL, FC2_ERR_CUDA if a copy
 * fails. */
fc2_status fc2_debug_spectra(fc2_plan p, double* re, double* im);

/* The time origin T0 the plan measures phases from (Sec. 3b); 0 on NULL. */
double fc2_debug_t0(fc2_plan p);

/* Fault injection for the tests of the bounded waits.  Every wait of the
 * bulk-copy transform passes (fc2_options.fft_kernel 1 or 3, passes after the
 * first of radix 2^8..2^12) on an mbarrier gives up after wait_cycles SM clock
 * cycles (0 = the default, about two seconds); a CTA that gives up sets
 * FC2_ERR_TIMEOUT, waits (again bounded) for its copies in flight and returns,
 * and fc2_execute returns FC2_ERR_TIMEOUT.  drop_tile >= 0 names the tile of
 * those passes whose barrier is armed but whose copy is never issued, so that
 * its wait runs out; -1 issues every copy.  Both settings stay with the plan.
 * FC2_ERR_INVALID_ARG on NULL, wait_cycles < 0 or drop_tile < -1. */
fc2_status fc2_debug_fault(fc2_plan p, long long wait_cycles, int drop_tile);

/* Fault injection for the tests of allocation failures: the k-th allocation
 * from the library's device pool after this call (k >= 1) fails as if the
 * device were out of memory, once; the caller sees FC2_ERR_OOM.  k <= 0
 * disarms.  Process-wide. */
void fc2_debug_fail_alloc(int64_t k);

/* Allocations the library has requested from its device pools so far in this
 * process (including those fc2_debug_fail_alloc made fail). */
int64_t fc2_debug_alloc_count(void);

/* Bytes of the library's device pool on `device` in use by live allocations,
 * after waiting for all work on the device (0 if the library never allocated
 * there, -1 on a CUDA error). */
int64_t fc2_debug_pool_used(int device);

/* Bins of the last execute that tier `tier` (2 or 3) handled, into out[0..cap).
 * Returns how many were copied, or -1 on a bad argument or a failed copy. */
int64_t fc2_debug_tier_bins(fc2_plan p, int tier, int64_t* out, int64_t cap);

/* Last tier of the mixed path's exact fix-up, for the process: 4 (default)
 * or 3 (double sums, as in the FP64 path).  Other values select 4. */
void fc2_debug_last_tier(int tier);

/* Delta chi^2 [H][nb] at bins[0..nb) from the exact sums of one tier
 * (1, 2, 3 or 4), written to out (H * nb doubles).  Overwrites those bins of the
 * plan's device output.  FC2_ERR_INVALID_ARG for a bin outside [0, N), a bad
 * tier, or nb above N or above the plan's exact-round size. */
fc2_status fc2_debug_exact_bins(fc2_plan p, const int64_t* bins, int64_t nb, int tier,
                                double* out);

/* Transform pass plans (host only, no GPU needed).  A plan is a list of
 * radices 2^r1, 2^r2, .. (first pass first) whose exponents add up to logM.
 *
 * fc2_debug_fft_plan: the fixed planner's plan for 2^logM points in float
 * (fp64 = 0) or double: radices into radices[0..P), returns P (-1 if it needs
 * more than max_passes or logM is out of 1..40).
 *
 * fc2_debug_fft_candidates: the plans the autotuner times, as entries
 * [P, r1, .., rP] one after another in radices[]; returns the entries'
 * length (-1 if max_entries is too small).
 *
 * fc2_debug_fft_plan_check: with validate != 0, 1 when the plan breaks a
 * precondition of the pass kernels for the given float kernel family
 * (fc2_options.fft_kernel; every radix has a kernel, every pass's tiles fit
 * the grid, and each next pass's tile width is at most the current radix);
 * otherwise (or with validate = 0) the host replay of the kernels' index
 * arithmetic for that plan -- the global loads of each pass's input, the
 * stores toward the next pass on each kernel's store path, the shared tile
 * slots those stores read, the inter-pass twiddle exponents -- over the
 * first, last and spread tiles of every pass: 0 when all are in range, else
 * 100 * (pass + 1) + the failing check, with info4 (may be NULL) = pass,
 * check, tile, index.  -1 on bad arguments. */
int fc2_debug_fft_plan(int logM, int fp64, int* radices, int max_passes);
int fc2_debug_fft_candidates(int logM, int fp64, int* radices, int max_entries);
int fc2_debug_fft_plan_check(int logM, int fp64, int fft_kernel, const int* radices, int P,
                             int validate, int64_t* info4);

/* Kernels launched by the last fc2_execute_batched call of this process. */
int64_t fc2_debug_batch_launches(void);

/* Counts of the last fc2_execute_batched call into out5[0..4]: entries
 * re-solved in double, entries recomputed by tier 1, tier 2 and tier 3, and
 * the number of chunk graphs launched.  No-op on NULL. */
void fc2_debug_batch_counts(int64_t* out5);

/* Host wall milliseconds of the last fc2_execute_batched call of this process
 * in seven phases (out7[0..6]): setup before the chunk loop; per chunk,
 * summed: buffer allocation and input uploads, per-curve moments and the wait for them, chunk
 * layout and table uploads, graph capture / update and launch, the wait for
 * the chunk's kernels and results; release at the end.  No-op on NULL. */
void fc2_debug_batch_phase_ms(double* out7);

/* Stage timing of the batched path on (enable != 0) or off, for the process.
 * While on, every chunk of fc2_execute_batched records CUDA events on its
 * stream (inside the chunk's graph) between (0) gather, phase reduction and
 * spreading, (1) FFT passes, (2) assembly, solve and double re-solve, (3) exact
 * fix-up, (4) peaks and their records. */
void fc2_debug_batch_timing(int enable);

/* Device milliseconds of the five stages of the last fc2_execute_batched call
 * with timing on, summed over its chunks (out6[0..4]), and the transforms'
 * algorithmic bytes (out6[5]: the kept spectra written, 3 H_c N_c complex
 * values per curve).  Zeros when timing was off.  No-op on NULL. */
void fc2_debug_batch_stage_ms(double* out6);

/* e^{2 pi i u_k 2^-64} for n 64-bit phases (host array, n in 1..2^24) as the
 * exact fix-up's double-float phasor evaluates it (table factors for the top
 * 16 bits, a small rotation for the rest): out4[4k..4k+3] = (re high, re low,
 * im high, im low), host floats.  For tests of its accuracy.
 * FC2_ERR_INVALID_ARG for bad arguments, FC2_ERR_CUDA on a CUDA failure. */
fc2_status fc2_debug_phasor(const uint64_t* u, int64_t n, float* out4);

/* The same for the phasor of the fix-up's last tier (sums exact in fixed
 * point): one double-float table entry e^{2 pi i m / 65536} for the top 16
 * bits, then the same small rotation.  Same arguments and errors. */
fc2_status fc2_debug_phasor16(const uint64_t* u, int64_t n, float* out4);

/* Launch configuration of the last fc2_execute_batched call's last chunk
 * (out12): [0] source (0 fixed, 1 tuning table or cache file, 2 tuned in the
 * call), [1] transform family (0 radix-16 in shared memory, 1 two register
 * stages, 2 bulk copies), [2] spreading tile (cells), [3] assembly block
 * (threads), [4] samples per exact-sum work item, [5] transform passes,
 * [6..9] their log2 radices, [10] configurations timed, [11] tuning
 * milliseconds (host wall time; the bits of a double), [12] grids taken
 * through both transform passes at a time (0 = all grids pass by pass). */
void fc2_debug_batch_config(int64_t* out13);

/* Fixed configuration of batched calls that do not tune (autotune = -1, or a
 * transform family requested): spreading tile 512 / 1024 / 2048 cells,
 * assembly block 128 / 256 threads (float), exact-sum work item 1024 / 2048 /
 * 4096 samples, transform groups of 8 / 16 / 32 grids; 0, or a value the
 * grid does not allow, keeps the default (1024 cells, or 128 below
 * 4096-point grids; 128 threads; 2048 samples; all grids pass by pass).
 * Process-wide; for tests and diagnostics. */
void fc2_debug_batch_force(int spread_tile, int asm_nt, int bx_ch, int fft_group);

/* Fixed transform plan of batched calls that do not tune (as
 * fc2_debug_batch_force): log2 radices rs[0..n), n <= 4, first pass first,
 * and the float kernel family (0 radix-16 stages in shared memory, 1 two
 * register stages, 2 bulk copies).  It is used only for grids whose length it
 * fits and where it is one of the autotuner's candidates; n = 0 clears it.
 * Process-wide; for tests. */
void fc2_debug_batch_force_plan(const int* rs, int n, int family);

/* Empty this process's tuning table of the batched path; the cache file is
 * read again at the next lookup. */
void fc2_debug_batch_forget_tuning(void);

/* on != 0: every spreading tile goes to the general kernel (running sums of
 * all of a tile's cells kept across sample batches and sample sets), also the
 * tiles of one sample set that fit one staging batch, which by default the
 * single-batch kernel computes cell by cell.  Both sum each cell's samples in
 * the same order with the same arithmetic.  0 restores the default.
 * Process-wide; for tests. */
void fc2_debug_spread_force_general(int on);

/* Stage timing of p on (enable != 0) or off; resets the accumulated times.
 * While on, each execute records CUDA events on the plan's stream around
 * (0) phase reduction and spreading, (1) FFT passes, (2) assembly and solve,
 * (3) exact fix-up, (4) peaks and coefficients.  FC2_ERR_CUDA if an event
 * cannot be created. */
fc2_status fc2_stage_timing(fc2_plan p, int enable);

/* Mean milliseconds per execute of each of the five stages since timing was
 * enabled (ms5[0..4], may be NULL), the kernels launched by the last execute
 * (may be NULL), and the algorithmic bytes of one execute's FFT passes (may
 * be NULL). */
fc2_status fc2_stage_times(fc2_plan p, double* ms5, int64_t* launches, double* fft_bytes);

#ifdef __cplusplus
}
#endif

#endif /* FC2_DIAG_H */
