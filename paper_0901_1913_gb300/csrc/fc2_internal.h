// fc2_internal.h -- plan object and kernel launchers shared by the libfc2
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fc2.h"

namespace fc2 {

// Scalars per curve written by the moments kernel (doubles).
enum ScalarSlot {
    SC_W = 0,        // sum w
    SC_XBAR = 1,     // weighted mean (Sec. 3b)
    SC_CHI0 = 2,     // chi2_0 (Sec. 3c)
    SC_S1 = 3,       // sum w (x - xbar), zero up to rounding
    SC_T0 = 4,       // min t (time origin for phase conditioning, Sec. 3b "T_0 <= all t_i")
    SC_TAUMAX = 5,   // max t - T0
    SC_SORTED = 6,   // 1 if t is non-decreasing
    SC_RW = 7,       // max(sqrt(sum w^2) / W, sqrt(sum w^2 d^2) / sqrt(W chi2_0)): scale of
                     // independent per-sample rounding errors relative to the sums
    SC_COUNT = 8
};

// Phasor tables of the exact sums (one device allocation): 512 double-float
// entries (e^{2 pi i a / 256}, then e^{2 pi i b / 65536}), the same 512 in
// double, then (single-curve plans) the 65536 double-float entries
// e^{2 pi i m / 65536} of the last tier's phasors, at DFTAB_T16 (16-byte
// units); a batch keeps the first two (2 * 512 * 16 bytes).
constexpr int DFTAB_T16 = 1024;
constexpr size_t DFTAB_BYTES = (size_t)(DFTAB_T16 + 65536) * 16;

// Float transform kernel families (double passes always use FFT_R16).
enum FftFamily {
    FFT_R16 = 0,   // radix-16 stages in shared memory (k_fft_pass)
    FFT_R64 = 1,   // two register stages of radix R/64 and 64 (k_fft_pass64) for radix
                   // 2^10..2^12, FFT_BULK's kernel for 2^8 and 2^9
    FFT_BULK = 2,  // radix-16 stages fed by bulk asynchronous copies (k_fft_pass_tma), 2^8..2^12
    FFT_R32 = 3,   // two register stages of radix 32 and 32 (k_fft_pass32, 512 threads) for
                   // radix 2^10; FFT_BULK's kernel for 2^8, 2^9, 2^11 and 2^12
    FFT_R32X = 4   // k_fft_pass32 for radix 2^9 (16 x 32) and 2^10; FFT_BULK's kernel for
                   // 2^8, 2^11 and 2^12
};

// Cells per spreading tile: the default for the grid length (1024, or 128 below
// 4096 points), or a requested width of 512, 1024 or 2048 when it is at most
// half the grid (the tile's three key ranges must be disjoint).
inline int spread_tile_of(int64_t M, int requested) {
    if ((requested == 512 || requested == 1024 || requested == 2048) && 2 * (int64_t)requested <= M &&
        M >= 4096)
        return requested;
    return M >= 4096 ? 1024 : 128;
}

// Family for fc2_options.fft_kernel (0 = library default).
inline int fft_family_of(int fft_kernel) {
    return fft_kernel == 2   ? FFT_R16
           : fft_kernel == 3 ? FFT_BULK
           : fft_kernel == 4 ? FFT_R32
           : fft_kernel == 5 ? FFT_R32X
                             : FFT_R64;
}

struct GridGeom {
    int k;            // harmonic multiple of this transform
    int kind;         // 0 = Q (weights), 1 = P (weighted data)
    int64_t L;        // occupied extent in cells (rows beyond are zero)
    int wraps;        // samples wrap the fold period -> keys need sorting
};

struct FftPass {
    int logR;
    int64_t Ns;       // product of the radices of earlier passes
    int64_t rows_nz;  // rows r < rows_nz may be nonzero (first pass), else R
};

struct Workspace;

}  // namespace fc2

struct fc2_plan_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fc2_options opt;

    int64_t n = 0;
    int H = 0;
    double f_min = 0, df = 0;
    int64_t N = 0;
    int oversample = 2;
    int64_t M = 0;
    int logM = 0;
    int G = 0;                 // number of grids: 3H, or H + ceil(H/2) when packed
    int w = 0;                 // spreading kernel width
    double beta = 0;
    // Packed transforms (mixed path, f_min = sh df, grids oversampled >= 4x):
    // every transform has real strengths and no modulation, and each complex
    // grid carries two of them: grid g < H holds Q_k + i P_k (k = g + 1, one
    // set of sample positions), grid H + q holds Q_{H+2q+1} + i Q_{H+2q+2}
    // (two sets).  Their spectra are kept at modes +-(sh + j).  Samples are
    // organised per source (nsrc = 2H: source t is transform Q_{t+1}, with
    // P_{t+1} as its imaginary part when t < H).  npk = number of packed grids
    // (all of them); kernel width and shape w_p, beta_p; deconvolution d_dec_p.
    bool packed = false;
    int nsrc = 0;              // sample sets (sources); 0 = one per grid
    int npk = 0;
    int64_t sh = 0;
    int w_p = 0;
    double beta_p = 0;
    void* d_dec_p = nullptr;
    double tau = 0;            // rank-drop threshold
    int top_k = 8;
    bool fp64 = true;

    // host copies of scalars
    double scal[fc2::SC_COUNT] = {0};

    // device memory
    double* d_t = nullptr;     // caller order (owned unless borrowed)
    double* d_x = nullptr;
    double* d_sigma = nullptr;
    bool borrowed = false;
    double* d_scal = nullptr;  // [SC_COUNT]
    int* d_status = nullptr;
    int32_t* d_perm = nullptr; // sorted position -> caller index
    double* d_tau = nullptr;   // sorted tau = t - T0
    double* d_wq = nullptr;    // sorted w
    double* d_wp = nullptr;    // sorted w (x - xbar)

    // per-transform sample arrays [G][n]
    int32_t* d_key = nullptr;
    void* d_dlt = nullptr;     // T
    void* d_cs = nullptr;      // cpx<T>
    // grids, ping-pong [G][M]
    void* d_grid[2] = {nullptr, nullptr};
    void* d_spec = nullptr;    // cpx<T> [G][N]
    void* d_dec = nullptr;     // cpx<T> [N] deconvolution factors
    void* d_twlo = nullptr;    // cpx<T>
    void* d_twhi = nullptr;
    int tw_shift = 0;
    void* d_twst = nullptr;    // cpx<T> in-CTA stage twiddles per radix
    int64_t twst_off[16] = {0};
    int64_t tw64_off[16] = {0};
    int fft_family = fc2::FFT_R64;  // kernel family of the float passes (fc2::FftFamily)
    int fft_group = 0;         // grids taken through all passes together (0 = all)
    int spread_tile = 0;       // cells per spreading tile (0 = default for M)
    double* d_dchi2 = nullptr; // [H][N]
    float* d_minpiv = nullptr; // unused slot kept for diagnostics
    int32_t* d_flag_list = nullptr;  // bins needing the exact fix-up
    int32_t* d_flag_count = nullptr;
    int64_t flag_cap = 0;
    int64_t* d_L = nullptr;    // [G] occupied extent of each grid
    int64_t* d_slot_soff = nullptr;  // batch: per-transform offset into the sample arrays
    int64_t* d_slot_n = nullptr;     // batch: per-transform sample count
    std::vector<int64_t> h_slot_soff, h_slot_n;  // batch: host copies
    double* d_part = nullptr;  // exact-sum partials [exact_cap][nch][6H]
    uint64_t* d_phA = nullptr; // fixed-point phases frac(f_min tau) 2^64 [n]
    uint64_t* d_phB = nullptr; // fixed-point phases frac(df tau) 2^64 [n]
    float* d_wq32 = nullptr;   // w as float [n], then the low parts w - (float)w [n]
    float* d_wp32 = nullptr;   // w (x - xbar) likewise [2n]
    void* d_dftab = nullptr;   // double-float phasor tables of the tier-2 sums [512]
    int64_t exact_cap = 0;
    void* d_red = nullptr;     // reduction scratch
    size_t red_bytes = 0;
    fc2_best* d_best = nullptr;  // [H + top_k]

    std::vector<fc2::GridGeom> geom;  // per source (sample set)
    std::vector<int64_t> h_L;         // occupied extent of each grid (d_L's host copy)
    std::vector<fc2::FftPass> passes;
    int64_t last_flag_count = 0;
    bool executed = false;     // the device output holds a completed execute
    bool paper = false;        // the paper's nearest-lower-cell gridding (one packed grid)
    int detrend = 0;           // degree of the polynomial removed from x (0 = none)
    double* d_xdet = nullptr;  // detrended x when the caller's x is borrowed
    int64_t s0 = 0;            // f_min / df (paper gridding)
    int64_t last_exact2_count = 0;
    int64_t last_exact3_count = 0;
    int64_t last_routed[3] = {0, 0, 0};  // bins first sent to fix-up tiers 1..3
    int64_t last_resolve_count = 0;
    bool has_perm = false;
    // stage timing (events recorded around each stage while enabled)
    bool timing = false;
    cudaEvent_t ev[8] = {nullptr};
    double stage_ms[8] = {0};
    int64_t stage_n = 0;
    int64_t launches = 0;      // kernels launched by the last execute
    double fft_bytes = 0;      // algorithmic bytes moved by the FFT passes per execute
    // trend fitted with the harmonics (fc2_options.trend_fit): degree D, the
    // scaled time u = (tau - jt_tc) jt_is, the normalised polynomial Gram factor
    // (lower triangle of chol(sum w u^(p+q) / W), row-major 4 x 4), the projected
    // data y_P = L_G^-1 (sum w (x - xbar) u^p) / sqrt(W chi2_poly), chi2_poly,
    // and the exact trend sums' partials [exact_cap][chunks][2 D H]
    bool joint = false;
    int D = 0;
    double jt_tc = 0, jt_is = 1;
    double jt_LG[16] = {0};
    double jt_yP[4] = {0};
    double jt_chi0 = 0;
    double* d_part_t = nullptr;
    // fault injection for the tests (fc2_debug_fault): limit of the bulk-copy
    // transform's mbarrier waits in SM cycles (0 = default, about two seconds),
    // and a tile whose copy that kernel arms but never issues (-1 = none)
    long long dbg_wait_cycles = 0;
    int dbg_drop_tile = -1;
};

namespace fc2 {

// k_prep.cu
cudaError_t launch_moments(const double* t, const double* x, const double* sigma,
                           const int64_t* offs, int64_t C, int64_t n_single,
                           double* scal, int* status, cudaStream_t s);
cudaError_t launch_moments_long(const double* t, const double* x, const double* sigma, int64_t n,
                                double* scal, int* status, void* scratch, cudaStream_t s);
size_t moments_scratch_bytes(int64_t n);
cudaError_t sort_by_time(const double* t, int64_t n, int32_t* perm, void* scratch,
                         size_t scratch_bytes, cudaStream_t s);
size_t sort_scratch_bytes(int64_t n);
cudaError_t launch_gather_sorted(const double* t, const double* x, const double* sigma,
                                 const int32_t* perm, int64_t n, const double* scal,
                                 double* tau, double* wq, double* wp, cudaStream_t s);
cudaError_t launch_phase(fc2_plan_s* p, cudaStream_t s);
cudaError_t sort_wrapping_keys(fc2_plan_s* p, cudaStream_t s);
cudaError_t launch_spread(fc2_plan_s* p, cudaStream_t s);
void force_spread_general(int on);  // every tile to the general spreading kernel (tests)
int device_sm_count();
// The paper's nearest-lower-cell binning into grid 0 (paper gridding).
cudaError_t launch_bin(fc2_plan_s* p, cudaStream_t s);
// Polynomial detrending of x (degree D <= 3) into xo; scal holds T0 and max tau.
size_t trend_scratch_bytes(int64_t n);
cudaError_t launch_detrend(const double* t, const double* x, const double* sigma, int64_t n,
                           int D, const double* scal, int* status, void* scratch, double* xo,
                           cudaStream_t s);

// k_fft.cu
cudaError_t init_twiddles(fc2_plan_s* p, cudaStream_t s);
cudaError_t init_deconv(fc2_plan_s* p, cudaStream_t s);
void plan_fft_passes(fc2_plan_s* p);
cudaError_t autotune_fft(fc2_plan_s* p, cudaStream_t s);  // choose and set up the pass plan
struct FftChoice {
    std::vector<int> rs;  // log2 radix of each pass
    int family;           // fc2::FftFamily
};
std::vector<FftChoice> fft_tune_candidates(int logM, bool fp64);
bool fft_choice_valid(int logM, bool fp64, const FftChoice& c);
cudaError_t set_fft_choice(fc2_plan_s* p, const FftChoice& c, cudaStream_t s);
// k_batch.cu: the batched path's tuning table and fixed configuration
void forget_batch_tuning();
void force_batch_config(int spread_tile, int asm_nt, int bx_ch, int fft_group);
void force_batch_plan(const int* rs, int n, int family);
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t s);  // library device pool
void drop_deconv_cache(int dev);  // k_fft.cu: cached deconvolution tables of a device
cudaError_t launch_fft(fc2_plan_s* p, cudaStream_t s);

// k_solve.cu
cudaError_t launch_assemble(fc2_plan_s* p, cudaStream_t s);
cudaError_t launch_fixup(fc2_plan_s* p, int64_t n1, int64_t n2, int64_t n3, cudaStream_t s);
cudaError_t launch_exact_bins(fc2_plan_s* p, int64_t nb, int tier, cudaStream_t s);
// The double tier's partial sums for H harmonics (k_exact_partial<H, 3>).
cudaError_t launch_exact_partial_tier3(fc2_plan_s* p, int H, const int32_t* b32,
                                       const int64_t* b64, const int32_t* cnt_dev, int64_t cnt,
                                       int64_t base, int64_t cap, cudaStream_t s);
// k_trend.cu: the trend fitted with the harmonics (p->joint)
cudaError_t launch_assemble_joint(fc2_plan_s* p, cudaStream_t s);
cudaError_t launch_fixup_joint(fc2_plan_s* p, int64_t n3, cudaStream_t s);
cudaError_t launch_records_joint(fc2_plan_s* p, const int64_t* rec_j, int nrec, int nch,
                                 cudaStream_t s);
size_t trend_part_bytes(int64_t cap, int H, int D);
// k_prep.cu: block partial sums of w u^k (k <= 2D) and w x u^p (p <= D) of the
// detrending (u on [-1, 1] over the span); nblk * 11 doubles into part
cudaError_t launch_trend_sums(const double* t, const double* x, const double* sigma, int64_t n,
                              int D, const double* scal, double* part, int* nblk, cudaStream_t s);
// Last tier of the mixed path's exact fix-up (4 by default, 3 for diagnostics).
void set_last_fixup_tier(int tier);
int last_fixup_tier();
// k_signif.cu: ln p(f) of the last execute (logp may be nullptr) and per row
// the minimising bin, its ln p and the adjusted-Delta chi^2 factor (device arrays).
cudaError_t launch_significance(fc2_plan_s* p, double* logp, int64_t* jmin, double* lpmin,
                                double* adj, cudaStream_t s);
cudaError_t launch_peaks(fc2_plan_s* p, cudaStream_t s);
size_t peaks_scratch_bytes(int64_t N, int H, int K);
size_t exact_scratch_bytes(int64_t n, int H, int64_t cap);
cudaError_t launch_phase_fx(fc2_plan_s* p, cudaStream_t s);
// Phasor tables of the exact sums (512 double-float pairs, then 512 double2)
// into tab (2 * 512 * 16 bytes).
cudaError_t launch_init_dftab(void* tab, bool with16, cudaStream_t s);  // with16: also DFTAB_T16's table
cudaError_t debug_phasor(const uint64_t* u, int64_t n, int table16, float* out4);  // diagnostics

// k_adjoint.cu: one entry = (curve << 32 | bin) of a curve table
struct AdjTab {
    const int64_t* off;      // [C+1]
    const int* H;            // [C]
    const double* fmin;      // [C]
    const double* df;        // [C]
    const double* scal;      // [C][SC_COUNT]
    const double* tau;       // sorted samples: t - T0
    const double* wq;        // w
    const double* wp;        // w (x - xbar)
    const int32_t* perm;     // sorted position -> caller position (global), or null
    const int64_t* ent;      // [E] (curve << 32 | j)
    const double* gout;      // [E] upstream gradients or null (= 1)
    int K;                   // entries per curve (output layout of d_dx / d_dsigma)
    double tol;              // Newton stopping step
    int max_iter;
};

struct AdjOut {
    double* f_ref;
    double* d_ref;
    double* d_df;
    double* d_dx;     // entry (c, r): K off[c] + r n_c + i, caller order within the curve
    double* d_dsig;
};


cudaError_t launch_backward_tab(const AdjTab& tb, int64_t E, const AdjOut& out, cudaStream_t s);
fc2_status plan_backward(fc2_plan_s* p, int K, const int64_t* peak_j, const double* grad_out,
                         double* f_ref, double* d_ref, double* d_df, double* d_dx,
                         double* d_dsig);

// k_batch.cu
fc2_status batched_execute(int64_t C, const int64_t* offsets, const double* t, const double* x,
                           const double* sigma, const int* H, const double* fmin,
                           const double* df, const int64_t* N, int oversample,
                           const fc2_options& opt, float* dchi2, fc2_best* peaks,
                           int64_t* launches_out, int64_t* stats_out);  // stats_out[18]
void set_batch_timing(bool on);  // stage events in the batched path's chunk graphs

fc2_status batched_backward(int64_t C, const int64_t* offsets, const double* t, const double* x,
                            const double* sigma, const int* H, const double* fmin,
                            const double* df, const int64_t* N, int K, const int64_t* peak_j,
                            const double* grad_out, const fc2_options& opt, double* f_ref,
                            double* d_ref, double* d_df, double* d_dx, double* d_dsig);

// host helpers (fc2_host.cpp)
void gauss_legendre(int nq, double* x, double* w);
double kernel_ft_host(int w, double beta, double xi, int nq, const double* gx, const double* gw);
int default_width(bool fp64, int oversample);

}  // namespace fc2
