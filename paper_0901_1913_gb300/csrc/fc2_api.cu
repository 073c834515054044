// fc2_api.cu -- the C ABI of libfc2: validation, plan lifetime, buffer
// management and the order of kernel launches.  No kernel arithmetic here.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <map>
#include <mutex>
#include <vector>

#include "fc2_common.cuh"
#include "../../include/fc2_diag.h"
#include "fc2_internal.h"

using namespace fc2;

static int64_t g_last_batch_launches = 0;
// re-solved, exact float / double-float / double, graphs; then the host
// milliseconds of the call's seven phases (as doubles' bits)
static int64_t g_last_batch_stats[32] = {0};

// Device memory comes from one stream-ordered pool per device owned by the
// library.  Memory that a destroyed plan returns stays mapped in the pool
// (unlimited release threshold), so plans created one after another reuse it
// instead of mapping gigabytes afresh; fc2_trim_device_memory hands it back.
namespace fc2 {
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t device_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = pool;
    return pool;
}

// Fault injection for the tests (fc2_debug_fail_alloc): the k-th pool
// allocation from now on fails as if the device were out of memory.
static std::atomic<int64_t> g_fail_alloc_in{0};
static std::atomic<int64_t> g_alloc_count{0};  // pool allocations so far (diagnostics)

cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t s) {
    g_alloc_count.fetch_add(1);
    int64_t k = g_fail_alloc_in.load();
    while (k > 0 && !g_fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaMallocAsync(ptr, bytes, s);
    return cudaMallocFromPoolAsync(ptr, bytes, pool, s);
}

static cudaMemPool_t existing_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    return it == g_pools.end() ? nullptr : it->second;
}
}  // namespace fc2

namespace {

struct Guard {  // returns FC2_ERR_CUDA on the first failing runtime call
    cudaError_t e = cudaSuccess;
    bool ok(cudaError_t r) {
        if (r != cudaSuccess && e == cudaSuccess) e = r;
        return e == cudaSuccess;
    }
};


fc2_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return FC2_OK;
    if (e == cudaErrorMemoryAllocation) return FC2_ERR_OOM;
    return FC2_ERR_CUDA;
}

template <typename P>
cudaError_t dalloc(P** ptr, size_t bytes, cudaStream_t s) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    return pool_alloc((void**)ptr, bytes, s);
}

template <typename P>
void dfree(P*& ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync((void*)ptr, s);
    ptr = nullptr;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

void free_plan_memory(fc2_plan_s* p) {
    cudaStream_t s = p->stream;
    if (!p->borrowed) { dfree(p->d_t, s); dfree(p->d_x, s); dfree(p->d_sigma, s); }
    dfree(p->d_xdet, s);
    dfree(p->d_scal, s); dfree(p->d_status, s); dfree(p->d_perm, s); dfree(p->d_part_t, s);
    dfree(p->d_tau, s); dfree(p->d_wq, s); dfree(p->d_wp, s);
    dfree(p->d_key, s); dfree(p->d_dlt, s); dfree(p->d_cs, s);
    dfree(p->d_grid[0], s); dfree(p->d_grid[1], s); dfree(p->d_spec, s);
    dfree(p->d_dec, s); dfree(p->d_dec_p, s); dfree(p->d_twlo, s); dfree(p->d_twhi, s); dfree(p->d_twst, s);
    dfree(p->d_dchi2, s); dfree(p->d_flag_list, s); dfree(p->d_flag_count, s);
    dfree(p->d_L, s); dfree(p->d_red, s); dfree(p->d_best, s); dfree(p->d_part, s);
    dfree(p->d_phA, s); dfree(p->d_phB, s); dfree(p->d_wq32, s); dfree(p->d_wp32, s);
    dfree(p->d_dftab, s);
}

}  // namespace

extern "C" {

fc2_status fc2_plan_create(const double* t, const double* x, const double* sigma, int64_t n,
                           int H, double f_min, double df, int64_t N, int oversample,
                           const fc2_options* opt_in, fc2_plan* out) {
    if (!out) return FC2_ERR_INVALID_ARG;
    *out = nullptr;
    fc2_options opt;
    if (opt_in) opt = *opt_in; else fc2_options_default(&opt);
    if (!t || !x || !sigma || n < 1 || n > (1ll << 31) - 1) return FC2_ERR_INVALID_ARG;
    if (H < 1 || H > FC2_MAX_H) return FC2_ERR_INVALID_ARG;
    if (!(isfinite(f_min) && f_min >= 0.0) || !finite_pos(df) || N < 2) return FC2_ERR_INVALID_ARG;
    if (!isfinite(f_min + (double)(N - 1) * df)) return FC2_ERR_INVALID_ARG;
    if (oversample < 2 || oversample > 64) return FC2_ERR_INVALID_ARG;
    if (opt.prec != FC2_PREC_FP64 && opt.prec != FC2_PREC_MIXED) return FC2_ERR_INVALID_ARG;
    if (opt.kernel_width != 0 && (opt.kernel_width < 2 || opt.kernel_width > 16))
        return FC2_ERR_INVALID_ARG;
    if (opt.top_k < 0 || opt.top_k > 64 || opt.alias_tau < 0.0) return FC2_ERR_INVALID_ARG;
    if (opt.fft_kernel < 0 || opt.fft_kernel > 5) return FC2_ERR_INVALID_ARG;
    if (opt.fft_group < 0) return FC2_ERR_INVALID_ARG;
    if (opt.autotune < -1 || opt.autotune > 1) return FC2_ERR_INVALID_ARG;
    if (opt.gridding < 0 || opt.gridding > 1) return FC2_ERR_INVALID_ARG;
    if (opt.detrend < 0 || opt.detrend > 3) return FC2_ERR_INVALID_ARG;
    if (opt.trend_fit < 0 || opt.trend_fit > 1) return FC2_ERR_INVALID_ARG;
    if (opt.trend_fit == 1 && opt.detrend == 0) return FC2_ERR_INVALID_ARG;  // no trend to fit
    if (opt.trend_fit == 1 && opt.gridding != 0) return FC2_ERR_UNSUPPORTED;
    if (H > 8) return FC2_ERR_UNSUPPORTED;
    int64_t M = fc2_grid_size(N, oversample);
    if (M == 0) return FC2_ERR_INVALID_ARG;
    // The paper's gridding (Sec. 3b-3c): trial frequencies are bins fhat = s0 + j
    // of one transform of length M whose multiples k fhat, k <= 2H, stay below M/2.
    int64_t s0 = 0;
    if (opt.gridding == 1) {
        const double r = f_min / df;
        const double rs = floor(r + 0.5);
        if (!(rs >= 0.0 && rs < 1e12 && fabs(r - rs) <= 1e-9 * std::max(1.0, r)))
            return FC2_ERR_INVALID_ARG;
        s0 = (int64_t)rs;
        const double top = 4.0 * H * (double)(s0 + N - 1) + 1.0;
        if (top > (double)(1ll << 30)) return FC2_ERR_UNSUPPORTED;
        M = 1024;
        while ((double)M < top) M <<= 1;
    }

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return FC2_ERR_CUDA;
    if (opt.device < 0 || opt.device >= ndev) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(opt.device) != cudaSuccess) return FC2_ERR_CUDA;

    fc2_plan_s* p = new (std::nothrow) fc2_plan_s();
    if (!p) return FC2_ERR_OOM;
    p->opt = opt;
    p->device = opt.device;
    if (opt.cuda_stream) {
        p->stream = (cudaStream_t)opt.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete p;
            return FC2_ERR_CUDA;
        }
        p->own_stream = true;
    }
    cudaStream_t s = p->stream;
    p->n = n; p->H = H; p->f_min = f_min; p->df = df; p->N = N; p->oversample = oversample;
    p->M = M;
    p->logM = 0;
    while ((1ll << p->logM) < M) ++p->logM;
    p->G = 3 * H;
    p->fp64 = (opt.prec == FC2_PREC_FP64);
    p->paper = (opt.gridding == 1);
    p->s0 = s0;
    p->detrend = opt.detrend;
    p->joint = (opt.trend_fit == 1);
    p->D = p->joint ? opt.detrend : 0;
    if (p->joint) p->G = 3 * H + p->D * H;  // the trend transforms w u^p e^{..}, p = 1..D
    if (p->paper) p->G = 1;
    p->w = opt.kernel_width ? opt.kernel_width : default_width(p->fp64, oversample);
    const double sig_eff = (double)M / (double)N;
    p->beta = 0.97 * M_PI * (1.0 - 0.5 / sig_eff) * (double)p->w;
    // Packed transforms: when f_min is a whole number sh of df steps, Q_k and
    // P_k share positions frac(k df tau) and need no modulation, so their
    // strengths w and w (x - xbar) are real and one complex grid carries both
    // (Q_k = (F(m) + conj F(-m)) / 2, P_k = (F(m) - conj F(-m)) / 2i at modes
    // m = sh + j).  The modes then reach |m| = sh + N - 1, so this needs a grid
    // with at least 2x oversampling of that range.
    {
        const double r = f_min / df;
        const double shd = floor(r + 0.5);
        const int64_t mmax = (int64_t)shd + N - 1;
        if (!p->paper && !p->fp64 && !p->joint && !opt.kernel_width && shd >= 0.0 && shd < 1e15 &&
            fabs(r - shd) <= 1e-9 * std::max(1.0, r) && 4 * std::max<int64_t>(mmax, 1) <= M) {
            p->packed = true;
            p->sh = (int64_t)shd;
            p->G = H + (H + 1) / 2;
            p->npk = p->G;
            p->nsrc = 2 * H;
            const double sig_p = (double)M / (2.0 * (double)std::max<int64_t>(mmax, 1));
            p->w_p = default_width(false, 2);
            p->beta_p = 0.97 * M_PI * (1.0 - 0.5 / std::min(sig_p, 2.0)) * (double)p->w_p;
        }
    }
    p->tau = opt.alias_tau > 0.0 ? opt.alias_tau : (p->fp64 ? 1e-9 : 1e-6);
    p->top_k = opt.top_k ? opt.top_k : 8;
    plan_fft_passes(p);
    p->fft_family = fft_family_of(opt.fft_kernel);
    p->fft_group = opt.fft_group;

    const size_t tsz = p->fp64 ? 8 : 4;
    const size_t csz = 2 * tsz;
    const int G = p->G;
    const int NSRC = p->nsrc ? p->nsrc : G;  // sample sets
    const size_t spec_rows = p->packed ? (size_t)2 * G : (size_t)G;
    const size_t spec_bytes = p->paper ? (size_t)M * csz : spec_rows * N * csz;
    // memory estimate
    size_t need = 0;
    need += (size_t)n * 8 * 6 + (size_t)n * 4;
    need += (size_t)NSRC * n * (4 + tsz + csz);
    need += 2 * (size_t)G * M * csz;
    need += spec_bytes + (size_t)N * tsz + (size_t)H * N * 8 + (size_t)N * 4;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) == cudaSuccess && need > freeb) {
        if (p->own_stream) cudaStreamDestroy(p->stream);
        delete p;
        return FC2_ERR_OOM;
    }

    Guard g;
    if (opt.inputs_on_device) {
        p->d_t = (double*)t; p->d_x = (double*)x; p->d_sigma = (double*)sigma;
        p->borrowed = true;
    } else {
        g.ok(dalloc(&p->d_t, n * 8, s)) && g.ok(dalloc(&p->d_x, n * 8, s)) &&
            g.ok(dalloc(&p->d_sigma, n * 8, s));
        if (g.e == cudaSuccess) {
            g.ok(cudaMemcpyAsync(p->d_t, t, n * 8, cudaMemcpyHostToDevice, s));
            g.ok(cudaMemcpyAsync(p->d_x, x, n * 8, cudaMemcpyHostToDevice, s));
            g.ok(cudaMemcpyAsync(p->d_sigma, sigma, n * 8, cudaMemcpyHostToDevice, s));
        }
    }
    const size_t grid_bytes = (size_t)G * M * csz;
    const size_t sort_b = sort_scratch_bytes(n);
    const size_t keysort_b = (size_t)n * (8 * 2 + 4 * 3 + tsz + csz) + 4096 +
                             (size_t)((n + 2047) / 2048) * 256 * 4;
    const size_t red_b = std::max({peaks_scratch_bytes(N, H, p->top_k), sort_b,
                                   moments_scratch_bytes(n), (size_t)8192});
    p->red_bytes = red_b;
    g.ok(dalloc(&p->d_scal, SC_COUNT * 8, s)) && g.ok(dalloc(&p->d_status, 16, s)) &&
        g.ok(dalloc(&p->d_perm, n * 4, s)) && g.ok(dalloc(&p->d_tau, n * 8, s)) &&
        g.ok(dalloc(&p->d_wq, n * 8, s)) && g.ok(dalloc(&p->d_wp, n * 8, s)) &&
        g.ok(dalloc(&p->d_key, (size_t)NSRC * n * 4, s)) &&
        g.ok(dalloc(&p->d_dlt, (size_t)NSRC * n * tsz, s)) &&
        g.ok(dalloc(&p->d_cs, (size_t)NSRC * n * csz, s)) &&
        g.ok(dalloc(&p->d_grid[0], grid_bytes, s)) &&
        g.ok(dalloc(&p->d_grid[1], std::max(grid_bytes, keysort_b), s)) &&
        g.ok(dalloc(&p->d_spec, spec_bytes, s)) &&
        g.ok(dalloc(&p->d_dec, (size_t)N * tsz, s)) &&
        g.ok(dalloc(&p->d_dec_p, (size_t)N * tsz, s)) &&
        g.ok(dalloc(&p->d_twlo, (size_t)(1ll << ((p->logM + 1) / 2)) * csz, s)) &&
        g.ok(dalloc(&p->d_twhi, (size_t)(M >> ((p->logM + 1) / 2)) * csz, s)) &&
        g.ok(dalloc(&p->d_twst, (size_t)(8 * 4096 + 256) * csz, s)) &&
        g.ok(dalloc(&p->d_dchi2, (size_t)H * N * 8, s)) &&
        g.ok(dalloc(&p->d_flag_list, (size_t)N * 4 * 4, s)) &&
        g.ok(dalloc(&p->d_flag_count, 16, s)) && g.ok(dalloc(&p->d_L, (size_t)G * 8, s)) &&
        g.ok(dalloc(&p->d_red, red_b, s)) &&
        g.ok(dalloc(&p->d_best, (size_t)(H + p->top_k) * sizeof(fc2_best), s));
    p->flag_cap = N;
    p->exact_cap = std::max<int64_t>(2048, H + p->top_k);
    if (p->joint) g.ok(dalloc(&p->d_part_t, trend_part_bytes(p->exact_cap, H, p->D), s));
    g.ok(dalloc(&p->d_part, exact_scratch_bytes(n, H, p->exact_cap), s)) &&
        g.ok(dalloc(&p->d_phA, (size_t)n * 8, s)) && g.ok(dalloc(&p->d_phB, (size_t)n * 8, s)) &&
        g.ok(dalloc(&p->d_wq32, (size_t)n * 8, s)) && g.ok(dalloc(&p->d_wp32, (size_t)n * 8, s)) &&
        g.ok(dalloc(&p->d_dftab, DFTAB_BYTES, s));
    if (g.e != cudaSuccess) {
        fc2_status st = map_err(g.e);
        free_plan_memory(p);
        cudaStreamSynchronize(s);
        if (p->own_stream) cudaStreamDestroy(p->stream);
        delete p;
        return st;
    }
    g.ok(cudaMemsetAsync(p->d_status, 0, 16, s));
    g.ok(launch_moments_long(p->d_t, p->d_x, p->d_sigma, n, p->d_scal, p->d_status, p->d_red, s));
    int status = 0;
    g.ok(cudaMemcpyAsync(p->scal, p->d_scal, sizeof(p->scal), cudaMemcpyDeviceToHost, s));
    g.ok(cudaMemcpyAsync(&status, p->d_status, 4, cudaMemcpyDeviceToHost, s));
    g.ok(cudaStreamSynchronize(s));
    fc2_status st = FC2_OK;
    if (g.e != cudaSuccess) st = map_err(g.e);
    else if (status != 0) st = (fc2_status)status;
    double trend_sum[11] = {0};  // joint trend fit: sum w u^k (k <= 2D), sum w x u^p (p <= D)
    if (st == FC2_OK && p->joint) {
        void* scratch = nullptr;
        int nblk = 0;
        g.ok(pool_alloc(&scratch, trend_scratch_bytes(n), s));
        if (g.e == cudaSuccess) {
            g.ok(launch_trend_sums(p->d_t, p->d_x, p->d_sigma, n, p->D, p->d_scal,
                                   (double*)scratch, &nblk, s));
            std::vector<double> part((size_t)nblk * 11);
            g.ok(cudaMemcpyAsync(part.data(), scratch, part.size() * 8, cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(scratch, s);
            g.ok(cudaStreamSynchronize(s));
            for (int b = 0; b < nblk; ++b)  // in block order
                for (int v = 0; v < 11; ++v) trend_sum[v] += part[(size_t)b * 11 + v];
        }
        if (g.e != cudaSuccess) st = map_err(g.e);
    }
    if (st == FC2_OK && p->detrend > 0 && !p->joint) {
        // Polynomial detrending (Sec. 4), then the moments of the residuals.
        // A borrowed x is left untouched: the residuals go to a plan buffer.
        double* xo = p->d_x;
        if (p->borrowed) {
            g.ok(dalloc(&p->d_xdet, (size_t)n * 8, s));
            xo = p->d_xdet;
        }
        void* scratch = nullptr;
        g.ok(pool_alloc(&scratch, trend_scratch_bytes(n), s));
        if (g.e == cudaSuccess) {
            g.ok(launch_detrend(p->d_t, p->d_x, p->d_sigma, n, p->detrend, p->d_scal, p->d_status,
                                scratch, xo, s));
            p->d_x = xo;
            g.ok(launch_moments_long(p->d_t, p->d_x, p->d_sigma, n, p->d_scal, p->d_status,
                                     p->d_red, s));
            g.ok(cudaMemcpyAsync(p->scal, p->d_scal, sizeof(p->scal), cudaMemcpyDeviceToHost, s));
            g.ok(cudaMemcpyAsync(&status, p->d_status, 4, cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(scratch, s);
            g.ok(cudaStreamSynchronize(s));
        }
        if (g.e != cudaSuccess) st = map_err(g.e);
        else if (status != 0) st = (fc2_status)status;
    }
    if (st == FC2_OK) {
        // Time origin: the earliest sample, moved back by (w/2 + 1) cells of
        // the k = 1 grid so no sample's spreading window reaches below cell 0
        // (the paper's gridding: T0 = min t, its "T0 <= all t_i").
        const double back =
            p->paper ? 0.0 : (0.5 * std::max(p->w, p->w_p) + 1.0) / ((double)M * df);
        if (p->joint) {
            // The trend's normal equations: G = sum w u^(p+q) / W (normalised, p, q <= D),
            // beta_P = sum w (x - xbar) u^p.  G = L_G L_G^T once; the polynomial's
            // own chi^2 is chi2_0 - |L_G^-1 beta_P|^2 / W, and y_P, normalised by
            // sqrt(W chi2_poly), is what every bin's elimination needs.
            const int D = p->D;
            const double W = trend_sum[0], xbar = p->scal[SC_XBAR];
            double Gm[4][4], L[4][4] = {{0}}, y[4];
            for (int a = 0; a <= D; ++a)
                for (int b = 0; b <= D; ++b) Gm[a][b] = trend_sum[a + b] / W;
            for (int r = 0; r <= D && st == FC2_OK; ++r) {
                for (int c = 0; c <= r; ++c) {
                    double v = Gm[r][c];
                    for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
                    if (r == c) {
                        if (!(v > 1e-14 * Gm[r][r])) { st = FC2_ERR_INVALID_ARG; break; }
                        L[r][r] = sqrt(v);
                    } else {
                        L[r][c] = v / L[c][c];
                    }
                }
            }
            if (st == FC2_OK) {
                double yy = 0.0;
                for (int r = 0; r <= D; ++r) {
                    double v = (trend_sum[2 * D + 1 + r] - xbar * trend_sum[r]) / sqrt(W);
                    for (int k = 0; k < r; ++k) v -= L[r][k] * y[k];
                    y[r] = v / L[r][r];
                    yy += y[r] * y[r];
                }
                const double chi_poly = p->scal[SC_CHI0] - yy;
                if (!(chi_poly > 0.0)) st = FC2_ERR_NUMERIC;  // the trend explains everything
                p->jt_chi0 = chi_poly;
                p->scal[SC_CHI0] = chi_poly;  // the null model's chi^2
                for (int r = 0; r < 4; ++r) {
                    for (int c = 0; c < 4; ++c) p->jt_LG[r * 4 + c] = (r <= D && c <= r) ? L[r][c] : 0.0;
                    p->jt_yP[r] = (r <= D && chi_poly > 0.0) ? y[r] / sqrt(chi_poly) : 0.0;
                }
                // u = (t - t_c) / s over the span: relative to tau = t - T0 (after
                // the shift below), u = (tau - jt_tc) jt_is
                const double tc_abs = p->scal[SC_T0] + 0.5 * p->scal[SC_TAUMAX];
                p->jt_is = p->scal[SC_TAUMAX] > 0.0 ? 2.0 / p->scal[SC_TAUMAX] : 1.0;
                p->jt_tc = tc_abs - (p->scal[SC_T0] - back);
            }
        }
        p->scal[SC_T0] -= back;
        p->scal[SC_TAUMAX] += back;
        g.ok(cudaMemcpyAsync(p->d_scal, p->scal, sizeof(p->scal), cudaMemcpyHostToDevice, s));
        const int32_t* perm = nullptr;
        if (p->scal[SC_SORTED] == 0.0) {
            g.ok(sort_by_time(p->d_t, n, p->d_perm, p->d_grid[1], std::max(grid_bytes, keysort_b), s));
            perm = p->d_perm;
        }
        p->has_perm = (perm != nullptr);
        g.ok(launch_gather_sorted(p->d_t, p->d_x, p->d_sigma, perm, n, p->d_scal, p->d_tau,
                                  p->d_wq, p->d_wp, s));
        g.ok(launch_phase_fx(p, s));
        // geometry of each transform
        // The occupied extent is rounded to whole first-pass rows, so that the
        // spread writes every cell the first pass reads.  With the autotuner the
        // first pass may have a radix as small as 2^8 (its candidates).
        const int LOGR1 = opt.autotune > 0 ? std::min(p->passes[0].logR, 8) : p->passes[0].logR;
        const int64_t S1 = M >> LOGR1;
        const int64_t tile = spread_tile_of(M, p->spread_tile);
        const int64_t unit = std::max(S1, tile);
        p->geom.resize(NSRC);
        std::vector<int64_t> Ls(NSRC), Lh(G);
        for (int gi = 0; gi < NSRC; ++gi) {  // per sample set
            GridGeom& gg = p->geom[gi];
            if (gi < 2 * H) { gg.k = gi + 1; gg.kind = 0; }
            else if (gi < 3 * H) { gg.k = gi - 2 * H + 1; gg.kind = 1; }
            else { gg.k = (gi - 3 * H) % H + 1; gg.kind = 3; }  // the trend transforms
            if (p->packed) gg.kind = 2;
            const int wg = p->packed ? p->w_p : p->w;
            const double c = (double)gg.k * df;
            const double pmax = c * p->scal[SC_TAUMAX];
            const double cells = pmax * (double)M;
            if (!(pmax < 1.0) || cells + wg + 2.0 >= (double)M) {
                gg.wraps = (pmax >= 1.0) ? 1 : 0;
                gg.L = M;
            } else {
                gg.wraps = 0;
                int64_t L = (int64_t)floor(cells) + wg + 3;
                L = ((L + unit - 1) / unit) * unit;
                gg.L = std::min(L, M);
            }
            Ls[gi] = gg.L;
        }
        for (int gi = 0; gi < G; ++gi) {  // a grid's occupied extent: that of its sets
            if (!p->packed || gi < H) {
                Lh[gi] = Ls[gi];
            } else {
                const int t0 = H + 2 * (gi - H);
                Lh[gi] = std::max(Ls[t0], t0 + 1 < NSRC ? Ls[t0 + 1] : 0);
            }
        }
        if (p->paper) {  // one array: cells floor(frac(df tau) M), all of them if it wraps
            const double cells = df * p->scal[SC_TAUMAX] * (double)M;
            int64_t L = M;
            if (df * p->scal[SC_TAUMAX] < 1.0 && cells + 2.0 < (double)M) {
                L = ((int64_t)floor(cells) + 2 + unit - 1) / unit * unit;
                L = std::min(L, M);
            }
            Lh[0] = L;
            p->geom[0].L = L;
            p->geom[0].wraps = (L == M) ? 1 : 0;
        }
        p->h_L = Lh;
        g.ok(cudaMemcpyAsync(p->d_L, Lh.data(), G * 8, cudaMemcpyHostToDevice, s));
        // Algorithmic bytes of the transform: each pass reads its input once
        // (the first pass only the rows that hold samples) and writes its output
        // once (the last pass only the N kept modes).
        {
            double fb = 0.0;
            const int P = (int)p->passes.size();
            for (int pi = 0; pi < P; ++pi) {
                const int64_t R = 1ll << p->passes[pi].logR, Sp = M / R;
                for (int gi = 0; gi < G; ++gi) {
                    int64_t rd = M;
                    if (pi == 0) rd = std::min(R, (Lh[gi] + Sp - 1) / Sp) * Sp;
                    const int64_t wr =
                        (pi == P - 1 && !p->paper) ? (gi < p->npk ? 2 * N : N) : M;
                    fb += (double)(rd + wr) * (double)csz;
                }
            }
            p->fft_bytes = fb;
        }
        if (opt.autotune > 0) g.ok(autotune_fft(p, s));  // sets the pass plan and its tables
        else g.ok(init_twiddles(p, s));
        if (p->paper) g.ok(cudaStreamSynchronize(s));  // no deconvolution
        else g.ok(init_deconv(p, s));                   // synchronises
        if (g.e != cudaSuccess) st = map_err(g.e);
    }
    if (st != FC2_OK) {
        cudaStreamSynchronize(s);
        free_plan_memory(p);
        cudaStreamSynchronize(s);
        if (p->own_stream) cudaStreamDestroy(p->stream);
        delete p;
        return st;
    }
    *out = p;
    return FC2_OK;
}

// Kernel launches per stage (for the launch count the benchmark reports).
static int64_t launches_front(const fc2_plan_s* p) {
    if (p->paper) return 1 + (int64_t)p->passes.size() + 1 + (p->fp64 ? 0 : 1);  // bin, fft, assemble(+resolve)
    int64_t n = 1 + 1 + (int64_t)p->passes.size() + 1 + (p->fp64 ? 0 : 1);  // phase, spread, fft, assemble(+resolve)
    int bits = 0;
    while ((1ll << bits) < p->M + 2 * std::max(p->w, p->w_p) + 2) ++bits;
    for (auto& g : p->geom)
        if (g.wraps) n += 2 + 3 * ((bits + 7) / 8);
    return n;
}

static void rec(fc2_plan_s* p, int i) {
    if (p->timing) cudaEventRecord(p->ev[i], p->stream);
}

static fc2_status run_pipeline(fc2_plan_s* p) {
    cudaStream_t s = p->stream;
    Guard g;
    rec(p, 0);
    if (p->paper) g.ok(launch_bin(p, s));
    else g.ok(launch_phase(p, s)) && g.ok(launch_spread(p, s));
    rec(p, 1);
    g.ok(launch_fft(p, s));
    rec(p, 2);
    g.ok(launch_assemble(p, s));
    rec(p, 3);
    int32_t fc[4] = {0, 0, 0, 0};  // tier-1 list, re-solve list, tier-2 list, tier-3 list
    g.ok(cudaMemcpyAsync(fc, p->d_flag_count, 16, cudaMemcpyDeviceToHost, s));
    g.ok(cudaStreamSynchronize(s));
    if (g.e != cudaSuccess) return map_err(g.e);
    if (p->paper) fc[0] = fc[2] = fc[3] = 0;  // no exact fix-up under the paper's gridding
    p->last_resolve_count = fc[1];
    p->last_flag_count = (int64_t)fc[0] + fc[2] + fc[3];
    p->last_routed[0] = fc[0]; p->last_routed[1] = fc[2]; p->last_routed[2] = fc[3];
    for (int i = 0; i < 4; ++i)
        if (fc[i] > p->flag_cap) return FC2_ERR_NUMERIC;
    const int64_t nfix = p->last_flag_count;
    if (nfix > 0) g.ok(launch_fixup(p, fc[0], fc[2], fc[3], s));
    rec(p, 4);
    g.ok(launch_peaks(p, s));
    rec(p, 5);
    const int64_t cap = p->exact_cap;
    const int64_t r1 = (nfix + cap - 1) / cap;
    p->launches = launches_front(p) + 6 * r1 + 6;  // fix-up rounds: 3 tiers x 2; peaks: 4 + records 2
    return map_err(g.e);
}

fc2_status fc2_execute(fc2_plan p, double* dchi2, fc2_best* best, fc2_best* peaks,
                       double* chi2_0) {
    if (!p) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return FC2_ERR_CUDA;
    cudaStream_t s = p->stream;
    // A device output buffer is written in place; otherwise results are copied.
    double* own = p->d_dchi2;
    bool direct = false;
    if (dchi2) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, dchi2) == cudaSuccess && at.type == cudaMemoryTypeDevice &&
            at.device == p->device) {
            p->d_dchi2 = dchi2;
            direct = true;
        }
        cudaGetLastError();
    }
    fc2_status st = run_pipeline(p);
    p->d_dchi2 = own;
    if (st != FC2_OK) {
        // a kernel's own report (e.g. a bounded wait that gave up, after which
        // later stages saw garbage) explains a failure better than its
        // consequences; the word starts at zero again for the next execute
        int status = 0;
        cudaStreamSynchronize(s);
        cudaGetLastError();
        if (cudaMemcpy(&status, p->d_status, 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
            status != 0) {
            cudaMemset(p->d_status, 0, 4);
            return (fc2_status)status;
        }
        cudaGetLastError();
        return st;
    }
    Guard g;
    const size_t bytes = (size_t)p->H * p->N * 8;
    if (dchi2 && !direct)
        g.ok(cudaMemcpyAsync(dchi2, p->d_dchi2, bytes, cudaMemcpyDefault, s));
    std::vector<fc2_best> recs((size_t)(p->H + p->top_k));
    int status = 0;
    if (best || peaks)
        g.ok(cudaMemcpyAsync(recs.data(), p->d_best, recs.size() * sizeof(fc2_best),
                             cudaMemcpyDeviceToHost, s));
    g.ok(cudaMemcpyAsync(&status, p->d_status, 4, cudaMemcpyDeviceToHost, s));
    int32_t tiers[2] = {0, 0};
    g.ok(cudaMemcpyAsync(tiers, p->d_flag_count + 2, 8, cudaMemcpyDeviceToHost, s));
    g.ok(cudaStreamSynchronize(s));
    if (g.e != cudaSuccess) return map_err(g.e);
    p->last_exact2_count = p->last_flag_count > 0 ? tiers[0] : 0;
    p->last_exact3_count = p->last_flag_count > 0 ? tiers[1] : 0;
    if (status != 0) {
        // a kernel reported a problem (e.g. a bounded wait that gave up): the
        // word starts at zero again for the next execute of this plan
        g.ok(cudaMemsetAsync(p->d_status, 0, 4, s));
        g.ok(cudaStreamSynchronize(s));
        return (fc2_status)status;
    }
    p->executed = true;
    if (best) memcpy(best, recs.data(), sizeof(fc2_best) * p->H);
    if (peaks) memcpy(peaks, recs.data() + p->H, sizeof(fc2_best) * p->top_k);
    if (chi2_0) *chi2_0 = p->scal[SC_CHI0];
    if (p->timing) {
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]);
            p->stage_ms[i] += ms;
        }
        p->stage_n += 1;
    }
    return FC2_OK;
}

fc2_status fc2_backward_batched(int64_t C, const int64_t* offsets, const double* t,
                                const double* x, const double* sigma, const int* H,
                                const double* f_min, const double* df, const int64_t* N, int K,
                                const int64_t* peak_j, const double* grad_out,
                                const fc2_options* opt_in, double* f_refined,
                                double* dchi2_refined, double* d_df, double* d_dx,
                                double* d_dsigma) {
    fc2_options opt;
    if (opt_in) opt = *opt_in; else fc2_options_default(&opt);
    return batched_backward(C, offsets, t, x, sigma, H, f_min, df, N, K, peak_j, grad_out, opt,
                            f_refined, dchi2_refined, d_df, d_dx, d_dsigma);
}

void fc2_plan_destroy(fc2_plan p) {
    if (!p) return;
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    for (int i = 0; i < 8; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    free_plan_memory(p);
    cudaStreamSynchronize(p->stream);
    if (p->own_stream) cudaStreamDestroy(p->stream);
    delete p;
}

fc2_status fc2_execute_batched(int64_t C, const int64_t* offsets, const double* t,
                               const double* x, const double* sigma, const int* H,
                               const double* f_min, const double* df, const int64_t* N,
                               int oversample, const fc2_options* opt_in, float* dchi2,
                               fc2_best* peaks) {
    fc2_options opt;
    if (opt_in) opt = *opt_in; else fc2_options_default(&opt);
    int64_t nl = 0;
    fc2_status st = batched_execute(C, offsets, t, x, sigma, H, f_min, df, N, oversample, opt,
                                    dchi2, peaks, &nl, g_last_batch_stats);
    g_last_batch_launches = nl;
    return st;
}

fc2_status fc2_backward(fc2_plan p, int K, const int64_t* peak_j, const double* grad_out,
                        double* f_refined, double* dchi2_refined, double* d_df, double* d_dx,
                        double* d_dsigma) {
    if (p && p->detrend > 0) return FC2_ERR_UNSUPPORTED;  // gradients through the detrend fit
    return plan_backward(p, K, peak_j, grad_out, f_refined, dchi2_refined, d_df, d_dx, d_dsigma);
}

/* Diagnostics (declared in fc2_diag.h): number of bins the last execute
 * sent to the exact fix-up, and the spectra of the last execute. */
int64_t fc2_debug_flag_count(fc2_plan p) { return p ? p->last_flag_count : -1; }

/* Counts of the last execute: [0] bins re-solved in double (mixed path),
 * [1] bins recomputed from exact sums, [2] of those, bins that went through
 * double-float sums (tier 2), [3] bins that went through all-double sums
 * (tier 3), [4..6] bins first routed to tiers 1, 2, 3. */
void fc2_debug_counts(fc2_plan p, int64_t* out7) {
    if (!p || !out7) return;
    out7[0] = p->last_resolve_count;
    out7[1] = p->last_flag_count;
    out7[2] = p->last_exact2_count;
    out7[3] = p->last_exact3_count;
    for (int i = 0; i < 3; ++i) out7[4 + i] = p->last_routed[i];
}

fc2_status fc2_debug_spectra(fc2_plan p, double* re, double* im) {
    if (!p || !re || !im) return FC2_ERR_INVALID_ARG;
    const size_t N = (size_t)p->N;
    if (p->paper) {  // one spectrum Z = Qhat + i Phat, mode m at [M/2 + m]
        const size_t M = (size_t)p->M;
        std::vector<char> zb(M * (p->fp64 ? 16 : 8));
        if (cudaMemcpy(zb.data(), p->d_spec, zb.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return FC2_ERR_CUDA;
        auto z = [&](int64_t m, double* r, double* i) {
            const size_t k = (size_t)((int64_t)(M / 2) + m);
            if (p->fp64) { *r = ((const double*)zb.data())[2 * k]; *i = ((const double*)zb.data())[2 * k + 1]; }
            else { *r = ((const float*)zb.data())[2 * k]; *i = ((const float*)zb.data())[2 * k + 1]; }
        };
        const int H = p->H;
        for (int r = 0; r < 3 * H; ++r) {
            const bool isq = r < 2 * H;
            const int k = isq ? r + 1 : r - 2 * H + 1;
            for (size_t j = 0; j < N; ++j) {
                const int64_t m = (int64_t)k * (p->s0 + (int64_t)j);
                double ar, ai, br, bi;
                z(m, &ar, &ai);
                z(-m, &br, &bi);
                const size_t o = (size_t)r * N + j;
                if (isq) { re[o] = 0.5 * (ar + br); im[o] = 0.5 * (ai - bi); }
                else { re[o] = 0.5 * (ai + bi); im[o] = 0.5 * (br - ar); }
            }
        }
        return FC2_OK;
    }
    const size_t rows = p->packed ? (size_t)2 * p->G : (size_t)3 * p->H;  // rows as stored
    const size_t cnt = rows * N;
    std::vector<char> buf(cnt * (p->fp64 ? 16 : 8));
    std::vector<char> dec(N * (p->fp64 ? 8 : 4)), decp(N * 4);
    if (cudaMemcpy(buf.data(), p->d_spec, buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FC2_ERR_CUDA;
    if (cudaMemcpy(dec.data(), p->d_dec, dec.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FC2_ERR_CUDA;
    if (p->packed &&
        cudaMemcpy(decp.data(), p->d_dec_p, decp.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FC2_ERR_CUDA;
    auto val = [&](size_t row, size_t j, double* r, double* i) {
        if (p->fp64) {
            const double* b = (const double*)buf.data();
            *r = b[2 * (row * N + j)]; *i = b[2 * (row * N + j) + 1];
        } else {
            const float* b = (const float*)buf.data();
            *r = b[2 * (row * N + j)]; *i = b[2 * (row * N + j) + 1];
        }
    };
    auto dd = [&](size_t j) {
        return p->fp64 ? ((const double*)dec.data())[j] : (double)((const float*)dec.data())[j];
    };
    // output rows: Q_1..Q_2H, then P_1..P_H
    const int H = p->H;
    for (int r = 0; r < 3 * H; ++r) {
        const bool isq = r < 2 * H;
        const int k = isq ? r + 1 : r - 2 * H + 1;
        for (size_t j = 0; j < N; ++j) {
            const size_t o = (size_t)r * N + j;
            double ar, ai, br, bi;
            if (p->packed) {
                // grid and part (0 = real, 1 = imaginary) of this transform
                int g, part;
                if (k <= H) { g = k - 1; part = isq ? 0 : 1; }
                else { g = H + (k - H - 1) / 2; part = (k - H - 1) & 1; }
                const double d = 0.5 * ((const float*)decp.data())[j];
                val(2 * (size_t)g, j, &ar, &ai);
                val(2 * (size_t)g + 1, j, &br, &bi);
                if (part == 0) { re[o] = (ar + br) * d; im[o] = (ai - bi) * d; }
                else { re[o] = (ai + bi) * d; im[o] = (br - ar) * d; }
            } else {
                val((size_t)r, j, &ar, &ai);
                re[o] = ar * dd(j); im[o] = ai * dd(j);
            }
        }
    }
    return FC2_OK;
}

double fc2_debug_t0(fc2_plan p) { return p ? p->scal[SC_T0] : 0.0; }

void fc2_debug_last_tier(int tier) { set_last_fixup_tier(tier); }

void fc2_debug_fail_alloc(int64_t k) { g_fail_alloc_in.store(k > 0 ? k : 0); }

int64_t fc2_debug_alloc_count(void) { return g_alloc_count.load(); }

int64_t fc2_debug_pool_used(int device) {
    cudaMemPool_t pool = existing_pool(device);
    if (!pool) return 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    uint64_t used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int64_t)used;
}

fc2_status fc2_debug_fault(fc2_plan p, long long wait_cycles, int drop_tile) {
    if (!p || wait_cycles < 0 || drop_tile < -1) return FC2_ERR_INVALID_ARG;
    p->dbg_wait_cycles = wait_cycles;
    p->dbg_drop_tile = drop_tile;
    return FC2_OK;
}

/* Bins of the last execute that tier `tier` (2 or 3) of the exact fix-up
 * handled; returns how many were copied (at most cap), or -1. */
int64_t fc2_debug_tier_bins(fc2_plan p, int tier, int64_t* out, int64_t cap) {
    if (!p || !out || cap < 0 || (tier != 2 && tier != 3)) return -1;
    const int64_t cnt = tier == 2 ? p->last_exact2_count : p->last_exact3_count;
    const int64_t nb = std::min(cap, std::min(cnt, (int64_t)p->flag_cap));
    std::vector<int32_t> b((size_t)std::max<int64_t>(nb, 1));
    if (nb > 0 && cudaMemcpy(b.data(), p->d_flag_list + (size_t)tier * p->flag_cap,
                             (size_t)nb * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    for (int64_t i = 0; i < nb; ++i) out[i] = b[(size_t)i];
    return nb;
}

/* Delta chi^2 [H][nb] at the given bins from the exact sums of one tier
 * (1 float, 2 double-float, 3 double), for tests of each tier.  Overwrites
 * those bins of the plan's internal output.  nb <= min(N, exact-round size). */
fc2_status fc2_debug_exact_bins(fc2_plan p, const int64_t* bins, int64_t nb, int tier,
                                double* out) {
    if (!p || !bins || !out || nb < 1 || nb > p->N || nb > p->exact_cap || tier < 1 || tier > 4)
        return FC2_ERR_INVALID_ARG;
    for (int64_t i = 0; i < nb; ++i)
        if (bins[i] < 0 || bins[i] >= p->N) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return FC2_ERR_CUDA;
    cudaStream_t s = p->stream;
    std::vector<int32_t> b32(bins, bins + nb);
    if (cudaMemcpyAsync(p->d_flag_list, b32.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return FC2_ERR_CUDA;
    if (launch_exact_bins(p, nb, tier, s) != cudaSuccess) return FC2_ERR_CUDA;
    for (int h = 0; h < p->H; ++h)
        for (int64_t i = 0; i < nb; ++i)
            if (cudaMemcpy(out + (size_t)h * nb + i, p->d_dchi2 + (size_t)h * p->N + bins[i], 8,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
                return FC2_ERR_CUDA;
    return FC2_OK;
}

/* e^{2 pi i u_k 2^-64} for n 64-bit phases as the exact fix-up's double-float
 * phasor computes it: out4[4k..4k+3] = (re hi, re lo, im hi, im lo).  For
 * tests of its accuracy.  n in 1..2^24. */
fc2_status fc2_debug_phasor(const uint64_t* u, int64_t n, float* out4) {
    if (!u || !out4 || n < 1 || n > (1 << 24)) return FC2_ERR_INVALID_ARG;
    return fc2::debug_phasor(u, n, 0, out4) == cudaSuccess ? FC2_OK : FC2_ERR_CUDA;
}

/* The last tier's phasor (one 65536-entry table, then the small rotation),
 * as fc2_debug_phasor. */
fc2_status fc2_debug_phasor16(const uint64_t* u, int64_t n, float* out4) {
    if (!u || !out4 || n < 1 || n > (1 << 24)) return FC2_ERR_INVALID_ARG;
    return fc2::debug_phasor(u, n, 1, out4) == cudaSuccess ? FC2_OK : FC2_ERR_CUDA;
}

/* Kernels launched by the last fc2_execute_batched call of this process. */
int64_t fc2_debug_batch_launches(void) { return g_last_batch_launches; }

/* Bins of the last fc2_execute_batched call that were re-solved in double,
 * recomputed from float, double-float and double exact sums, and the number
 * of chunk graphs launched (out5[0..4]). */
void fc2_debug_batch_counts(int64_t* out5) {
    if (out5)
        for (int i = 0; i < 5; ++i) out5[i] = g_last_batch_stats[i];
}

/* Host wall milliseconds of the last fc2_execute_batched call in seven phases
 * (out7[0..6]): setup before the chunk loop; per chunk (summed): buffer
 * allocation and input uploads, moments and the wait for them, chunk layout and table uploads,
 * graph capture / update and launch, the wait for the chunk's kernels and
 * results; release of the buffers at the end. */
void fc2_debug_batch_timing(int enable) { set_batch_timing(enable != 0); }

/* Launch configuration of the last fc2_execute_batched call's last chunk
 * (out12): [0] source (0 fixed, 1 tuning table, 2 tuned in the call),
 * [1] transform family (0 radix-16 shared memory, 1 two register stages,
 * 2 bulk copies), [2] spreading tile cells, [3] assembly block threads,
 * [4] samples per exact-sum work item, [5] transform passes, [6..9] their
 * log2 radices, [10] configurations timed, [11] tuning milliseconds (host
 * wall time, as the bits of a double), [12] grids per transform group (0 =
 * all). */
void fc2_debug_batch_config(int64_t* out13) {
    if (out13)
        for (int i = 0; i < 13; ++i) out13[i] = g_last_batch_stats[18 + i];
}

/* Fixed configuration for batched calls that do not tune (autotune -1 or a
 * transform family requested): spreading tile 512 / 1024 / 2048 cells,
 * assembly block 128 / 256 threads, work item 1024 / 2048 / 4096 samples;
 * 0 (or a value the grid does not allow) keeps the default. */
void fc2_debug_batch_force(int spread_tile, int asm_nt, int bx_ch, int fft_group) {
    fc2::force_batch_config(spread_tile, asm_nt, bx_ch, fft_group);
}

/* Fixed transform plan for batched calls that do not tune: log2 radices
 * rs[0..n) and kernel family (0 radix-16 shared memory, 1 register stages,
 * 2 bulk copies); used only when it is one of the tuner's candidates for the
 * grid length; n = 0 clears it. */
void fc2_debug_batch_force_plan(const int* rs, int n, int family) {
    if (n < 0 || n > 4 || (n > 0 && !rs)) return;
    fc2::force_batch_plan(rs, n, family);
}

/* Forget the batched path's tuning table of this process (the cache file is
 * read again at the next lookup). */
void fc2_debug_batch_forget_tuning(void) { fc2::forget_batch_tuning(); }
void fc2_debug_spread_force_general(int on) { fc2::force_spread_general(on); }

void fc2_debug_batch_stage_ms(double* out6) {
    if (out6)
        for (int i = 0; i < 6; ++i) std::memcpy(&out6[i], &g_last_batch_stats[12 + i], 8);
}

void fc2_debug_batch_phase_ms(double* out7) {
    if (out7)
        for (int i = 0; i < 7; ++i) std::memcpy(&out7[i], &g_last_batch_stats[5 + i], 8);
}

/* Stage timing: while enabled, each execute records CUDA events on the plan's
 * stream around (0) phase reduction + spreading, (1) FFT passes, (2) assembly
 * and solve, (3) exact fix-up, (4) peaks and coefficients; fc2_stage_times
 * returns the mean milliseconds per execute of each stage since enabling.
 * Also reports the kernels launched by the last execute and the algorithmic
 * bytes of the FFT passes. */
fc2_status fc2_stage_timing(fc2_plan p, int enable) {
    if (!p) return FC2_ERR_INVALID_ARG;
    if (enable && !p->ev[0])
        for (int i = 0; i < 8; ++i)
            if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return FC2_ERR_CUDA;
    p->timing = enable != 0;
    for (int i = 0; i < 8; ++i) p->stage_ms[i] = 0.0;
    p->stage_n = 0;
    return FC2_OK;
}

fc2_status fc2_significance(fc2_plan p, double* log_p, int64_t* j_min, double* log_p_min,
                            double* adj_scale) {
    if (!p || !p->executed) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return FC2_ERR_CUDA;
    cudaStream_t s = p->stream;
    const int H = p->H;
    const size_t cells = (size_t)H * p->N;
    bool direct = false;
    if (log_p) {
        cudaPointerAttributes at;
        direct = cudaPointerGetAttributes(&at, log_p) == cudaSuccess &&
                 at.type == cudaMemoryTypeDevice && at.device == p->device;
        cudaGetLastError();
    }
    Guard g;
    double* dlp = nullptr;
    char* small = nullptr;  // jmin [H] int64, lpmin [H], adj [H]
    if (log_p && !direct) g.ok(pool_alloc((void**)&dlp, cells * 8, s));
    g.ok(pool_alloc((void**)&small, (size_t)H * 24, s));
    if (g.e == cudaSuccess) {
        int64_t* djmin = (int64_t*)small;
        double* dlpmin = (double*)(small + (size_t)H * 8);
        double* dadj = (double*)(small + (size_t)H * 16);
        g.ok(launch_significance(p, direct ? log_p : dlp, djmin, dlpmin, dadj, s));
        std::vector<char> hs((size_t)H * 24);
        g.ok(cudaMemcpyAsync(hs.data(), small, hs.size(), cudaMemcpyDeviceToHost, s));
        if (log_p && !direct) g.ok(cudaMemcpyAsync(log_p, dlp, cells * 8, cudaMemcpyDeviceToHost, s));
        g.ok(cudaStreamSynchronize(s));
        if (g.e == cudaSuccess) {
            if (j_min) memcpy(j_min, hs.data(), (size_t)H * 8);
            if (log_p_min) memcpy(log_p_min, hs.data() + (size_t)H * 8, (size_t)H * 8);
            if (adj_scale) memcpy(adj_scale, hs.data() + (size_t)H * 16, (size_t)H * 8);
        }
    }
    if (dlp) cudaFreeAsync(dlp, s);
    if (small) cudaFreeAsync(small, s);
    return map_err(g.e);
}

fc2_status fc2_trim_device_memory(int device) {
    cudaMemPool_t pool = existing_pool(device);
    if (!pool) return FC2_OK;
    if (cudaSetDevice(device) != cudaSuccess) return FC2_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return FC2_ERR_CUDA;
    drop_deconv_cache(device);
    if (cudaDeviceSynchronize() != cudaSuccess) return FC2_ERR_CUDA;
    return cudaMemPoolTrimTo(pool, 0) == cudaSuccess ? FC2_OK : FC2_ERR_CUDA;
}

fc2_status fc2_stage_times(fc2_plan p, double* ms5, int64_t* launches, double* fft_bytes) {
    if (!p) return FC2_ERR_INVALID_ARG;
    if (ms5)
        for (int i = 0; i < 5; ++i) ms5[i] = p->stage_n ? p->stage_ms[i] / (double)p->stage_n : 0.0;
    if (launches) *launches = p->launches;
    if (fft_bytes) *fft_bytes = p->fft_bytes;
    return FC2_OK;
}

}  // extern "C"
