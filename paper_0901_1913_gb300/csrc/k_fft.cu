// k_fft.cu -- FFTs of the spread grids and the kernel-transform deconvolution table.
//
// Paper: Sec. 2 ("P and Q can be efficiently computed by the application of the
// FFT to p and q"), Sec. 3b (FFT of the gridded arrays).  The sign is
// e^{+i 2 pi f t} as in Eq. "eqPQ".
//
// Layout: grid g occupies M = 2^logM complex cells.  The transform is a
// sequence of Stockham passes through HBM; each pass gives every CTA J
// adjacent columns of R = 2^logR rows (a tile of R x J complex values staged
// in shared memory), applies the inter-pass twiddles, runs an in-CTA
// Stockham DFT of length R built from radix-16/8/4/2 register butterflies and
// writes the tile back in autosorted order.  The first pass reads only the
// rows that hold samples (the rest of the grid is zero padding); the last
// pass keeps only the N centred modes and writes them, in trial-frequency
// order, to the spectrum array.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "fc2_common.cuh"
#include "fc2_internal.h"

namespace fc2 {

// ------------------------------------------------------------------ twiddles
// w_M^q = hi[q >> sh] * lo[q & (2^sh - 1)], each table entry rounded once from
// a double sincospi with an exact rational argument.
template <typename T>
__global__ void k_init_tw(cpx<T>* lo, int64_t nlo, cpx<T>* hi, int64_t nhi, int logM, int sh) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double inv = ldexp(2.0, -logM);  // 2 / M
    double s, c;
    if (i < nlo) {
        sincospi((double)i * inv, &s, &c);
        lo[i] = mk<T>((T)c, (T)s);
    }
    if (i < nhi) {
        sincospi((double)(i << sh) * inv, &s, &c);
        hi[i] = mk<T>((T)c, (T)s);
    }
}

template <typename T>
FC2_D cpx<T> twiddle(const cpx<T>* __restrict__ lo, const cpx<T>* __restrict__ hi, int sh,
                     int64_t q) {
    return mul(hi[q >> sh], lo[q & ((1ll << sh) - 1)]);
}

// ---------------------------------------------------------- deconvolution
// dec[j] = 1 / phihat((j - hN) / M), phihat the kernel's Fourier transform,
// evaluated from a Chebyshev expansion in xi^2 fitted on the host.
__host__ __device__ inline double cheb_clenshaw(const double* c, int nc, double x) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = nc - 1; k >= 1; --k) {
        double b0 = 2.0 * x * b1 - b2 + c[k];
        b2 = b1;
        b1 = b0;
    }
    return x * b1 - b2 + c[0];
}

constexpr int CHEB_N = 64;

// phihat is even: thread m (0 <= m <= max(hN, N - hN)) fills both j = hN + m and
// j = hN - m.
template <typename T>
__global__ void k_init_dec(T* dec, int64_t N, int64_t hN, int64_t M, const double* cheb,
                           int nc, double ymax) {
    __shared__ double c[CHEB_N];
    if (threadIdx.x < CHEB_N) c[threadIdx.x] = cheb[threadIdx.x];
    __syncthreads();
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m > hN && m >= N - hN) return;
    double xi = (double)m / (double)M;
    double y = xi * xi;
    double xx = 2.0 * y / ymax - 1.0;
    T v = (T)(1.0 / cheb_clenshaw(c, nc, xx));
    if (hN + m < N) dec[hN + m] = v;
    if (m > 0 && hN - m >= 0) dec[hN - m] = v;
}

// dec[j] = 1 / phihat((sh + j) / M), j < N.
__global__ void k_init_dec_shift(float* dec, int64_t N, int64_t sh, int64_t M,
                                 const double* cheb, int nc, double ymax) {
    __shared__ double c[CHEB_N];
    if (threadIdx.x < CHEB_N) c[threadIdx.x] = cheb[threadIdx.x];
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double xi = (double)(sh + j) / (double)M;
    dec[j] = (float)(1.0 / cheb_clenshaw(c, nc, 2.0 * xi * xi / ymax - 1.0));
}

int cheb_fit_kernel_ft(int w, double beta, double xi_max, double* coef, double trim) {
    int nq = 2 * w + 16;
    std::vector<double> gx(nq), gw(nq);
    gauss_legendre(nq, gx.data(), gw.data());
    const double ymax = xi_max * xi_max;
    std::vector<double> f(CHEB_N);
    for (int i = 0; i < CHEB_N; ++i) {
        double xc = cos(M_PI * (i + 0.5) / CHEB_N);
        double y = 0.5 * ymax * (xc + 1.0);
        f[i] = kernel_ft_host(w, beta, sqrt(y), nq, gx.data(), gw.data());
    }
    for (int k = 0; k < CHEB_N; ++k) {
        double acc = 0.0;
        for (int i = 0; i < CHEB_N; ++i) acc += f[i] * cos(M_PI * k * (i + 0.5) / CHEB_N);
        coef[k] = acc * 2.0 / CHEB_N;
    }
    coef[0] *= 0.5;
    // drop the negligible tail of the expansion
    double mx = 0.0;
    for (int k = 0; k < CHEB_N; ++k) mx = std::max(mx, fabs(coef[k]));
    int nc = CHEB_N;
    while (nc > 2 && fabs(coef[nc - 1]) < trim * mx) --nc;
    return nc;
}

double cheb_eval_host(const double* coef, double xi, double xi_max) {
    double ymax = xi_max * xi_max;
    return cheb_clenshaw(coef, CHEB_N, 2.0 * xi * xi / ymax - 1.0);
}

// Deconvolution tables depend only on the plan's geometry (device, N, M, the
// kernel, the shift, the precision), so plans of the same geometry copy them
// from a small process-wide cache instead of evaluating N Chebyshev sums in
// double again.  Entries are kept in the library's device pool until
// fc2_trim_device_memory drops them; at most DEC_CACHE_MAX at a time.
struct DecKey {
    int dev, kind, fp64, w;
    int64_t N, M, sh;
    double beta;
    bool operator<(const DecKey& o) const {
        return std::tie(dev, kind, fp64, w, N, M, sh, beta) <
               std::tie(o.dev, o.kind, o.fp64, o.w, o.N, o.M, o.sh, o.beta);
    }
};
constexpr size_t DEC_CACHE_MAX = 8;
static std::mutex g_dec_mu;
static std::map<DecKey, std::pair<void*, uint64_t>> g_dec_cache;  // table, last use
static uint64_t g_dec_clock = 0;

// Copy a cached table into dst (true), or return false.
static bool dec_cache_get(const DecKey& k, void* dst, size_t bytes, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_dec_mu);
    auto it = g_dec_cache.find(k);
    if (it == g_dec_cache.end()) return false;
    // finish the copy before the lock is released: an entry is only freed
    // under the lock, so no copy from it is ever pending then
    if (cudaMemcpyAsync(dst, it->second.first, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    it->second.second = ++g_dec_clock;
    return true;
}

// Keep a copy of a freshly computed table (best effort: a failed allocation
// only means no caching).
static void dec_cache_put(const DecKey& k, const void* src, size_t bytes, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_dec_mu);
    if (g_dec_cache.count(k)) return;
    if (g_dec_cache.size() >= DEC_CACHE_MAX) {
        auto old = g_dec_cache.begin();
        for (auto it = g_dec_cache.begin(); it != g_dec_cache.end(); ++it)
            if (it->second.second < old->second.second) old = it;
        cudaFreeAsync(old->second.first, s);
        g_dec_cache.erase(old);
    }
    void* buf = nullptr;
    if (pool_alloc(&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaMemcpyAsync(buf, src, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(buf, s);
        return;
    }
    g_dec_cache[k] = {buf, ++g_dec_clock};
}

void drop_deconv_cache(int dev) {
    std::lock_guard<std::mutex> lk(g_dec_mu);
    for (auto it = g_dec_cache.begin(); it != g_dec_cache.end();) {
        if (it->first.dev == dev) {
            cudaFreeAsync(it->second.first, (cudaStream_t)0);
            it = g_dec_cache.erase(it);
        } else {
            ++it;
        }
    }
}

cudaError_t init_deconv(fc2_plan_s* p, cudaStream_t s) {
    double coef[CHEB_N];
    int dev = 0;
    cudaGetDevice(&dev);
    double* d_coef = (double*)p->d_red;  // scratch, consumed before any other use
    cudaError_t e;
    if (p->packed) goto packed;  // every grid is packed: only the shifted table is used
    {
    const int64_t hN = p->N / 2;
    const double xi_max = (double)std::max(hN, p->N - hN) / (double)p->M;
    // drop the expansion's tail below the table's precision
    const int nc = cheb_fit_kernel_ft(p->w, p->beta, xi_max, coef, p->fp64 ? 1e-18 : 1e-11);
    e = cudaMemcpyAsync(d_coef, coef, sizeof(coef), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const int64_t mmax = std::max(hN, p->N - hN);
    unsigned blocks = (unsigned)((mmax + 256) / 256);
    const DecKey key{dev, 0, p->fp64 ? 1 : 0, p->w, p->N, p->M, 0, p->beta};
    const size_t bytes = (size_t)p->N * (p->fp64 ? 8 : 4);
    if (!dec_cache_get(key, p->d_dec, bytes, s)) {
        if (p->fp64)
            k_init_dec<double><<<blocks, 256, 0, s>>>((double*)p->d_dec, p->N, hN, p->M, d_coef,
                                                      nc, xi_max * xi_max);
        else
            k_init_dec<float><<<blocks, 256, 0, s>>>((float*)p->d_dec, p->N, hN, p->M, d_coef,
                                                     nc, xi_max * xi_max);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dec_cache_put(key, p->d_dec, bytes, s);
    }
    }
packed:
    if (p->npk > 0) {
        // packed grids: dec_p[j] = 1 / phihat_p((sh + j) / M) (the modes -(sh + j)
        // share it: phihat is even)
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        const DecKey key{dev, 1, 0, p->w_p, p->N, p->M, p->sh, p->beta_p};
        const size_t bytes = (size_t)p->N * 4;
        if (!dec_cache_get(key, p->d_dec_p, bytes, s)) {
            const double xi_p = (double)(p->sh + p->N) / (double)p->M;
            const int ncp = cheb_fit_kernel_ft(p->w_p, p->beta_p, xi_p, coef, 1e-11);
            e = cudaMemcpyAsync(d_coef, coef, sizeof(coef), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
            k_init_dec_shift<<<(unsigned)((p->N + 255) / 256), 256, 0, s>>>(
                (float*)p->d_dec_p, p->N, p->sh, p->M, d_coef, ncp, xi_p * xi_p);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            dec_cache_put(key, p->d_dec_p, bytes, s);
        }
    }
    // the coefficients live in reduction scratch: finish before it is reused
    return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------ in-CTA DFT
// Shared tile of R rows x J columns; element (r, jj) has logical index
// e = r * J + jj and lives at phys(e) = e + e / 32 (one pad slot per 32
// elements keeps the strided butterfly writes free of bank conflicts).
FC2_HD constexpr int phys(int e) { return e + (e >> 5); }

// ------------------------------------------------ index arithmetic of the stores
// Shared by the pass kernels and the host replay that checks a plan's index
// ranges (fc2_debug_fft_plan_check).
//
// Element e of a tile on its way to the next pass (tile width 2^LOGJ, next
// pass's tile width 2^LOGJn): jj = its column, k = its output row.
struct TileElem {
    int k, jj;
};
FC2_HD TileElem tile_elem(int e, int LOGJn, int LOGJ) {
    const int kl = e & ((1 << LOGJn) - 1);
    const int jj = (e >> LOGJn) & ((1 << LOGJ) - 1);
    const int kb = e >> (LOGJn + LOGJ);
    return TileElem{(kb << LOGJn) + kl, jj};
}
// Logical (Stockham autosort) index of output k of column j of a pass of radix
// 2^LOGR after passes of radix product 2^logNs.
FC2_HD int64_t stockham_out(int64_t j, int k, int logNs, int LOGR) {
    return ((j >> logNs) << (logNs + LOGR)) + (j & ((1ll << logNs) - 1)) + ((int64_t)k << logNs);
}
// Where the next pass (radix 2^logRn, tile width 2^LOGJn, logSn = logM - logRn)
// finds logical index i in its blocked layout: tile i mod Sn / Jn, row
// i / Sn, column i mod Jn.
FC2_HD int64_t blocked_pos(int64_t i, int logSn, int LOGJn, int logBlk) {
    const int64_t jn = i & ((1ll << logSn) - 1), rn = i >> logSn;
    return ((jn >> LOGJn) << logBlk) + (rn << LOGJn) + (jn & ((1ll << LOGJn) - 1));
}
// The same when the logical index is j R + kr (a first pass whose radix and
// the next one's multiply to the grid length): row kr of column j.
FC2_HD int64_t rowcol_pos(int kr, int64_t j, int LOGJn, int logBlk) {
    return ((int64_t)(kr >> LOGJn) << logBlk) + (j << LOGJn) + (kr & ((1 << LOGJn) - 1));
}

// Stage decomposition of a length-2^LOGR DFT: the first stage takes LOGR % 4
// bits (if nonzero), every other stage 4 bits (radix 16).
FC2_HD constexpr int stage_bits(int LOGR, int DONE) {
    return (DONE == 0 && (LOGR % 4) != 0) ? (LOGR % 4) : ((LOGR - DONE) >= 4 ? 4 : (LOGR - DONE));
}
// Twiddles of stage (Ns = 2^DONE, radix Q): table entry [(k-1) Ns + pm] =
// w_{Ns Q}^{k pm}; stages are stored one after the other.
FC2_HD constexpr int stage_tw_size(int LOGR) {
    int tot = 0, done = 0;
    while (done < LOGR) {
        int qb = stage_bits(LOGR, done);
        if (done > 0) tot += ((1 << qb) - 1) * (1 << done);
        done += qb;
    }
    return tot;
}

template <typename T>
__global__ void k_init_stage_tw(cpx<T>* tw, int LOGR) {
    // thread i computes entry i of the concatenated stage tables
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0, done = 0;
    while (done < LOGR) {
        int qb = stage_bits(LOGR, done);
        if (done > 0) {
            int ns = 1 << done, q = 1 << qb;
            int sz = (q - 1) * ns;
            if (i >= off && i < off + sz) {
                int k = (i - off) / ns + 1, pm = (i - off) % ns;
                double sn, cn;
                // w_{ns q}^{k pm}: exact rational argument 2 k pm / (ns q)
                sincospi(2.0 * (double)(k * pm) / (double)(ns * q), &sn, &cn);
                tw[i] = mk<T>((T)cn, (T)sn);
                return;
            }
            off += sz;
        }
        done += qb;
    }
}

struct TwgArgs {
    int j0;       // first column of the tile
    int nsg_mask; // NsG - 1 (NsG = product of earlier passes' radices)
    int lts;      // log2(M / (NsG R))
    int tws;      // two-level table split
};

// One in-CTA Stockham stage of radix Q (Ns = 2^DONE): butterfly (pp, jj) reads
// rows pp + k R/Q, multiplies by w_{Ns Q}^{k (pp % Ns)} and writes rows
// (pp / Ns) Ns Q + pp % Ns + k Ns.  With TWG (first stage of a later pass) the
// inter-pass twiddle w_M^{r (j % NsG) M/(NsG R)} of each element is applied as
// it is read; it is built as base * step^k from four table lookups per
// butterfly.
template <typename T, int R, int J, int NT, int QB, int DONE, int TOFF, bool TWG>
FC2_D void cta_stage(cpx<T>* s, const cpx<T>* st, const TwgArgs& tg,
                     const cpx<T>* __restrict__ twlo, const cpx<T>* __restrict__ twhi) {
    constexpr int Q = 1 << QB;
    constexpr int NS = 1 << DONE;
    constexpr int NB = (R / Q) * J;
    constexpr int PER = NB / NT;
    static_assert(PER * NT == NB, "butterflies must divide evenly");
    cpx<T> v[PER][Q];
    int idx[PER], jj_[PER];
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int bi = threadIdx.x + b * NT;
        const int jj = bi % J, pp = bi / J;
#pragma unroll
        for (int k = 0; k < Q; ++k) v[b][k] = s[phys((pp + k * (R / Q)) * J + jj)];
        if constexpr (TWG) {
            const int jm = (tg.j0 + jj) & tg.nsg_mask;
            if (jm != 0) {
                const cpx<T> base = twiddle(twlo, twhi, tg.tws, (int64_t)((pp * jm) << tg.lts));
                const cpx<T> st1 = twiddle(twlo, twhi, tg.tws, (int64_t)(((R / Q) * jm) << tg.lts));
                cpx<T> lo[4], hi[4];
                lo[0] = mk<T>((T)1, (T)0);
                lo[1] = st1;
                if constexpr (Q > 2) { lo[2] = mul(st1, st1); lo[3] = mul(lo[2], st1); }
                if constexpr (Q > 4) {
                    hi[1] = mul(lo[2], lo[2]);
                    if constexpr (Q > 8) { hi[2] = mul(hi[1], hi[1]); hi[3] = mul(hi[2], hi[1]); }
                }
                v[b][0] = mul(v[b][0], base);
#pragma unroll
                for (int k = 1; k < Q; ++k) {
                    cpx<T> w = base;
                    if ((k & 3) != 0) w = mul(w, lo[k & 3]);
                    if ((k >> 2) != 0) w = mul(w, hi[k >> 2]);
                    v[b][k] = mul(v[b][k], w);
                }
            }
        }
        const int pm = pp % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int k = 1; k < Q; ++k) v[b][k] = mul(v[b][k], st[TOFF + (k - 1) * NS + pm]);
        }
        SmallDFT<T, Q>::run(v[b]);
        idx[b] = (pp / NS) * NS * Q + pm;
        jj_[b] = jj;
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < PER; ++b)
#pragma unroll
        for (int k = 0; k < Q; ++k) s[phys((idx[b] + k * NS) * J + jj_[b])] = v[b][k];
    __syncthreads();
}

template <typename T, int LOGR, int J, int NT, int DONE, int TOFF>
struct CtaDft {
    static FC2_D void run(cpx<T>* s, const cpx<T>* st, const TwgArgs& tg, bool twg,
                          const cpx<T>* twlo, const cpx<T>* twhi) {
        constexpr int R = 1 << LOGR;
        if constexpr (DONE < LOGR) {
            constexpr int QB = stage_bits(LOGR, DONE);
            constexpr int NTOFF = TOFF + (DONE > 0 ? ((1 << QB) - 1) * (1 << DONE) : 0);
            if (DONE == 0 && twg)
                cta_stage<T, R, J, NT, QB, DONE, TOFF, true>(s, st, tg, twlo, twhi);
            else
                cta_stage<T, R, J, NT, QB, DONE, TOFF, false>(s, st, tg, twlo, twhi);
            CtaDft<T, LOGR, J, NT, DONE + QB, NTOFF>::run(s, st, tg, twg, twlo, twhi);
        }
    }
};

FC2_D void cp_async8(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
FC2_D void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
FC2_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <typename T>
FC2_D void cp_elem(cpx<T>* smem, const cpx<T>* gmem) {
    if constexpr (sizeof(cpx<T>) == 16) cp_async16(smem, gmem);
    else cp_async8(smem, gmem);
}

struct PassArgs {
    int logM;
    int logNs;         // log2 of the product of the radices of earlier passes
    int first, last;
    int logRn, logJn;  // radix and tile width of the next pass (blocked output layout)
    int N, hN;
    int tws;
    int npk, sh;       // packed grids (g < npk) keep modes +-(sh + j), others j - hN
    int g0, ng;        // this launch covers grids g0 .. g0 + ng - 1
};

// Last pass: mode m of grid g goes to its place in the spectra.  Grid
// g < npk (packed) stores F(sh + j) at [2g][j] and F(-(sh + j)) at [2g + 1][j];
// any other grid stores F(j - hN) at [npk + g][j].
template <typename T>
FC2_D void store_mode(cpx<T>* __restrict__ spec, const PassArgs& a, int g, int m, cpx<T> v) {
    if (g < a.npk) {
        const int jp = m - a.sh;
        if (jp >= 0 && jp < a.N) spec[(int64_t)(2 * g) * a.N + jp] = v;
        const int jm = -m - a.sh;
        if (jm >= 0 && jm < a.N) spec[(int64_t)(2 * g + 1) * a.N + jm] = v;
    } else {
        const int jf = m + a.hN;
        if (jf >= 0 && jf < a.N) spec[(int64_t)(a.npk + g) * a.N + jf] = v;
    }
}

// One pass of the transform.  Logical Stockham indexing: column j (0 <= j < S,
// S = M / R) takes rows r of X[j + r S]; output k of its length-R DFT is
// X'[(j / Ns) Ns R + (j % Ns) + k Ns].
// Physical layouts: the first pass reads the spread grid directly (row r of a
// tile is J contiguous cells at j0 + r S; rows r >= ceil(L_g / S) are zero
// padding and are not read).  Every later pass reads its input in the
// "blocked" layout its predecessor wrote: the R x J tile of columns
// [b J, (b + 1) J) is one contiguous run, element (r, jj) at b R J + r J + jj.
// The last pass writes only the N centred modes m = o or o - M (o the output
// index), in trial-frequency order, to spec[g][m + hN].
template <typename T, int LOGR, int LOGJ, int NT>
__global__ void __launch_bounds__(NT, 2) k_fft_pass(const cpx<T>* __restrict__ in,
                                                    cpx<T>* __restrict__ out, PassArgs a,
                                                    const int64_t* __restrict__ Lg,
                                                    const cpx<T>* __restrict__ twlo,
                                                    const cpx<T>* __restrict__ twhi,
                                                    const cpx<T>* __restrict__ twst) {
    constexpr int R = 1 << LOGR;
    constexpr int J = 1 << LOGJ;
    constexpr int E = R * J;
    constexpr int NST = stage_tw_size(LOGR);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* st = s + phys(E - 1) + 1;
    const int M = 1 << a.logM;
    const int S = M >> LOGR;
    const int g = a.g0 + (int)blockIdx.y;
    const int j0 = blockIdx.x * J;
    const cpx<T>* gin = in + (int64_t)g * M;
    if (a.first) {
        const int L = (int)Lg[g];
        int rows = (L + S - 1) / S;
        if (rows > R) rows = R;
        for (int e = threadIdx.x; e < E; e += NT) {
            const int r = e >> LOGJ, jj = e & (J - 1);
            if (r < rows) cp_elem(&s[phys(e)], &gin[j0 + jj + r * S]);
            else s[phys(e)] = mk<T>((T)0, (T)0);
        }
    } else {
        const cpx<T>* src = gin + (int64_t)blockIdx.x * E;
        for (int e = threadIdx.x; e < E; e += NT) cp_elem(&s[phys(e)], &src[e]);
    }
    for (int i = threadIdx.x; i < NST; i += NT) cp_elem(&st[i], &twst[i]);
    cp_async_wait_all();
    __syncthreads();
    TwgArgs tg;
    tg.j0 = j0;
    tg.nsg_mask = (1 << a.logNs) - 1;
    tg.lts = a.logM - a.logNs - LOGR;
    tg.tws = a.tws;
    CtaDft<T, LOGR, J, NT, 0, 0>::run(s, st, tg, a.logNs > 0, twlo, twhi);
    const int logNs = a.logNs;
    if (!a.last) {
        cpx<T>* gout = out + (int64_t)g * M;
        const int LOGJn = a.logJn;
        const int logBlk = a.logRn + a.logJn;  // Rn * Jn
        if (logNs == 0 && a.logM - a.logRn == LOGR) {
            // two-pass plan: logical output j R + k is column k, row j of the
            // next (last) pass
            for (int e = threadIdx.x; e < E; e += NT) {
                const TileElem te = tile_elem(e, LOGJn, LOGJ);
                gout[rowcol_pos(te.k, j0 + te.jj, LOGJn, logBlk)] = s[phys(te.k * J + te.jj)];
            }
        } else {
            const int logSn = a.logM - a.logRn;
            for (int e = threadIdx.x; e < E; e += NT) {
                const TileElem te = tile_elem(e, LOGJn, LOGJ);
                const int64_t i = stockham_out(j0 + te.jj, te.k, logNs, LOGR);
                gout[blocked_pos(i, logSn, LOGJn, logBlk)] = s[phys(te.k * J + te.jj)];
            }
        }
    } else {
        for (int e = threadIdx.x; e < E; e += NT) {
            const int k = e >> LOGJ, jj = e & (J - 1);
            const int o = j0 + jj + (k << logNs);
            const int m = (o < M / 2) ? o : o - M;
            store_mode<T>(out, a, g, m, s[phys(e)]);
        }
    }
}

// Store of a transformed tile, staged in shared memory (tile element k J + jj
// at shared index sidx(k J + jj)), into the blocked layout the next pass
// reads: logical output i of column j = j0 + jj goes to row i >> logSn,
// column i mod Sn of that layout.  In a first pass into a pass of smaller
// radix (logNs = 0, R | Sn) the row and column block of i = j R + k depend on
// j alone, so element (kb, kl, jj), k = kb Jn + kl, lands at base(j) +
// kb Rn Jn + kl; each thread keeps jj and kl and walks kb.
template <int LOGR, int LOGJ, int NT, typename T, typename SIdx>
FC2_D void store_tile_blocked(cpx<T>* __restrict__ gout, const cpx<T>* s, SIdx sidx, int j0,
                              const PassArgs& a, int tid) {
    constexpr int J = 1 << LOGJ, E = (1 << LOGR) * J;
    const int logNs = a.logNs;
    const int LOGJn = a.logJn, Jn = 1 << a.logJn;
    const int logBlk = a.logRn + a.logJn;
    const int logSn = a.logM - a.logRn;
    if (logNs == 0 && LOGR <= logSn && LOGJn <= LOGR && (Jn << LOGJ) <= NT) {
        const int kl = tid & (Jn - 1);
        const int jj = (tid >> LOGJn) & (J - 1);
        const int kb0 = tid >> (LOGJn + LOGJ);
        const int i0 = (j0 + jj) << LOGR;
        const int jb = i0 & ((1 << logSn) - 1), rn = i0 >> logSn;
        cpx<T>* dst = gout + ((int64_t)((jb >> LOGJn) + kb0) << logBlk) + (rn << LOGJn) + kl;
        const int e0 = (kb0 << (LOGJn + LOGJ)) + (kl << LOGJ) + jj;  // k J + jj
        const int dkb = NT >> (LOGJn + LOGJ);
#pragma unroll 8
        for (int it = 0; it < E / NT; ++it) dst[(int64_t)(it * dkb) << logBlk] = s[sidx(e0 + it * NT)];
        return;
    }
    for (int e = tid; e < E; e += NT) {
        const TileElem te = tile_elem(e, LOGJn, LOGJ);
        const int64_t i = stockham_out(j0 + te.jj, te.k, logNs, LOGR);
        gout[blocked_pos(i, logSn, LOGJn, logBlk)] = s[sidx(te.k * J + te.jj)];
    }
}

// ------------------------------------------------- pruned small transform
// Q-point DFT (sign +) of v when only v[0..MZ) can be nonzero: with
// k = (Q/MZ) k1 + k2, X_k = sum_{n<MZ} (v_n w_Q^{n k2}) w_MZ^{n k1}, i.e. Q/MZ
// twiddled MZ-point transforms (MZ = 1: every output is v_0).
template <typename T, int Q, int MZ>
struct PrunedDFT {
    static FC2_D void run(cpx<T>* v) {
        constexpr int D = Q / MZ;
        cpx<T> x[MZ];
#pragma unroll
        for (int n = 0; n < MZ; ++n) x[n] = v[n];
#pragma unroll
        for (int k2 = 0; k2 < D; ++k2) {
            cpx<T> y[MZ];
#pragma unroll
            for (int n = 0; n < MZ; ++n)
                y[n] = (n * k2 == 0) ? x[n] : mul(x[n], root64<T>(((64 / Q) * n * k2) & 63));
            SmallDFT<T, MZ>::run(y);
#pragma unroll
            for (int k1 = 0; k1 < MZ; ++k1) v[D * k1 + k2] = y[k1];
        }
    }
};

// ------------------------------------------------- two-stage radix-64 pass
// Float passes of radix R = 2^10..2^12 in two register stages, QA = R/64 then
// 64, with 128 threads per 8192-element tile.  Stage A reads its butterfly
// straight from global memory (coalesced along the tile's columns), applies
// the inter-pass twiddle and writes to shared memory; stage B reads, applies
// the stage twiddle w_R^{k pp}, and writes its outputs back to the same slots;
// then the tile is stored as by k_fft_pass.  Shared memory holds one tile,
// swizzled (bits [LOGJ, LOGJ + 3) of the element index XORed with bits
// [7, 10)) so both stages' access patterns reach the minimum number of
// shared-memory wavefronts, plus the stage-B twiddles.  The kernel is
// persistent: each CTA walks tiles with a stride of the grid size and asks L2
// to prefetch its next tile while it computes the current one.
// With 16-column tiles (LOGJ = 4) a row is one 128-byte bank row, and the
// row's low four bits are XORed into the column instead: the stage-A writes
// (rows pp QA + k, columns across a warp), the stage-B reads with columns
// across a warp and those with 16 consecutive rows across a warp (the
// row-first store below) then each take the minimum two wavefronts.
template <int LOGJ>
FC2_HD int swz(int e) {
    if constexpr (LOGJ == 4) return e ^ ((e >> 4) & 15);
    else return e ^ (((e >> 7) & 7) << LOGJ);
}

FC2_D void prefetch_l2_bulk(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
FC2_D void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }

// Stage-B twiddles of the register passes: entry (k - 1) QA + pm = w_R^{k pm},
// k = 1 .. RB - 1, pm < QA = R / RB (RB = 2^LRB).
template <typename T>
__global__ void k_init_tw64(cpx<T>* tw, int LOGR, int LRB) {
    const int QA = 1 << (LOGR - LRB);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ((1 << LRB) - 1) * QA) return;
    const int k = i / QA + 1, pm = i % QA;
    double sn, cn;
    sincospi(2.0 * (double)(k * pm) / (double)(1 << LOGR), &sn, &cn);
    tw[i] = mk<T>((T)cn, (T)sn);
}

constexpr int P64_NT = 256;                 // threads of a radix-64 pass CTA (one CTA per SM)
constexpr int P64_LOGE = 14;                // log2 of its tile: 64 elements per thread
constexpr int P32_NT = 512;                 // threads of the radix-32 variant (same tile)

// The pass body for a stage-B radix RB (64: 256 threads of 64 elements; 32:
// 512 threads of 32 elements -- the same tile with twice the warps and half
// the registers per thread).
template <int RB, int LOGR, int LOGJ>
FC2_D void regpass_body(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                        const PassArgs& a, const int64_t* __restrict__ Lg,
                        const cpx<float>* __restrict__ twlo, const cpx<float>* __restrict__ twhi,
                        const cpx<float>* __restrict__ tw64, int G) {
    using T = float;
    constexpr int LRB = RB == 64 ? 6 : 5;
    constexpr int R = 1 << LOGR, J = 1 << LOGJ, E = R * J, NT = RB == 64 ? P64_NT : P32_NT;
    constexpr int QAB = LOGR - LRB, QA = 1 << QAB;
    constexpr int PERA = RB / QA;  // stage-A butterflies per thread
    static_assert(RB == 64 || RB == 32, "stage-B radix 64 or 32");
    static_assert(E == RB * NT, "tile must be RB elements per thread");
    static_assert(PERA * NT == RB * J, "stage-A butterflies must divide evenly");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* s = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* st = s + E;
    const int M = 1 << a.logM;
    const int S = M >> LOGR;
    const int tiles_x = S >> LOGJ;
    const int ntiles = tiles_x * G;
    const int nsg_mask = (1 << a.logNs) - 1;
    const int lts = a.logM - a.logNs - LOGR;
    for (int i = threadIdx.x; i < (RB - 1) * QA; i += NT) cp_elem(&st[i], &tw64[i]);
    cp_async_wait_all();
    auto rows_of = [&](int g) {
        int rows = R;
        if (a.first) {
            const int L = (int)Lg[g];
            rows = (L + S - 1) / S;
            if (rows > R) rows = R;
        }
        return rows;
    };
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int gl = tile / tiles_x;
        const int g = a.g0 + gl;
        const int bx = tile - gl * tiles_x;
        const int j0 = bx * J;
        const cpx<T>* gin = in + (int64_t)g * M;
        // ask L2 for the tile this CTA handles next
        {
            const int tn = tile + gridDim.x;
            if (tn < ntiles) {
                const int gnl = tn / tiles_x, bn = tn - gnl * tiles_x, gn = a.g0 + gnl;
                const cpx<T>* ginn = in + (int64_t)gn * M;
                if (!a.first) {
                    constexpr int CH = 4096;  // bytes per prefetch request
                    constexpr int NCH = E * (int)sizeof(cpx<T>) / CH;
                    const char* base = reinterpret_cast<const char*>(ginn + (int64_t)bn * E);
                    if (threadIdx.x < NCH) prefetch_l2_bulk(base + threadIdx.x * CH, CH);
                } else {
                    const int rn = rows_of(gn);
                    for (int r = threadIdx.x; r < rn; r += NT) prefetch_l2(ginn + bn * J + r * S);
                }
            }
        }
        const int rows = rows_of(g);
        // ---- stage A: radix QA, rows pp + k RB -> rows pp QA + k.  In the first
        // pass only rows < `rows` hold samples, so only the leading
        // ceil(rows / RB) inputs of each stage-A transform can be nonzero: a
        // pruned transform (PrunedDFT) skips the zeros.
        auto stage_a = [&](auto mz_tag) {
            constexpr int MZ = decltype(mz_tag)::value;
#pragma unroll
            for (int b = 0; b < PERA; ++b) {
                const int bi = threadIdx.x + b * NT;
                const int jj = bi % J, pp = bi / J;  // pp < RB
                cpx<T> v[QA];
                if constexpr (MZ < QA) {
#pragma unroll
                    for (int k = 0; k < MZ; ++k) {
                        const int r = pp + k * RB;
                        v[k] = (r < rows) ? gin[j0 + jj + r * S] : mk<T>(0.f, 0.f);
                    }
                    PrunedDFT<T, QA, MZ>::run(v);
                } else {
                    if (a.first) {
#pragma unroll
                        for (int k = 0; k < QA; ++k) {
                            const int r = pp + k * RB;
                            v[k] = (r < rows) ? gin[j0 + jj + r * S] : mk<T>(0.f, 0.f);
                        }
                    } else {
                        const cpx<T>* src = gin + (int64_t)bx * E;
#pragma unroll
                        for (int k = 0; k < QA; ++k) v[k] = src[(pp + k * RB) * J + jj];
                    }
                    const int jm = (j0 + jj) & nsg_mask;
                    if (a.logNs > 0 && jm != 0) {
                        // w_M^{(pp + RB k) jm 2^lts} = base * step^k, step^k = lo[k & 7] hi[k >> 3];
                        // every factor is a table lookup (no chains of products)
                        // (base lo[q] formed once per q: the same products as per k)
                        cpx<T> bl[8], hi[8];
                        bl[0] = twiddle(twlo, twhi, a.tws, (int64_t)((pp * jm) << lts));
                        hi[0] = mk<T>(1.f, 0.f);
#pragma unroll
                        for (int q = 1; q < 8; ++q) {
                            bl[q] = mul(bl[0], twiddle(twlo, twhi, a.tws, (int64_t)((RB * q * jm) << lts)));
                            // only the factors k >> 3 < QA / 8 of this radix: their
                            // exponents stay below M (larger ones would not)
                            if (8 * q < QA)
                                hi[q] = twiddle(twlo, twhi, a.tws, (int64_t)((8 * RB * q * jm) << lts));
                        }
#pragma unroll
                        for (int k = 0; k < QA; ++k) {
                            cpx<T> w = bl[k & 7];
                            if ((k >> 3) != 0) w = mul(w, hi[k >> 3]);
                            v[k] = mul(v[k], w);
                        }
                    }
                    SmallDFT<T, QA>::run(v);
                }
#pragma unroll
                for (int k = 0; k < QA; ++k) s[swz<LOGJ>((pp * QA + k) * J + jj)] = v[k];
            }
        };
        int mz = QA;
        if (a.first) {
            const int kz = (rows + RB - 1) >> LRB;
            mz = 1;
            while (mz < kz && mz < QA) mz <<= 1;
        }
        if (mz >= QA) stage_a(std::integral_constant<int, QA>{});
        else if (mz == 1) stage_a(std::integral_constant<int, 1>{});
        else if (mz == 2) stage_a(std::integral_constant<int, 2>{});
        else if (mz == 4) stage_a(std::integral_constant<int, 4>{});
        else if (mz == 8) stage_a(std::integral_constant<int, (QA > 8 ? 8 : QA)>{});
        else if (mz == 16) stage_a(std::integral_constant<int, (QA > 16 ? 16 : QA)>{});
        else stage_a(std::integral_constant<int, (QA > 32 ? 32 : QA)>{});
        __syncthreads();
        // ---- stage B: radix RB, rows pp + k QA.  Where a warp's stores from
        // registers hit the same 32-byte sectors as a smem-staged store would
        // (the last pass, and a next pass of the same radix), the results go
        // straight to global memory; otherwise they are staged in place.
        const int logNs = a.logNs;
        const bool same_radix = (logNs == 0 && a.logM - a.logRn == LOGR);
        {
            // a store of the next pass's rows from registers fills whole lines when
            // a warp holds 16 consecutive rows of one column (the next pass's
            // layout is row-contiguous within a column): row-first lanes for
            // 16-column tiles; otherwise columns across the warp
            const bool rows_first = (LOGJ == 4) && same_radix && !a.last;
            const int jj = rows_first ? (int)(threadIdx.x >> QAB) : (int)(threadIdx.x % J);
            const int pp = rows_first ? (int)(threadIdx.x & (QA - 1)) : (int)(threadIdx.x / J);  // pp < QA
            cpx<T> v[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) v[k] = s[swz<LOGJ>((pp + k * QA) * J + jj)];
            if constexpr (QA > 1) {
#pragma unroll
                for (int k = 1; k < RB; ++k) v[k] = mul(v[k], st[(k - 1) * QA + pp]);
            }
            SmallDFT<T, RB>::run(v);
            if (a.last) {
                // output index o of element k grows by QA Ns per k; mode m = o or o - M
                const int o0 = j0 + jj + (pp << logNs);
                const int step = QA << logNs;
                if (g < a.npk) {
                    cpx<T>* plus = out + (int64_t)(2 * g) * a.N;
                    cpx<T>* minus = plus + a.N;
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        const int o = o0 + k * step;
                        const int jp = o - a.sh;                    // mode +(sh + jp)
                        const int jm = ((M - o) & (M - 1)) - a.sh;  // mode -(sh + jm)
                        if ((unsigned)jp < (unsigned)a.N) plus[jp] = v[k];
                        if ((unsigned)jm < (unsigned)a.N) minus[jm] = v[k];
                    }
                } else {
                    cpx<T>* spec = out + (int64_t)(a.npk + g) * a.N;
                    const int lo_end = a.N - a.hN, hi_start = M - a.hN;
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        const int o = o0 + k * step;
                        if (o < lo_end) spec[o + a.hN] = v[k];
                        else if (o >= hi_start) spec[o - hi_start] = v[k];
                    }
                }
            } else if (same_radix) {
                cpx<T>* gout = out + (int64_t)g * M;
                const int LOGJn = a.logJn;
                const int logBlk = a.logRn + a.logJn;
#pragma unroll
                for (int k = 0; k < RB; ++k)
                    gout[rowcol_pos(pp + k * QA, j0 + jj, LOGJn, logBlk)] = v[k];
            } else {
#pragma unroll
                for (int k = 0; k < RB; ++k) s[swz<LOGJ>((pp + k * QA) * J + jj)] = v[k];
            }
        }
        if (!a.last && !same_radix) {
            __syncthreads();
            store_tile_blocked<LOGR, LOGJ, NT>(out + (int64_t)g * M, s,
                                               [](int e) { return swz<LOGJ>(e); }, j0, a,
                                               threadIdx.x);
        }
        __syncthreads();  // the tile buffer is reused by the next iteration
    }
}

template <int LOGR, int LOGJ>
__global__ void __launch_bounds__(P64_NT, 1) k_fft_pass64(const cpx<float>* __restrict__ in,
                                                       cpx<float>* __restrict__ out, PassArgs a,
                                                       const int64_t* __restrict__ Lg,
                                                       const cpx<float>* __restrict__ twlo,
                                                       const cpx<float>* __restrict__ twhi,
                                                       const cpx<float>* __restrict__ tw64,
                                                       int G) {
    regpass_body<64, LOGR, LOGJ>(in, out, a, Lg, twlo, twhi, tw64, G);
}

template <int LOGR, int LOGJ>
__global__ void __launch_bounds__(P32_NT, 1) k_fft_pass32(const cpx<float>* __restrict__ in,
                                                       cpx<float>* __restrict__ out, PassArgs a,
                                                       const int64_t* __restrict__ Lg,
                                                       const cpx<float>* __restrict__ twlo,
                                                       const cpx<float>* __restrict__ twhi,
                                                       const cpx<float>* __restrict__ tw32,
                                                       int G) {
    regpass_body<32, LOGR, LOGJ>(in, out, a, Lg, twlo, twhi, tw32, G);
}

// ------------------------------------------- radix-16 pass fed by bulk copies
// Float passes of radix R = 2^8..2^12 as the in-CTA Stockham stages of
// k_fft_pass (radix 16; the first stage takes LOGR mod 4 bits when that is
// nonzero), on tiles of 8192 elements with one persistent 512-thread CTA per
// SM.  A later pass reads each tile -- one contiguous 64 KB run of the blocked
// layout -- with bulk asynchronous copies (cp.async.bulk, completion counted
// on an mbarrier) into one of two input buffers, so the next tile streams in
// while the current one is transformed; the first pass reads the occupied
// rows of the spread grid with plain loads.  Stage 1 reads the input buffer
// and writes the padded work buffer, the middle stages work in place there,
// and the last stage's results go from registers straight to global memory
// where that fills whole 32-byte sectors (the last pass; a next pass of the
// same radix), otherwise through the work buffer.  Every mbarrier wait is
// bounded (wait_cycles SM cycles): a CTA that gives up sets FC2_ERR_TIMEOUT in
// *status, waits (again bounded) for each copy it still has in flight and
// returns.
constexpr int PT_NT = 512;
constexpr int PT_LOGE = 13;
constexpr long long PT_WAIT_CYCLES = 4000000000ll;  // about two seconds

FC2_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
FC2_D void mbar_init(uint64_t* m, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count)
                 : "memory");
}
FC2_D void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
FC2_D void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
FC2_D void mbar_expect_tx(uint64_t* m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}
FC2_D void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}
FC2_D bool mbar_try_wait(uint64_t* m, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity` of *m (at most `cycles`
// SM clock cycles).
FC2_D bool mbar_wait_bounded(uint64_t* m, unsigned parity, long long cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(m, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

// The 16-point transform of SmallDFT<T, 16> where only outputs 0..3 and
// 12..15 are wanted (a last pass that keeps the centred half of the modes):
// the same operations for those outputs, the other eight not formed.
template <typename T>
FC2_D void dft16_centred(cpx<T>* v) {
    cpx<T> e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    SmallDFT<T, 8>::run(e);
    SmallDFT<T, 8>::run(o);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = add(e[k], k == 0 ? o[0] : mul(o[k], root16<T>(k)));
#pragma unroll
    for (int k = 4; k < 8; ++k) v[k + 8] = sub(e[k], k == 4 ? mul_i(o[4]) : mul(o[k], root16<T>(k)));
}

// First-stage radix bits of the bulk-copy pass: radix 32 for 2^9 passes (two
// stages, 32 x 16: the first with half the threads, one butterfly of 32
// each), else as the other shared-memory stages (2^9 would otherwise take
// 2 x 16 x 16, one more pass through shared memory).
FC2_HD constexpr int bulk_stage1_bits(int LOGR) { return LOGR == 9 ? 5 : stage_bits(LOGR, 0); }

template <int LOGR>
constexpr size_t pass_tma_smem() {
    return (size_t)(2 * (1 << PT_LOGE) + phys((1 << PT_LOGE) - 1) + 1 + stage_tw_size(LOGR)) *
               sizeof(cpx<float>) +
           2 * sizeof(uint64_t);
}

template <int LOGR>
__global__ void __launch_bounds__(PT_NT, 1) k_fft_pass_tma(const cpx<float>* __restrict__ in,
                                                        cpx<float>* __restrict__ out, PassArgs a,
                                                        const int64_t* __restrict__ Lg,
                                                        const cpx<float>* __restrict__ twlo,
                                                        const cpx<float>* __restrict__ twhi,
                                                        const cpx<float>* __restrict__ twst,
                                                        int G, int* __restrict__ status,
                                                        long long wait_cycles, int drop_tile) {
    using T = float;
    constexpr int R = 1 << LOGR, LOGJ = PT_LOGE - LOGR, J = 1 << LOGJ, E = 1 << PT_LOGE;
    constexpr int NT = PT_NT;
    constexpr int NST = stage_tw_size(LOGR);
    constexpr int NWK = phys(E - 1) + 1;
    static_assert(LOGR >= 8 && LOGR <= 12, "radix 2^8..2^12");
    // stage 1 (radix Q1), middle stages of radix 16, last stage of radix 16
    constexpr int QB1 = bulk_stage1_bits(LOGR), Q1 = 1 << QB1;
    constexpr int NB1 = (R / Q1) * J;                      // stage-1 butterflies
    constexpr bool HALF1 = NB1 < NT;                       // threads tid >= NB1 idle in stage 1
    constexpr int PER1 = HALF1 ? 1 : NB1 / NT;
    constexpr int DL = LOGR - 4, NSL = 1 << DL;            // last stage: Ns = R / 16
    constexpr int TOFF_L = NST - 15 * NSL;                 // its twiddle table
    static_assert(HALF1 ? (NT % NB1 == 0 && Q1 == 32) : PER1 * NT == NB1,
                  "stage-1 butterflies must divide evenly");
    static_assert(Q1 <= 32, "stage-1 radix");
    static_assert(NSL * J == NT, "one last-stage butterfly per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* ib = reinterpret_cast<cpx<T>*>(smem_raw);  // [2][E] input buffers
    cpx<T>* wk = ib + 2 * E;                             // padded work buffer
    cpx<T>* st = wk + NWK;                               // stage twiddles
    uint64_t* mbar = reinterpret_cast<uint64_t*>(st + NST);
    const int tid = threadIdx.x;
    const int M = 1 << a.logM;
    const int S = M >> LOGR;
    const int tiles_x = S >> LOGJ;
    const int ntiles = tiles_x * G;
    const bool bulk = !a.first;
    for (int i = tid; i < NST; i += NT) st[i] = twst[i];
    if (bulk && tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0: copy tile t into input buffer b (four 16 KB pieces, one mbarrier)
    // (drop_tile >= 0, a fault-injection setting of the tests: that tile's
    // barrier is armed but its copy is never issued, so its wait runs out)
    auto issue = [&](int t, int b) {
        const int gtl = t / tiles_x, bt = t - gtl * tiles_x, gt = a.g0 + gtl;
        const cpx<T>* src = in + (int64_t)gt * M + (int64_t)bt * E;
        mbar_expect_tx(&mbar[b], (unsigned)(E * sizeof(cpx<T>)));
        if (t == drop_tile) return;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            bulk_g2s(ib + b * E + c * (E / 4), src + c * (E / 4),
                     (unsigned)(E / 4 * sizeof(cpx<T>)), &mbar[b]);
    };
    if (bulk && tid == 0) {
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
    }
    const int nsg_mask = (1 << a.logNs) - 1;
    const int lts = a.logM - a.logNs - LOGR;
    const int logNs = a.logNs;
    const bool same_radix = (logNs == 0 && a.logM - a.logRn == LOGR);
    int it = 0;
    // Inter-pass twiddles of stage 1 (later passes): butterfly b of thread tid
    // holds rows pp = (tid >> LOGJ) + b R/16 (+ k R/Q1) of column jj = tid mod J,
    // so w^{pp jm 2^lts} = t0 * w^{b (R/16) jm 2^lts}: t0 is one lookup per thread
    // and tile, the second factor (and the step w^{(R/Q1) jm 2^lts}) one lookup per
    // (column, b) and tile, kept in shared memory -- instead of two lookups per
    // butterfly.
    // (a radix-32 stage 1: per column the powers step^q, q = 1, 2, 3, 4, 8,
    // 12, 16 of step = w^{(R/Q1) jm 2^lts}, each a table lookup; element k's
    // factor is t0 step^(k mod 4) step^(4 ((k >> 2) mod 4)) step^(16 (k >> 4)),
    // three products of looked-up values)
    constexpr int TW1 = HALF1 ? 7 : PER1 + 1;
    __shared__ cpx<T> tw1[J * TW1];
    cpx<T> t0 = mk<T>(1.f, 0.f);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const int gl = tile / tiles_x;
        const int g = a.g0 + gl;
        const int bx = tile - gl * tiles_x;
        const int j0 = bx * J;
        if (bulk && logNs > 0) {
            // read by the previous tile's stage 1, which every thread has left (its
            // later stages passed barriers)
            for (int q = tid; q < J * TW1; q += NT) {
                const int cj = q / TW1, bb = q - cj * TW1;
                const int jm = (j0 + cj) & nsg_mask;
                int64_t e;
                if constexpr (HALF1) e = (int64_t)(R / Q1) * jm * (bb < 3 ? bb + 1 : 4 * (bb - 2));
                else e = (bb < PER1) ? (int64_t)bb * (R / 16) * jm : (int64_t)(R / Q1) * jm;
                tw1[q] = twiddle(twlo, twhi, a.tws, e << lts);
            }
            const int jm = (j0 + (tid & (J - 1))) & nsg_mask;
            t0 = twiddle(twlo, twhi, a.tws, (int64_t)(((tid >> LOGJ) * jm)) << lts);
        }
        if (bulk) {
            const bool ok = mbar_wait_bounded(&mbar[buf], (unsigned)((it >> 1) & 1), wait_cycles);
            if (!__syncthreads_and(ok)) {
                // give up: report, then wait (again bounded) for every copy this CTA
                // still has in flight -- the one just waited for and the next
                // tile's into the other buffer -- so that none is left writing
                // into the shared memory of a CTA that has exited
                if (tid == 0 && status) atomicExch(status, (int)FC2_ERR_TIMEOUT);
                mbar_wait_bounded(&mbar[buf], (unsigned)((it >> 1) & 1), wait_cycles);
                if (tile + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(&mbar[buf ^ 1], (unsigned)(((it + 1) >> 1) & 1), wait_cycles);
                return;
            }
        }
        // ---- stage 1: radix Q1 from the input (buffer or grid) into the work buffer
        {
            const cpx<T>* gin = in + (int64_t)g * M;
            const cpx<T>* src = ib + buf * E;
            int rows = R;
            if (!bulk) {
                rows = (int)((Lg[g] + S - 1) / S);
                if (rows > R) rows = R;
            }
#pragma unroll
            for (int b = 0; b < PER1; ++b) {
                const int bi = tid + b * NT;
                if (HALF1 && bi >= NB1) break;
                const int jj = bi & (J - 1), pp = bi >> LOGJ;
                cpx<T> v[Q1];
                if (!bulk) {
#pragma unroll
                    for (int k = 0; k < Q1; ++k) {
                        const int r = pp + k * (R / Q1);
                        v[k] = (r < rows) ? gin[j0 + jj + (int64_t)r * S] : mk<T>(0.f, 0.f);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < Q1; ++k) v[k] = src[(pp + k * (R / Q1)) * J + jj];
                    const int jm = (j0 + jj) & nsg_mask;
                    if constexpr (HALF1) {
                        if (logNs > 0 && jm != 0) {
                            // w_M^{(pp + k R/Q1) jm 2^lts} = t0 step^(k & 3) step^(k & 12) step^(k & 16)
                            const cpx<T>* sq = tw1 + jj * TW1;  // step^1, 2, 3, 4, 8, 12, 16
                            cpx<T> lo[4];
                            lo[0] = t0;
#pragma unroll
                            for (int q = 1; q < 4; ++q) lo[q] = mul(t0, sq[q - 1]);
#pragma unroll
                            for (int k = 0; k < Q1; ++k) {
                                cpx<T> w = lo[k & 3];
                                if (((k >> 2) & 3) != 0) w = mul(w, sq[2 + ((k >> 2) & 3)]);
                                if ((k >> 4) != 0) w = mul(w, sq[6]);
                                v[k] = mul(v[k], w);
                            }
                        }
                    } else if (logNs > 0 && jm != 0) {
                        // w_M^{(pp + k R/Q1) jm 2^lts} = base * step^k, step^k = lo[k & 3] hi[k >> 2]
                        const cpx<T> base = mul(t0, tw1[jj * TW1 + b]);
                        const cpx<T> st1 = tw1[jj * TW1 + PER1];
                        cpx<T> lo[4], hi[4];
                        lo[0] = mk<T>(1.f, 0.f);
                        lo[1] = st1;
                        lo[2] = mul(st1, st1);
                        lo[3] = mul(lo[2], st1);
                        hi[0] = mk<T>(1.f, 0.f);
                        hi[1] = mul(lo[2], lo[2]);
                        hi[2] = mul(hi[1], hi[1]);
                        hi[3] = mul(hi[2], hi[1]);
                        v[0] = mul(v[0], base);
#pragma unroll
                        for (int k = 1; k < Q1; ++k) {
                            cpx<T> w = base;
                            if ((k & 3) != 0) w = mul(w, lo[k & 3]);
                            if ((k >> 2) != 0) w = mul(w, hi[k >> 2]);
                            v[k] = mul(v[k], w);
                        }
                    }
                }
                SmallDFT<T, Q1>::run(v);
#pragma unroll
                for (int k = 0; k < Q1; ++k) wk[phys((pp * Q1 + k) * J + jj)] = v[k];
            }
        }
        __syncthreads();
        // the input buffer is free: ask for the tile after next
        if (bulk && tid == 0 && tile + 2 * (int)gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(tile + 2 * gridDim.x, buf);
        }
        // ---- middle stages, in place
        TwgArgs tg;
        tg.j0 = j0;
        tg.nsg_mask = nsg_mask;
        tg.lts = lts;
        tg.tws = a.tws;
        if constexpr (LOGR - QB1 > 4) {
            cta_stage<T, R, J, NT, 4, QB1, 0, false>(wk, st, tg, twlo, twhi);
            if constexpr (LOGR - QB1 > 8) {
                constexpr int TOFF3 = 15 * (1 << QB1);
                cta_stage<T, R, J, NT, 4, QB1 + 4, TOFF3, false>(wk, st, tg, twlo, twhi);
            }
        }
        // ---- last stage (radix 16, Ns = R / 16): registers
        const int jj = tid & (J - 1), pp = tid >> LOGJ;  // pp < NSL
        cpx<T> v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = wk[phys((pp + k * NSL) * J + jj)];
#pragma unroll
        for (int k = 1; k < 16; ++k) v[k] = mul(v[k], st[TOFF_L + (k - 1) * NSL + pp]);
        // a last pass keeping the centred half of the modes (N = M / 2) only
        // needs elements k < 4 (o < M / 4) and k >= 12 (o >= 3 M / 4): the
        // last stage's step is M / 16
        const bool centred = a.last && g >= a.npk && 2 * a.N == M && 2 * a.hN == a.N &&
                             16 * (NSL << logNs) == M;
        if (centred) dft16_centred(v);
        else SmallDFT<T, 16>::run(v);
        __syncthreads();  // every thread has read the work buffer
        // output row of element k: pp + k NSL
        if (a.last) {
            const int o0 = j0 + jj + (pp << logNs);
            const int step = NSL << logNs;
            if (centred) {
                cpx<T>* spec = out + (int64_t)(a.npk + g) * a.N;
#pragma unroll
                for (int k = 0; k < 4; ++k) spec[o0 + k * step + a.hN] = v[k];
#pragma unroll
                for (int k = 12; k < 16; ++k) spec[o0 + k * step - (M - a.hN)] = v[k];
            } else if (g < a.npk) {
                cpx<T>* plus = out + (int64_t)(2 * g) * a.N;
                cpx<T>* minus = plus + a.N;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int o = o0 + k * step;
                    const int jp = o - a.sh;
                    const int jmi = ((M - o) & (M - 1)) - a.sh;
                    if ((unsigned)jp < (unsigned)a.N) plus[jp] = v[k];
                    if ((unsigned)jmi < (unsigned)a.N) minus[jmi] = v[k];
                }
            } else {
                cpx<T>* spec = out + (int64_t)(a.npk + g) * a.N;
                const int lo_end = a.N - a.hN, hi_start = M - a.hN;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int o = o0 + k * step;
                    if (o < lo_end) spec[o + a.hN] = v[k];
                    else if (o >= hi_start) spec[o - hi_start] = v[k];
                }
            }
        } else if (same_radix) {
            cpx<T>* gout = out + (int64_t)g * M;
            const int LOGJn = a.logJn;
            const int logBlk = a.logRn + a.logJn;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                gout[rowcol_pos(pp + k * NSL, j0 + jj, LOGJn, logBlk)] = v[k];
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) wk[phys((pp + k * NSL) * J + jj)] = v[k];
            __syncthreads();
            store_tile_blocked<LOGR, LOGJ, NT>(out + (int64_t)g * M, wk,
                                               [](int e) { return phys(e); }, j0, a, tid);
            __syncthreads();
        }
    }
}

// Whether a float pass of radix 2^logR runs on the radix-32 register kernel.
static bool r32_pass(int family, int logR) {
    return (family == FFT_R32 && logR == 10) || (family == FFT_R32X && (logR == 9 || logR == 10));
}

cudaError_t init_twiddles(fc2_plan_s* p, cudaStream_t s) {
    int sh = (p->logM + 1) / 2;
    int64_t nlo = 1ll << sh, nhi = p->M >> sh;
    p->tw_shift = sh;
    int64_t nmax = std::max(nlo, nhi);
    unsigned blocks = (unsigned)((nmax + 255) / 256);
    bool assigned[16] = {false};
    for (int i = 0; i < 16; ++i) { p->twst_off[i] = 0; p->tw64_off[i] = 0; }
    int64_t off = 0;
    for (auto& ps : p->passes) {
        if (assigned[ps.logR]) continue;
        assigned[ps.logR] = true;
        p->twst_off[ps.logR] = off;
        int n = stage_tw_size(ps.logR);
        unsigned b2 = (unsigned)((n + 255) / 256);
        if (n > 0) {
            if (p->fp64) k_init_stage_tw<double><<<b2, 256, 0, s>>>((cpx<double>*)p->d_twst + off, ps.logR);
            else k_init_stage_tw<float><<<b2, 256, 0, s>>>((cpx<float>*)p->d_twst + off, ps.logR);
        }
        off += n + 16;
    }
    // tables of the two-stage register float kernels (stage-B twiddles; radix
    // 32 for the radix-32 family's 2^10 passes, else 64)
    for (auto& ps : p->passes) {
        if (p->fp64 || p->tw64_off[ps.logR] != 0) continue;
        if (!((ps.logR >= 10 && ps.logR <= 12 && p->fft_family == FFT_R64) ||
              r32_pass(p->fft_family, ps.logR)))
            continue;
        p->tw64_off[ps.logR] = off;
        const int lrb = r32_pass(p->fft_family, ps.logR) ? 5 : 6;
        const int n = ((1 << lrb) - 1) * (1 << (ps.logR - lrb));
        k_init_tw64<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((cpx<float>*)p->d_twst + off,
                                                                      ps.logR, lrb);
        off += n + 16;
    }
    if (p->fp64)
        k_init_tw<double><<<blocks, 256, 0, s>>>((cpx<double>*)p->d_twlo, nlo,
                                                 (cpx<double>*)p->d_twhi, nhi, p->logM, sh);
    else
        k_init_tw<float><<<blocks, 256, 0, s>>>((cpx<float>*)p->d_twlo, nlo,
                                                (cpx<float>*)p->d_twhi, nhi, p->logM, sh);
    return cudaGetLastError();
}

// -------------------------------------------------------------- pass plan
// fp32: tiles of 2^13 complex (64 KB), radix <= 2^12; fp64: 2^12 (64 KB), <= 2^11.
template <typename T> struct FftCfg;
template <> struct FftCfg<float> { static constexpr int LOGE = 13; static constexpr int NT = 512; static constexpr int MAXR = 12; };
template <> struct FftCfg<double> { static constexpr int LOGE = 12; static constexpr int NT = 256; static constexpr int MAXR = 11; };

void plan_fft_passes(fc2_plan_s* p) {
    const int maxr = p->fp64 ? FftCfg<double>::MAXR : FftCfg<float>::MAXR;
    p->passes.clear();
    const int logM = p->logM;
    if (logM <= maxr) {
        p->passes.push_back({logM, 1, 0});
        return;
    }
    const int P = (logM + maxr - 1) / maxr;
    std::vector<int> rs(P, logM / P);
    for (int i = 0; i < logM % P; ++i) rs[i] += 1;
    int64_t Ns = 1;
    for (int i = 0; i < P; ++i) {
        p->passes.push_back({rs[i], Ns, 0});
        Ns <<= rs[i];
    }
}

// The fixed planner's radices for a grid of 2^logM points (first pass first).
static std::vector<int> balanced_plan(int logM, bool fp64) {
    const int maxr = fp64 ? FftCfg<double>::MAXR : FftCfg<float>::MAXR;
    if (logM <= maxr) return {logM};
    const int P = (logM + maxr - 1) / maxr;
    std::vector<int> rs(P, logM / P);
    for (int i = 0; i < logM % P; ++i) rs[i] += 1;
    return rs;
}

// ------------------------------------------------------------ pass kernels
// Which kernel runs a pass of radix 2^logR (as run_radix chooses), its tile
// (2^loge elements, 2^logj columns) and threads.
enum PassKernel { PK_SINGLE = 0, PK_R16 = 1, PK_R64 = 2, PK_BULK = 3, PK_R32 = 4 };
struct PassShape {
    int kind, loge, logj, nt;
};
static PassShape pass_shape(int logM, bool fp64, int family, int logR) {
    if (logR == logM) {
        const int nt = (1 << logR) / 16 < 32 ? 32 : (1 << logR) / 16;
        return PassShape{PK_SINGLE, logR, 0, nt};
    }
    if (!fp64 && family == FFT_R64 && logR >= 10 && logR <= 12)
        return PassShape{PK_R64, P64_LOGE, P64_LOGE - logR, P64_NT};
    if (!fp64 && r32_pass(family, logR))
        return PassShape{PK_R32, P64_LOGE, P64_LOGE - logR, P32_NT};
    if (!fp64 && family != FFT_R16 && logR >= 8 && logR <= 12)
        return PassShape{PK_BULK, PT_LOGE, PT_LOGE - logR, PT_NT};
    const int loge = fp64 ? FftCfg<double>::LOGE : FftCfg<float>::LOGE;
    return PassShape{PK_R16, loge, loge - logR, fp64 ? FftCfg<double>::NT : FftCfg<float>::NT};
}

// What the pass kernels assume of a plan (radices rs, first pass first):
//  - the radices multiply to the grid length, each has a kernel (2^5..2^12 in
//    float, 2^5..2^11 in double; a single pass at least 2^9);
//  - every pass's tiles fit the grid (M / R columns hold at least one tile);
//  - a non-last pass stores its tile's R outputs per column as rows of the
//    next pass's tiles, Jn columns at a time: the next tile width Jn must not
//    exceed R (otherwise a tile's store walks past its R rows -- out of its
//    shared memory and out of the grid).
static bool fft_plan_valid(int logM, bool fp64, int family, const std::vector<int>& rs) {
    if (rs.empty()) return false;
    int sum = 0;
    for (int r : rs) sum += r;
    if (sum != logM) return false;
    const int maxr = fp64 ? FftCfg<double>::MAXR : FftCfg<float>::MAXR;
    if (rs.size() == 1) return logM >= 9 && logM <= maxr;
    for (size_t i = 0; i < rs.size(); ++i) {
        if (rs[i] < 5 || rs[i] > maxr) return false;
        const PassShape sh = pass_shape(logM, fp64, family, rs[i]);
        if (sh.logj < 0 || logM - rs[i] < sh.logj) return false;
        if (i + 1 < rs.size()) {
            const PassShape nx = pass_shape(logM, fp64, family, rs[i + 1]);
            if (nx.logj > rs[i]) return false;
        }
    }
    return true;
}

// ------------------------------------------------------ transform autotuner
// Candidate pass plans for a length-2^logM transform: the balanced split into
// the fewest passes (the fixed planner's choice), for two passes of unequal
// radix also the smaller radix first, and, when every radix stays at 2^8 or
// above, the balanced split into one pass more; float plans are
// tried with both kernel families.  Only pass shapes the fixed planner also
// produces for some length are searched: a wider search (unbalanced splits,
// small radices in three-pass plans) is not covered by the tests.  Each
// candidate runs on the plan's own buffers and the fastest is kept for the
// process, keyed by device, size, grid count and precision.
static void set_passes(fc2_plan_s* p, const std::vector<int>& rs) {
    p->passes.clear();
    int64_t Ns = 1;
    for (int r : rs) {
        p->passes.push_back({r, Ns, 0});
        Ns <<= r;
    }
}

static std::vector<int> balanced_split(int logM, int P) {
    std::vector<int> rs(P, logM / P);
    for (int i = 0; i < logM % P; ++i) rs[i] += 1;
    return rs;
}

static std::vector<std::vector<int>> fft_candidates(int logM, int maxr) {
    std::vector<std::vector<int>> out;
    if (logM <= maxr) {
        out.push_back({logM});
        return out;
    }
    const int P = (logM + maxr - 1) / maxr;
    const std::vector<int> bal = balanced_split(logM, P);
    out.push_back(bal);
    // the same two radices in the other order (the smaller first)
    if (P == 2 && bal[0] != bal[1] && bal[1] >= 8) out.push_back({bal[1], bal[0]});
    const std::vector<int> more = balanced_split(logM, P + 1);
    if (more.back() >= 8) out.push_back(more);
    return out;
}

struct TuneKey {
    int dev, logM, G, fp64, packed;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, logM, G, fp64, packed) < std::tie(o.dev, o.logM, o.G, o.fp64, o.packed);
    }
};
struct TuneChoice {
    std::vector<int> rs;
    int family, group;
};
static std::map<TuneKey, TuneChoice> g_tuned;
static std::mutex g_tune_mu;

cudaError_t autotune_fft(fc2_plan_s* p, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    const TuneKey key{dev, p->logM, p->G, p->fp64 ? 1 : 0, p->packed ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            set_passes(p, it->second.rs);
            p->fft_family = it->second.family;
            p->fft_group = it->second.group;
            return init_twiddles(p, s);
        }
    }
    const int maxr = p->fp64 ? FftCfg<double>::MAXR : FftCfg<float>::MAXR;
    const auto cands = fft_candidates(p->logM, maxr);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cudaGetLastError();
    }
    float best = 1e30f;
    std::vector<int> best_rs = cands.front();
    int best_fam = FFT_R64, best_grp = 0;
    cudaError_t e = cudaSuccess;
    const int fams_f32[5] = {FFT_BULK, FFT_R64, FFT_R32, FFT_R32X, FFT_R16};
    const int nfam = p->fp64 ? 1 : 5;
    std::vector<int> groups{0};
    if (p->G > 1) groups.push_back(1);
    if (p->G > 2) groups.push_back(2);
    for (const auto& rs : cands) {
        for (int fi = 0; fi < nfam && e == cudaSuccess; ++fi) {
            for (int grp : groups) {
                const int fam = p->fp64 ? FFT_R16 : fams_f32[fi];
                if (!fft_plan_valid(p->logM, p->fp64, fam, rs)) continue;
                set_passes(p, rs);
                p->fft_family = fam;
                p->fft_group = grp;
                if ((e = init_twiddles(p, s)) != cudaSuccess) break;
                if ((e = launch_fft(p, s)) != cudaSuccess) break;  // warm-up
                cudaEventRecord(e0, s);
                for (int it = 0; it < 3 && e == cudaSuccess; ++it) e = launch_fft(p, s);
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_rs = rs;
                    best_fam = fam;
                    best_grp = grp;
                }
            }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    set_passes(p, best_rs);
    p->fft_family = best_fam;
    p->fft_group = best_grp;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = TuneChoice{best_rs, best_fam, best_grp};
    }
    return init_twiddles(p, s);
}

// The (pass plan, family) pairs the batched path's autotuner times: the same
// plans as above with every float family (group 0: all grids pass by pass),
// each checked by the plan validator.
std::vector<FftChoice> fft_tune_candidates(int logM, bool fp64) {
    std::vector<FftChoice> out;
    const int maxr = fp64 ? FftCfg<double>::MAXR : FftCfg<float>::MAXR;
    const int fams[5] = {FFT_R64, FFT_R32, FFT_R32X, FFT_BULK, FFT_R16};
    for (const auto& rs : fft_candidates(logM, maxr))
        for (int fi = 0; fi < (fp64 ? 1 : 5); ++fi) {
            const int fam = fp64 ? FFT_R16 : fams[fi];
            if (fft_plan_valid(logM, fp64, fam, rs)) out.push_back(FftChoice{rs, fam});
        }
    return out;
}

bool fft_choice_valid(int logM, bool fp64, const FftChoice& c) {
    int sum = 0;
    for (int r : c.rs) {
        if (r < 1 || r > 12) return false;
        sum += r;
    }
    if (sum != logM || c.rs.empty()) return false;
    if (c.family != FFT_R64 && c.family != FFT_R32 && c.family != FFT_R32X && c.family != FFT_BULK &&
        c.family != FFT_R16)
        return false;
    if (fp64 && c.family != FFT_R16) return false;
    // only shapes the candidate list can hold
    bool listed = false;
    for (const auto& d : fft_tune_candidates(logM, fp64))
        if (d.rs == c.rs && d.family == c.family) listed = true;
    return listed;
}

cudaError_t set_fft_choice(fc2_plan_s* p, const FftChoice& c, cudaStream_t s) {
    if (!fft_choice_valid(p->logM, p->fp64, c)) return cudaErrorInvalidValue;
    set_passes(p, c.rs);
    p->fft_family = c.family;
    p->fft_group = 0;
    return init_twiddles(p, s);
}

// Tile width (columns) of the pass with radix 2^logR.
template <typename T>
static int logj_of(const fc2_plan_s* p, int logR) {
    return pass_shape(p->logM, sizeof(T) == 8, p->fft_family, logR).logj;
}


// ------------------------------------------------------ per-device launch state
// The SM count of the current device, and the dynamic shared-memory limit of a
// kernel raised once per (device, kernel): cudaFuncSetAttribute acts on the
// current device only, so a process that drives several devices needs it on
// each.  Both are guarded by one mutex (plans may run on several host threads).
static std::mutex g_launch_mu;
static std::map<std::pair<int, const void*>, size_t> g_smem_raised;  // (device, kernel) -> bytes
static std::map<int, int> g_sm_count;

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    return dev;
}

// SMs of the current device (queried once per device).
int device_sm_count() {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_sm_count.find(dev);
    if (it != g_sm_count.end()) return it->second;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        nsm = 152;
    }
    g_sm_count[dev] = nsm;
    return nsm;
}

static cudaError_t raise_smem_limit(const void* kern, size_t smem) {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_launch_mu);
    const auto key = std::make_pair(dev, kern);
    auto it = g_smem_raised.find(key);
    if (it != g_smem_raised.end() && it->second >= smem) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_smem_raised[key] = smem;
    return cudaSuccess;
}

template <typename T, int LOGR, int LOGJ, int NT>
static cudaError_t run_pass(fc2_plan_s* p, const void* in, void* out, const PassArgs& a,
                            cudaStream_t s) {
    constexpr int R = 1 << LOGR, J = 1 << LOGJ, E = R * J;
    const int64_t S = p->M >> LOGR;
    const size_t smem = (size_t)(phys(E - 1) + 1 + stage_tw_size(LOGR) + 1) * sizeof(cpx<T>);
    auto kern = k_fft_pass<T, LOGR, LOGJ, NT>;
    if (smem > 48 * 1024) {
        const cudaError_t e = raise_smem_limit((const void*)kern, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(S / J), (unsigned)a.ng);
    kern<<<grid, NT, smem, s>>>((const cpx<T>*)in, (cpx<T>*)out, a, p->d_L,
                                (const cpx<T>*)p->d_twlo, (const cpx<T>*)p->d_twhi,
                                (const cpx<T>*)p->d_twst + p->twst_off[LOGR]);
    return cudaGetLastError();
}

template <int RB, int LOGR>
static cudaError_t run_pass64(fc2_plan_s* p, const void* in, void* out, const PassArgs& a,
                              cudaStream_t s) {
    constexpr int LOGJ = P64_LOGE - LOGR, E = 1 << P64_LOGE;
    constexpr int NT = RB == 64 ? P64_NT : P32_NT;
    const int64_t S = p->M >> LOGR;
    const size_t smem = (size_t)(E + (RB - 1) * ((1 << LOGR) / RB)) * sizeof(cpx<float>);
    const void* kfn;
    if constexpr (RB == 64) kfn = (const void*)k_fft_pass64<LOGR, LOGJ>;
    else kfn = (const void*)k_fft_pass32<LOGR, LOGJ>;
    {
        const cudaError_t e = raise_smem_limit(kfn, smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntiles = (S >> LOGJ) * (int64_t)a.ng;
    const int nsm = device_sm_count();
    const unsigned blocks = (unsigned)std::min<int64_t>(ntiles, (int64_t)nsm);
    const cpx<float>* tw = (const cpx<float>*)p->d_twst + p->tw64_off[LOGR];
    if constexpr (RB == 64)
        k_fft_pass64<LOGR, LOGJ><<<blocks, NT, smem, s>>>((const cpx<float>*)in, (cpx<float>*)out, a,
                                                          p->d_L, (const cpx<float>*)p->d_twlo,
                                                          (const cpx<float>*)p->d_twhi, tw, a.ng);
    else
        k_fft_pass32<LOGR, LOGJ><<<blocks, NT, smem, s>>>((const cpx<float>*)in, (cpx<float>*)out, a,
                                                          p->d_L, (const cpx<float>*)p->d_twlo,
                                                          (const cpx<float>*)p->d_twhi, tw, a.ng);
    return cudaGetLastError();
}

template <int LOGR>
static cudaError_t run_pass_tma(fc2_plan_s* p, const void* in, void* out, const PassArgs& a,
                                cudaStream_t s) {
    constexpr int LOGJ = PT_LOGE - LOGR;
    const int64_t S = p->M >> LOGR;
    constexpr size_t smem = pass_tma_smem<LOGR>();
    auto kern = k_fft_pass_tma<LOGR>;
    {
        const cudaError_t e = raise_smem_limit((const void*)kern, smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntiles = (S >> LOGJ) * (int64_t)a.ng;
    const int nsm = device_sm_count();
    const unsigned blocks = (unsigned)std::min<int64_t>(ntiles, (int64_t)nsm);
    kern<<<blocks, PT_NT, smem, s>>>((const cpx<float>*)in, (cpx<float>*)out, a, p->d_L,
                                     (const cpx<float>*)p->d_twlo, (const cpx<float>*)p->d_twhi,
                                     (const cpx<float>*)p->d_twst + p->twst_off[LOGR], a.ng,
                                     p->d_status,
                                     p->dbg_wait_cycles > 0 ? p->dbg_wait_cycles : PT_WAIT_CYCLES,
                                     p->dbg_drop_tile);
    return cudaGetLastError();
}

template <typename T, int LOGR>
static cudaError_t run_radix(fc2_plan_s* p, const void* in, void* out, const PassArgs& a,
                             cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && LOGR >= 10 && LOGR <= 12) {
        if (LOGR != p->logM && p->fft_family == FFT_R64) return run_pass64<64, LOGR>(p, in, out, a, s);
    }
    if constexpr (sizeof(T) == 4 && (LOGR == 9 || LOGR == 10)) {
        if (LOGR != p->logM && r32_pass(p->fft_family, LOGR)) return run_pass64<32, LOGR>(p, in, out, a, s);
    }
    if constexpr (sizeof(T) == 4 && LOGR >= 8 && LOGR <= 12) {
        if (LOGR != p->logM && p->fft_family != FFT_R16) return run_pass_tma<LOGR>(p, in, out, a, s);
    }
    if (LOGR == p->logM) {
        constexpr int NT = (1 << LOGR) / 16 < 32 ? 32 : (1 << LOGR) / 16;
        if constexpr ((1 << LOGR) % (16 * NT) == 0 || (1 << LOGR) >= 16 * NT)
            return run_pass<T, LOGR, 0, NT>(p, in, out, a, s);
        return cudaErrorInvalidValue;
    }
    constexpr int LOGJ = FftCfg<T>::LOGE - LOGR;
    if constexpr (LOGJ >= 0) return run_pass<T, LOGR, LOGJ, FftCfg<T>::NT>(p, in, out, a, s);
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t fft_impl(fc2_plan_s* p, cudaStream_t s) {
    // Grids go through all passes a group at a time (p->fft_group grids per
    // group, 0 = all at once): with one or two grids per group the
    // intermediate between passes largely stays in L2.
    const int P = (int)p->passes.size();
    const int grp = (p->fft_group > 0) ? std::min(p->fft_group, p->G) : p->G;
    for (int g0 = 0; g0 < p->G; g0 += grp) {
        int src = 0;
        for (int i = 0; i < P; ++i) {
            const FftPass& ps = p->passes[i];
            PassArgs a;
            a.logM = p->logM;
            a.logNs = 0;
            while ((1ll << a.logNs) < ps.Ns) ++a.logNs;
            a.first = (i == 0);
            a.last = (i == P - 1);
            a.logRn = a.last ? 0 : p->passes[i + 1].logR;
            a.logJn = a.last ? 0 : logj_of<T>(p, p->passes[i + 1].logR);
            // the paper's gridding keeps every mode: mode m at spec[M/2 + m]
            a.N = p->paper ? (int)p->M : (int)p->N;
            a.hN = p->paper ? (int)(p->M / 2) : (int)(p->N / 2);
            a.tws = p->tw_shift;
            a.npk = p->paper ? 0 : p->npk;
            a.sh = (int)p->sh;
            a.g0 = g0;
            a.ng = std::min(grp, p->G - g0);
            const void* in = p->d_grid[src];
            void* out = a.last ? p->d_spec : p->d_grid[1 - src];
            cudaError_t e;
            switch (ps.logR) {
                case 8: e = run_radix<T, 8>(p, in, out, a, s); break;
                case 9: e = run_radix<T, 9>(p, in, out, a, s); break;
                case 10: e = run_radix<T, 10>(p, in, out, a, s); break;
                case 11: e = run_radix<T, 11>(p, in, out, a, s); break;
                case 12:
                    if constexpr (sizeof(T) == 4) { e = run_radix<T, 12>(p, in, out, a, s); break; }
                    return cudaErrorInvalidValue;
                case 7: e = run_radix<T, 7>(p, in, out, a, s); break;
                case 6: e = run_radix<T, 6>(p, in, out, a, s); break;
                case 5: e = run_radix<T, 5>(p, in, out, a, s); break;
                default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            src = 1 - src;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_fft(fc2_plan_s* p, cudaStream_t s) {
    std::vector<int> rs;
    for (const auto& ps : p->passes) rs.push_back(ps.logR);
    if (!fft_plan_valid(p->logM, p->fp64, p->fft_family, rs)) return cudaErrorInvalidValue;
    return p->fp64 ? fft_impl<double>(p, s) : fft_impl<float>(p, s);
}

// ------------------------------------------------ host replay of a plan's indices
// Every global and shared-memory index the pass kernels form for the plan's
// tiles, replayed on the host with the kernels' own index functions: loads of
// a pass's input, the stores toward the next pass on each kernel's store path
// (rows of a same-radix or two-pass plan, the one-stride fast path, the
// general blocked layout), the shared tile slots read by those stores, and the
// inter-pass twiddle exponents.  Returns 0 when all of them are in range for
// the tiles of every pass (all tiles up to 64 per pass, else the first and
// last 16 and 32 spread between them -- the index functions are monotone
// pieces in the tile number), else 100 * (pass + 1) + the failing check;
// info[0..3] = pass, check, tile, index.
static int replay_plan(int logM, bool fp64, int family, const std::vector<int>& rs,
                       int64_t* info) {
    const int64_t M = 1ll << logM;
    const int P = (int)rs.size();
    int logNs = 0;
    auto fail = [&](int pi, int check, int64_t tile, int64_t idx) {
        if (info) { info[0] = pi; info[1] = check; info[2] = tile; info[3] = idx; }
        return 100 * (pi + 1) + check;
    };
    for (int pi = 0; pi < P; ++pi) {
        const int LOGR = rs[pi];
        const int64_t R = 1ll << LOGR, S = M >> LOGR;
        const PassShape sh = pass_shape(logM, fp64, family, LOGR);
        const int LOGJ = sh.logj, J = 1 << LOGJ;
        const int64_t E = R << LOGJ;
        const bool first = pi == 0, last = pi == P - 1;
        const int logRn = last ? 0 : rs[pi + 1];
        const int LOGJn = last ? 0 : pass_shape(logM, fp64, family, logRn).logj;
        const int logBlk = logRn + LOGJn, logSn = logM - logRn;
        const int64_t tiles = S >> LOGJ;
        if (tiles < 1) return fail(pi, 1, 0, S);
        std::vector<int64_t> pick;
        if (tiles <= 64) {
            for (int64_t t = 0; t < tiles; ++t) pick.push_back(t);
        } else {
            for (int64_t t = 0; t < 16; ++t) pick.push_back(t);
            for (int64_t t = 16; t < tiles - 16; t += (tiles - 32) / 32 + 1) pick.push_back(t);
            for (int64_t t = tiles - 16; t < tiles; ++t) pick.push_back(t);
        }
        const bool same_radix = (logNs == 0 && logM - logRn == LOGR);
        for (int64_t bx : pick) {
            const int64_t j0 = bx << LOGJ;
            // loads: the first pass reads rows r < R of columns j0 .. j0 + J - 1;
            // later passes read one contiguous tile of the blocked layout
            const int64_t ld_max = first ? j0 + (J - 1) + (R - 1) * S : bx * E + E - 1;
            if (ld_max >= M) return fail(pi, 2, bx, ld_max);
            // inter-pass twiddle exponents (q < M keeps both table lookups in range)
            if (!first) {
                const int64_t jmax = (1ll << logNs) - 1;
                const int lts = logM - logNs - LOGR;
                int64_t qmax = 0;
                if (sh.kind == PK_R64 || sh.kind == PK_R32) {
                    const int RB = sh.kind == PK_R64 ? 64 : 32, QA = (1 << LOGR) / RB;
                    qmax = std::max<int64_t>(((RB - 1) * jmax) << lts, ((7 * RB) * jmax) << lts);
                    if (QA > 8)
                        qmax = std::max<int64_t>(qmax, ((8 * RB * ((QA / 8) - 1)) * jmax) << lts);
                } else if (sh.kind == PK_BULK && bulk_stage1_bits(LOGR) == 5) {
                    // radix-32 stage 1: t0 up to (R/16 - 1) jm, steps (R/32) jm x 1, 4, 16
                    qmax = std::max<int64_t>(((R / 16 - 1) * jmax) << lts, ((R / 32) * 16 * jmax) << lts);
                } else {
                    const int Q1 = 1 << stage_bits(LOGR, 0);
                    qmax = std::max<int64_t>(((R / Q1 - 1) * jmax) << lts, ((R / Q1) * jmax) << lts);
                }
                if (qmax >= M) return fail(pi, 3, bx, qmax);
            }
            if (last) continue;  // the last pass's mode stores are range-checked
            if ((sh.kind == PK_R64 || sh.kind == PK_R32 || sh.kind == PK_BULK) && same_radix) {
                for (int64_t kr = 0; kr < R; ++kr)
                    for (int jj = 0; jj < J; ++jj) {
                        const int64_t gi = rowcol_pos((int)kr, j0 + jj, LOGJn, logBlk);
                        if (gi < 0 || gi >= M) return fail(pi, 4, bx, gi);
                    }
                continue;
            }
            const bool fast = (sh.kind == PK_R64 || sh.kind == PK_R32 || sh.kind == PK_BULK) &&
                              logNs == 0 &&
                              LOGR <= logSn && LOGJn <= LOGR && (((1 << LOGJn) << LOGJ) <= sh.nt);
            if (fast) {
                const int Jn = 1 << LOGJn, NT = sh.nt;
                const int dkb = NT >> (LOGJn + LOGJ);
                for (int tid = 0; tid < NT; ++tid) {
                    const int kl = tid & (Jn - 1);
                    const int jj = (tid >> LOGJn) & (J - 1);
                    const int kb0 = tid >> (LOGJn + LOGJ);
                    const int64_t i0 = (j0 + jj) << LOGR;
                    const int64_t jb = i0 & ((1ll << logSn) - 1), rn = i0 >> logSn;
                    const int e0 = (kb0 << (LOGJn + LOGJ)) + (kl << LOGJ) + jj;
                    for (int64_t it = 0; it < E / NT; ++it) {
                        const int64_t gi = (((jb >> LOGJn) + kb0 + it * dkb) << logBlk) +
                                           (rn << LOGJn) + kl;
                        const int64_t se = e0 + it * NT;
                        if (gi < 0 || gi >= M) return fail(pi, 5, bx, gi);
                        if (se < 0 || se >= E) return fail(pi, 6, bx, se);
                    }
                }
                continue;
            }
            const bool rowcol = sh.kind == PK_R16 && same_radix;
            for (int64_t e = 0; e < E; ++e) {
                const TileElem te = tile_elem((int)e, LOGJn, LOGJ);
                if (te.k >= R || te.jj >= J) return fail(pi, 7, bx, (int64_t)te.k * J + te.jj);
                const int64_t gi = rowcol ? rowcol_pos(te.k, j0 + te.jj, LOGJn, logBlk)
                                          : blocked_pos(stockham_out(j0 + te.jj, te.k, logNs, LOGR),
                                                        logSn, LOGJn, logBlk);
                if (gi < 0 || gi >= M) return fail(pi, 8, bx, gi);
            }
        }
        logNs += LOGR;
    }
    return 0;
}

}  // namespace fc2

extern "C" int fc2_debug_fft_plan(int logM, int fp64, int* radices, int max_passes) {
    if (!radices || logM < 1 || logM > 40) return -1;
    const std::vector<int> rs = fc2::balanced_plan(logM, fp64 != 0);
    if ((int)rs.size() > max_passes) return -1;
    for (size_t i = 0; i < rs.size(); ++i) radices[i] = rs[i];
    return (int)rs.size();
}

extern "C" int fc2_debug_fft_candidates(int logM, int fp64, int* radices, int max_entries) {
    if (!radices || logM < 1 || logM > 40) return -1;
    const int maxr = fp64 ? fc2::FftCfg<double>::MAXR : fc2::FftCfg<float>::MAXR;
    int n = 0;
    for (const auto& rs : fc2::fft_candidates(logM, maxr)) {
        if (n + (int)rs.size() + 1 > max_entries) return -1;
        radices[n++] = (int)rs.size();
        for (int r : rs) radices[n++] = r;
    }
    return n;
}

extern "C" int fc2_debug_fft_plan_check(int logM, int fp64, int fft_kernel, const int* radices,
                                        int P, int validate, int64_t* info4) {
    if (!radices || P < 1 || P > 8 || logM < 1 || logM > 40) return -1;
    std::vector<int> rs(radices, radices + P);
    int sum = 0;
    for (int r : rs) {
        if (r < 1 || r > 16) return -1;
        sum += r;
    }
    if (sum != logM) return -1;
    const int fam = fc2::fft_family_of(fft_kernel);
    if (validate && !fc2::fft_plan_valid(logM, fp64 != 0, fam, rs)) return 1;
    return fc2::replay_plan(logM, fp64 != 0, fam, rs, info4);
}
