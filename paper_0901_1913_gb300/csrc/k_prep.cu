// k_prep.cu -- moments, time ordering, per-transform phase reduction and the
// deterministic spreading (gridding) of weights and weighted data.
//
// Paper: Sec. 3b (weighted mean subtraction, gridded p and q), Sec. 2 Eq. "eqPQ"
// (P and Q are Fourier transforms of the weighted data and of the weights).
// The paper grids by nearest-lower-cell binning; this library instead spreads
// each sample over w cells with a kernel of known Fourier transform and divides
// that transform out after the FFT, which is what makes the 1e-4 chi2_0
// agreement with direct sums reachable at practical grid sizes.
#include <cuda_runtime.h>

#include "fc2_common.cuh"
#include "fc2_internal.h"

namespace fc2 {

// ----------------------------------------------------------------- moments
// One CTA per curve.  Fixed per-thread striding and a fixed reduction tree
// make the result bitwise reproducible.
template <int NT>
__global__ void __launch_bounds__(NT) k_moments(const double* __restrict__ t,
                                                const double* __restrict__ x,
                                                const double* __restrict__ sg,
                                                const int64_t* __restrict__ offs,
                                                int64_t n_single, double* __restrict__ scal,
                                                int* __restrict__ status) {
    const int c = blockIdx.x;
    const int64_t a = offs ? offs[c] : 0;
    const int64_t b = offs ? offs[c + 1] : n_single;
    __shared__ double sh_s[NT], sh_c[NT], sh_s2[NT], sh_c2[NT], sh_mn[NT], sh_mx[NT], sh_q[NT];
    __shared__ int sh_bad, sh_unsorted;
    if (threadIdx.x == 0) { sh_bad = 0; sh_unsorted = 0; }
    __syncthreads();
    CompSum<double> W, WX;
    W.init(); WX.init();
    double mn = INFINITY, mx = -INFINITY, w2 = 0.0;
    int bad = 0, unsorted = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += NT) {
        double ti = t[i], xi = x[i], si = sg[i];
        if (!isfinite(ti) || !isfinite(xi) || !isfinite(si) || !(si > 0.0)) { bad = 1; continue; }
        double w = 1.0 / (si * si);
        if (!isfinite(w) || w == 0.0) { bad = 1; continue; }
        w2 += w * w;
        W.add(w);
        WX.add(__dmul_rn(w, xi));
        mn = fmin(mn, ti);
        mx = fmax(mx, ti);
        if (i + 1 < b && t[i + 1] < ti) unsorted = 1;
    }
    if (bad) atomicOr(&sh_bad, 1);
    if (unsorted) atomicOr(&sh_unsorted, 1);
    sh_s[threadIdx.x] = W.s; sh_c[threadIdx.x] = W.c;
    sh_s2[threadIdx.x] = WX.s; sh_c2[threadIdx.x] = WX.c;
    sh_mn[threadIdx.x] = mn; sh_mx[threadIdx.x] = mx;
    sh_q[threadIdx.x] = w2;
    __syncthreads();
    for (int st = NT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            CompSum<double> u; u.s = sh_s[threadIdx.x]; u.c = sh_c[threadIdx.x];
            u.add(sh_s[threadIdx.x + st]); u.c += sh_c[threadIdx.x + st];
            sh_s[threadIdx.x] = u.s; sh_c[threadIdx.x] = u.c;
            CompSum<double> v; v.s = sh_s2[threadIdx.x]; v.c = sh_c2[threadIdx.x];
            v.add(sh_s2[threadIdx.x + st]); v.c += sh_c2[threadIdx.x + st];
            sh_s2[threadIdx.x] = v.s; sh_c2[threadIdx.x] = v.c;
            sh_mn[threadIdx.x] = fmin(sh_mn[threadIdx.x], sh_mn[threadIdx.x + st]);
            sh_mx[threadIdx.x] = fmax(sh_mx[threadIdx.x], sh_mx[threadIdx.x + st]);
            sh_q[threadIdx.x] += sh_q[threadIdx.x + st];
        }
        __syncthreads();
    }
    const double W2 = sh_q[0];
    const double Wv = sh_s[0] + sh_c[0];
    const double xbar = (sh_s2[0] + sh_c2[0]) / Wv;
    const double T0 = sh_mn[0], Tmax = sh_mx[0];
    __syncthreads();
    CompSum<double> C0, S1;
    C0.init(); S1.init();
    double q2 = 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += NT) {
        double si = sg[i];
        double w = 1.0 / (si * si);
        double d = x[i] - xbar;
        C0.add(__dmul_rn(__dmul_rn(w, d), d));
        S1.add(__dmul_rn(w, d));
        q2 += (w * d) * (w * d);
    }
    __syncthreads();
    sh_s[threadIdx.x] = C0.s; sh_c[threadIdx.x] = C0.c;
    sh_s2[threadIdx.x] = S1.s; sh_c2[threadIdx.x] = S1.c;
    sh_q[threadIdx.x] = q2;
    __syncthreads();
    for (int st = NT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            CompSum<double> u; u.s = sh_s[threadIdx.x]; u.c = sh_c[threadIdx.x];
            u.add(sh_s[threadIdx.x + st]); u.c += sh_c[threadIdx.x + st];
            sh_s[threadIdx.x] = u.s; sh_c[threadIdx.x] = u.c;
            CompSum<double> v; v.s = sh_s2[threadIdx.x]; v.c = sh_c2[threadIdx.x];
            v.add(sh_s2[threadIdx.x + st]); v.c += sh_c2[threadIdx.x + st];
            sh_s2[threadIdx.x] = v.s; sh_c2[threadIdx.x] = v.c;
            sh_q[threadIdx.x] += sh_q[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = scal + (int64_t)c * SC_COUNT;
        const double chi0 = sh_s[0] + sh_c[0];
        const double rq = (Wv > 0.0) ? sqrt(W2) / Wv : 1.0;
        const double rp = (chi0 > 0.0) ? sqrt(sh_q[0] / (Wv * chi0)) : 0.0;
        o[SC_W] = Wv;
        o[SC_XBAR] = xbar;
        o[SC_CHI0] = sh_s[0] + sh_c[0];
        o[SC_S1] = sh_s2[0] + sh_c2[0];
        o[SC_T0] = T0;
        o[SC_TAUMAX] = Tmax - T0;
        o[SC_SORTED] = sh_unsorted ? 0.0 : 1.0;
        o[SC_RW] = fmax(rq, rp);
        if (sh_bad || b <= a) set_status(status, FC2_ERR_INVALID_ARG);
    }
}

// Multi-CTA variant for one long curve: fixed chunks per CTA, partials
// combined in chunk order by a single CTA (reproducible).
constexpr int MOM_NT = 256;
constexpr int MOM_CHUNK = 8192;

struct MomPart { double s[4], c[4]; double mn, mx; int bad, unsorted; };

__global__ void __launch_bounds__(MOM_NT) k_mom_partial(const double* __restrict__ t,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ sg, int64_t n,
                                                        int pass, const double* __restrict__ scal,
                                                        MomPart* __restrict__ part) {
    __shared__ double sh[MOM_NT][4][2];
    __shared__ double smn[MOM_NT], smx[MOM_NT];
    __shared__ int sbad, suns;
    if (threadIdx.x == 0) { sbad = 0; suns = 0; }
    __syncthreads();
    const int64_t a = (int64_t)blockIdx.x * MOM_CHUNK;
    const int64_t b = min(n, a + MOM_CHUNK);
    CompSum<double> A, B, C;
    A.init(); B.init(); C.init();
    double mn = INFINITY, mx = -INFINITY;
    int bad = 0, uns = 0;
    const double xbar = pass ? scal[SC_XBAR] : 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += MOM_NT) {
        double ti = t[i], xi = x[i], si = sg[i];
        if (pass == 0) {
            if (!isfinite(ti) || !isfinite(xi) || !isfinite(si) || !(si > 0.0)) { bad = 1; continue; }
            double w = 1.0 / (si * si);
            if (!isfinite(w) || w == 0.0) { bad = 1; continue; }
            A.add(w);
            B.add(__dmul_rn(w, xi));
            C.add(__dmul_rn(w, w));
            mn = fmin(mn, ti);
            mx = fmax(mx, ti);
            if (i + 1 < n && t[i + 1] < ti) uns = 1;
        } else {
            double w = 1.0 / (si * si);
            double d = xi - xbar;
            A.add(__dmul_rn(__dmul_rn(w, d), d));
            B.add(__dmul_rn(w, d));
            const double wd = __dmul_rn(w, d);
            C.add(__dmul_rn(wd, wd));
        }
    }
    if (bad) atomicOr(&sbad, 1);
    if (uns) atomicOr(&suns, 1);
    sh[threadIdx.x][0][0] = A.s; sh[threadIdx.x][0][1] = A.c;
    sh[threadIdx.x][1][0] = B.s; sh[threadIdx.x][1][1] = B.c;
    sh[threadIdx.x][2][0] = C.s; sh[threadIdx.x][2][1] = C.c;
    smn[threadIdx.x] = mn; smx[threadIdx.x] = mx;
    __syncthreads();
    for (int st = MOM_NT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            for (int q = 0; q < 3; ++q) {
                CompSum<double> u; u.s = sh[threadIdx.x][q][0]; u.c = sh[threadIdx.x][q][1];
                u.add(sh[threadIdx.x + st][q][0]); u.c += sh[threadIdx.x + st][q][1];
                sh[threadIdx.x][q][0] = u.s; sh[threadIdx.x][q][1] = u.c;
            }
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + st]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        MomPart pp;
        for (int q = 0; q < 4; ++q) { pp.s[q] = 0; pp.c[q] = 0; }
        pp.s[0] = sh[0][0][0]; pp.c[0] = sh[0][0][1];
        pp.s[1] = sh[0][1][0]; pp.c[1] = sh[0][1][1];
        pp.s[2] = sh[0][2][0]; pp.c[2] = sh[0][2][1];
        pp.mn = smn[0]; pp.mx = smx[0]; pp.bad = sbad; pp.unsorted = suns;
        part[blockIdx.x] = pp;
    }
}

__global__ void k_mom_final(const MomPart* __restrict__ part, int nblk, int pass,
                            double* __restrict__ scal, int* __restrict__ status) {
    if (threadIdx.x != 0) return;
    CompSum<double> A, B, C;
    A.init(); B.init(); C.init();
    double mn = INFINITY, mx = -INFINITY;
    int bad = 0, uns = 0;
    for (int k = 0; k < nblk; ++k) {
        A.add(part[k].s[0]); A.c += part[k].c[0];
        B.add(part[k].s[1]); B.c += part[k].c[1];
        C.add(part[k].s[2]); C.c += part[k].c[2];
        mn = fmin(mn, part[k].mn); mx = fmax(mx, part[k].mx);
        bad |= part[k].bad; uns |= part[k].unsorted;
    }
    if (pass == 0) {
        scal[SC_W] = A.val();
        scal[SC_XBAR] = B.val() / A.val();
        scal[SC_T0] = mn;
        scal[SC_TAUMAX] = mx - mn;
        scal[SC_SORTED] = uns ? 0.0 : 1.0;
        scal[SC_RW] = sqrt(C.val()) / A.val();
        if (bad) set_status(status, FC2_ERR_INVALID_ARG);
    } else {
        scal[SC_CHI0] = A.val();
        scal[SC_S1] = B.val();
        const double rp = (A.val() > 0.0) ? sqrt(C.val() / (scal[SC_W] * A.val())) : 0.0;
        scal[SC_RW] = fmax(scal[SC_RW], rp);
    }
}

size_t moments_scratch_bytes(int64_t n) {
    return (size_t)((n + MOM_CHUNK - 1) / MOM_CHUNK) * sizeof(MomPart) + 256;
}

cudaError_t launch_moments_long(const double* t, const double* x, const double* sigma, int64_t n,
                                double* scal, int* status, void* scratch, cudaStream_t s) {
    const int nblk = (int)((n + MOM_CHUNK - 1) / MOM_CHUNK);
    MomPart* part = (MomPart*)scratch;
    for (int pass = 0; pass < 2; ++pass) {
        k_mom_partial<<<nblk, MOM_NT, 0, s>>>(t, x, sigma, n, pass, scal, part);
        k_mom_final<<<1, 32, 0, s>>>(part, nblk, pass, scal, status);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------- polynomial detrending
// "Detrend the data with a polynomial fit" (Sec. 4): the weighted least-squares
// polynomial of degree D <= 3 in u = (t - t_c) / s (t_c, s the centre and
// half-width of the span, from the moments' T0 and max tau) is subtracted from
// x.  Per block: sums of w u^k (k <= 2D) and w x u^p (p <= D); one thread adds
// the block sums in block order, solves the (D+1)-square normal equations by
// Cholesky, and a last kernel writes x - poly(u).
constexpr int TR_NT = 256;
constexpr int TR_NV = 11;  // 2D + 1 + D + 1 at D = 3

__global__ void __launch_bounds__(TR_NT) k_trend_partial(const double* __restrict__ t,
                                                         const double* __restrict__ x,
                                                         const double* __restrict__ sigma,
                                                         int64_t n, const double* __restrict__ scal,
                                                         int D, double* __restrict__ part) {
    __shared__ double red[TR_NT / 32][TR_NV];
    const double tc = scal[SC_T0] + 0.5 * scal[SC_TAUMAX];
    const double is = scal[SC_TAUMAX] > 0.0 ? 2.0 / scal[SC_TAUMAX] : 1.0;
    double acc[TR_NV];
#pragma unroll
    for (int v = 0; v < TR_NV; ++v) acc[v] = 0.0;
    const int64_t i = (int64_t)blockIdx.x * TR_NT + threadIdx.x;
    if (i < n) {
        const double w = 1.0 / (sigma[i] * sigma[i]);
        const double u = (t[i] - tc) * is;
        double uk = 1.0;
        for (int k = 0; k <= 2 * D; ++k) {
            acc[k] = w * uk;
            if (k <= D) acc[2 * D + 1 + k] = w * x[i] * uk;
            uk *= u;
        }
    }
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < TR_NV; ++v) {
        double y = acc[v];
        for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
        if (lane == 0) red[wi][v] = y;
    }
    __syncthreads();
    if (threadIdx.x < TR_NV) {
        double y = 0.0;
        for (int q = 0; q < TR_NT / 32; ++q) y += red[q][threadIdx.x];
        part[(int64_t)blockIdx.x * TR_NV + threadIdx.x] = y;
    }
}

__global__ void k_trend_solve(const double* __restrict__ part, int nblk, int D,
                              double* __restrict__ coef, int* __restrict__ status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double sum[TR_NV];
    for (int v = 0; v < TR_NV; ++v) sum[v] = 0.0;
    for (int b = 0; b < nblk; ++b)
        for (int v = 0; v < TR_NV; ++v) sum[v] += part[(int64_t)b * TR_NV + v];
    const int m = D + 1;
    double L[4][4], z[4];
    for (int r = 0; r < m; ++r) {
        for (int c = 0; c <= r; ++c) {
            double v = sum[r + c];
            for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
            if (r == c) {
                if (!(v > 1e-14 * sum[2 * r])) {  // samples cannot fix this degree
                    if (status) atomicExch(status, (int)FC2_ERR_INVALID_ARG);
                    for (int q = 0; q < 4; ++q) coef[q] = 0.0;
                    return;
                }
                L[r][r] = sqrt(v);
            } else {
                L[r][c] = v / L[c][c];
            }
        }
    }
    for (int r = 0; r < m; ++r) {
        double v = sum[2 * D + 1 + r];
        for (int k = 0; k < r; ++k) v -= L[r][k] * z[k];
        z[r] = v / L[r][r];
    }
    for (int r = m - 1; r >= 0; --r) {
        double v = z[r];
        for (int k = r + 1; k < m; ++k) v -= L[k][r] * coef[k];
        coef[r] = v / L[r][r];
    }
    for (int q = m; q < 4; ++q) coef[q] = 0.0;
}

__global__ void k_trend_apply(const double* __restrict__ t, const double* __restrict__ x,
                              int64_t n, const double* __restrict__ scal,
                              const double* __restrict__ coef, int D, double* __restrict__ xo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double tc = scal[SC_T0] + 0.5 * scal[SC_TAUMAX];
    const double is = scal[SC_TAUMAX] > 0.0 ? 2.0 / scal[SC_TAUMAX] : 1.0;
    const double u = (t[i] - tc) * is;
    double v = coef[D];
    for (int k = D - 1; k >= 0; --k) v = fma(v, u, coef[k]);
    xo[i] = x[i] - v;
}

cudaError_t launch_trend_sums(const double* t, const double* x, const double* sigma, int64_t n,
                              int D, const double* scal, double* part, int* nblk, cudaStream_t s) {
    *nblk = (int)((n + TR_NT - 1) / TR_NT);
    k_trend_partial<<<*nblk, TR_NT, 0, s>>>(t, x, sigma, n, scal, D, part);
    return cudaGetLastError();
}

size_t trend_scratch_bytes(int64_t n) {
    return (size_t)((n + TR_NT - 1) / TR_NT) * TR_NV * sizeof(double) + 64;
}

cudaError_t launch_detrend(const double* t, const double* x, const double* sigma, int64_t n,
                           int D, const double* scal, int* status, void* scratch, double* xo,
                           cudaStream_t s) {
    const int nblk = (int)((n + TR_NT - 1) / TR_NT);
    double* part = (double*)scratch;
    double* coef = part + (size_t)nblk * TR_NV;
    k_trend_partial<<<nblk, TR_NT, 0, s>>>(t, x, sigma, n, scal, D, part);
    k_trend_solve<<<1, 32, 0, s>>>(part, nblk, D, coef, status);
    k_trend_apply<<<nblk, TR_NT, 0, s>>>(t, x, n, scal, coef, D, xo);
    return cudaGetLastError();
}

cudaError_t launch_moments(const double* t, const double* x, const double* sigma,
                           const int64_t* offs, int64_t C, int64_t n_single, double* scal,
                           int* status, cudaStream_t s) {
    k_moments<256><<<(unsigned)C, 256, 0, s>>>(t, x, sigma, offs, n_single, scal, status);
    return cudaGetLastError();
}

// --------------------------------------------------------------- radix sort
// Stable LSD radix sort of 64-bit keys with 32-bit payloads, 8-bit digits.
// Stability makes the permutation unique, so the ordering is deterministic.
static constexpr int RS_TILE = 2048;
static constexpr int RS_NT = 256;

__device__ __forceinline__ uint64_t order_key(double v) {
    uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_rs_init(const double* __restrict__ t, int64_t n, uint64_t* __restrict__ keys,
                          int32_t* __restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { keys[i] = order_key(t[i]); vals[i] = (int32_t)i; }
}

__global__ void __launch_bounds__(RS_NT) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                   int shift, uint32_t* __restrict__ hist,
                                                   int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int e = threadIdx.x; e < RS_TILE; e += RS_NT) {
        int64_t i = base + e;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of hist[256 * nblk] in place (digit-major), single CTA
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ hist, int64_t total) {
    __shared__ uint32_t carry;
    __shared__ uint32_t part[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < total; base += 1024) {
        int64_t i = base + threadIdx.x;
        uint32_t v = (i < total) ? hist[i] : 0u;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            uint32_t add = (threadIdx.x >= off) ? part[threadIdx.x - off] : 0u;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        uint32_t incl = part[threadIdx.x];
        if (i < total) hist[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// Stable scatter: warp w of the CTA owns a contiguous sub-range of the tile.
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                      const int32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout,
                                                      int32_t* __restrict__ vout, int64_t n,
                                                      int shift, const uint32_t* __restrict__ hist,
                                                      int nblk) {
    constexpr int NW = RS_NT / 32;
    constexpr int PER_W = RS_TILE / NW;
    __shared__ uint32_t cnt[NW][256];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < NW * 256; d += RS_NT) (&cnt[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)wp * PER_W;
    for (int e = 0; e < PER_W; e += 32) {
        int64_t i = base + e + lane;
        bool ok = i < n;
        uint32_t dg = ok ? (uint32_t)((kin[i] >> shift) & 255) : 256u + lane;
        unsigned same = __match_any_sync(0xffffffffu, dg);
        if (ok && lane == __ffs(same) - 1) cnt[wp][dg] += __popc(same);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the global offset
    {
        int d = threadIdx.x;  // RS_NT == 256 digits
        uint32_t run = hist[(int64_t)d * nblk + blockIdx.x];
        for (int q = 0; q < NW; ++q) {
            uint32_t v = cnt[q][d];
            cnt[q][d] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int e = 0; e < PER_W; e += 32) {
        int64_t i = base + e + lane;
        bool ok = i < n;
        uint64_t k = ok ? kin[i] : 0ull;
        uint32_t dg = ok ? (uint32_t)((k >> shift) & 255) : 256u + lane;
        unsigned same = __match_any_sync(0xffffffffu, dg);
        unsigned lower = same & ((1u << lane) - 1u);
        if (ok) {
            uint32_t pos = cnt[wp][dg] + __popc(lower);
            kout[pos] = k;
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (ok && lane == __ffs(same) - 1) cnt[wp][dg] += __popc(same);
        __syncwarp();
    }
}

size_t sort_scratch_bytes(int64_t n) {
    int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
    return (size_t)n * (2 * sizeof(uint64_t) + sizeof(int32_t)) + (size_t)nblk * 256 * 4 + 1024;
}

cudaError_t sort_by_time(const double* t, int64_t n, int32_t* perm, void* scratch,
                         size_t scratch_bytes, cudaStream_t s) {
    if (scratch_bytes < sort_scratch_bytes(n)) return cudaErrorInvalidValue;
    int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
    char* p = (char*)scratch;
    uint64_t* k0 = (uint64_t*)p; p += (size_t)n * 8;
    uint64_t* k1 = (uint64_t*)p; p += (size_t)n * 8;
    int32_t* v1 = (int32_t*)p; p += (size_t)n * 4;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    uint32_t* hist = (uint32_t*)p;
    int32_t* v0 = perm;
    k_rs_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, n, k0, v0);
    for (int pass = 0; pass < 8; ++pass) {
        int shift = pass * 8;
        k_rs_hist<<<(unsigned)nblk, RS_NT, 0, s>>>(k0, n, shift, hist, (int)nblk);
        k_rs_scan<<<1, 1024, 0, s>>>(hist, nblk * 256);
        k_rs_scatter<<<(unsigned)nblk, RS_NT, 0, s>>>(k0, v0, k1, v1, n, shift, hist, (int)nblk);
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        int32_t* tv = v0; v0 = v1; v1 = tv;
    }
    // 8 passes: result is back in (k0, v0) == original buffers -> perm holds it
    return cudaGetLastError();
}

__global__ void k_gather_sorted(const double* __restrict__ t, const double* __restrict__ x,
                                const double* __restrict__ sg, const int32_t* __restrict__ perm,
                                int64_t n, const double* __restrict__ scal,
                                double* __restrict__ tau, double* __restrict__ wq,
                                double* __restrict__ wp) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t i = perm ? perm[s] : s;
    double si = sg[i];
    double w = 1.0 / (si * si);
    tau[s] = __dsub_rn(t[i], scal[SC_T0]);
    wq[s] = w;
    wp[s] = __dmul_rn(w, __dsub_rn(x[i], scal[SC_XBAR]));
}

cudaError_t launch_gather_sorted(const double* t, const double* x, const double* sigma,
                                 const int32_t* perm, int64_t n, const double* scal,
                                 double* tau, double* wq, double* wp, cudaStream_t s) {
    k_gather_sorted<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, x, sigma, perm, n, scal, tau,
                                                                wq, wp);
    return cudaGetLastError();
}

// ------------------------------------------------------------ phase reduction
// Transform g evaluates sum_i c_i exp(+2 pi i k f_j tau_i) for j = 0..N-1 (Eq. "eqPQ"
// at the multiple k f_j).  Since k f_j = k f_min + j (k df), write
//   u_i = frac(k df tau_i)            (exact fold: e^{2 pi i j u} has period 1 in u)
//   theta_i = k f_min tau_i + hN u_i  (hN = floor(N/2); centres the modes m = j - hN)
// so the sum is a type-1 non-uniform DFT over modes m in [-hN, N - hN):
//   sum_i c_i e^{2 pi i theta_i} e^{2 pi i m u_i}.
// All products and differences use explicit round-to-nearest intrinsics so no
// contraction changes the reduced phase.
// Transforms g >= 3H (the trend fitted with the harmonics) carry the strengths
// w u^p e^{..} at multiple k: g = 3H + (p - 1) H + k - 1, u = (tau - tc) is.
template <typename T>
__global__ void k_phase(const double* __restrict__ tau, const double* __restrict__ wq,
                        const double* __restrict__ wp, int64_t n, int H, double f_min,
                        double df, int64_t N, int64_t M, int w, double tc, double is,
                        int32_t* __restrict__ key, T* __restrict__ dlt,
                        cpx<T>* __restrict__ cs) {
    const int g = blockIdx.y;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int k, kind, pw = 0;
    if (g < 2 * H) { k = g + 1; kind = 0; }
    else if (g < 3 * H) { k = g - 2 * H + 1; kind = 1; }
    else { pw = (g - 3 * H) / H + 1; k = (g - 3 * H) % H + 1; kind = 3; }
    const double ts = tau[s];
    const double c = __dmul_rn((double)k, df);
    const double p = __dmul_rn(c, ts);
    const double u = __dsub_rn(p, floor(p));
    const double X = __dmul_rn((double)M, u);             // exact (power of two)
    const double Xs = __dsub_rn(X, 0.5 * (double)w);      // exact
    const double fl = floor(Xs);
    const int32_t kk = (int32_t)fl + 1;
    const double de = __dsub_rn(Xs, fl);
    const double q1 = __dmul_rn(__dmul_rn((double)k, f_min), ts);
    const double q2 = __dmul_rn((double)(N / 2), u);
    const double th = __dadd_rn(__dsub_rn(q1, floor(q1)), __dsub_rn(q2, floor(q2)));
    double sn, cn;
    sincospi(2.0 * th, &sn, &cn);
    double amp = kind == 1 ? wp[s] : wq[s];
    if (kind == 3) {
        const double u = (ts - tc) * is;
        for (int q = 0; q < pw; ++q) amp *= u;
    }
    const int64_t o = (int64_t)g * n + s;
    key[o] = kk;
    dlt[o] = (T)de;
    cs[o] = mk<T>((T)(amp * cn), (T)(amp * sn));
}

// Mixed-precision phase reduction from the plan's exact fixed-point phases
// A_i = frac(f_min tau_i) 2^64 and B_i = frac(df tau_i) 2^64: for harmonic k,
// u_i 2^64 = k B_i and theta_i 2^64 = k A_i + hN k B_i, both exact modulo
// 2^64 in integer arithmetic, so no double instruction is needed.  The cell
// offset keeps 24 fraction bits (the spreading runs in float).
__global__ void k_phase_fx32(const uint64_t* __restrict__ A, const uint64_t* __restrict__ B,
                             const float* __restrict__ wq32, const float* __restrict__ wp32,
                             int64_t n, int H, int64_t N, int logM, int w, int npk, int w_p,
                             const double* __restrict__ tau, double tc, double is,
                             int32_t* __restrict__ key, float* __restrict__ dlt,
                             cpx<float>* __restrict__ cs) {
    const int g = blockIdx.y;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    // g indexes sample sets: Q_{g+1}, P_{g-2H+1} unpacked, then the trend
    // transforms (w u^p at multiple k, g = 3H + (p - 1) H + k - 1); packed
    // (npk > 0): set g is Q_{g+1}, carrying P_{g+1} as imaginary part when
    // g < H and otherwise placed in the real (even g - H) or imaginary part of
    // its grid
    int k, kind, pw = 0;
    if (g < 2 * H) { k = g + 1; kind = 0; }
    else if (g < 3 * H) { k = g - 2 * H + 1; kind = 1; }
    else { pw = (g - 3 * H) / H + 1; k = (g - 3 * H) % H + 1; kind = 3; }
    if (npk > 0) { kind = 2; w = w_p; }
    const uint64_t uk = (uint64_t)k * B[s];
    const int32_t cell = (int32_t)(uk >> (64 - logM));                 // floor(M u)
    const float fx = (float)(uint32_t)((uk << logM) >> 40) * 5.9604644775390625e-08f;  // 2^-24
    int32_t kk;
    float de;
    if ((w & 1) == 0) {
        kk = cell - w / 2 + 1;
        de = fx;
    } else if (fx >= 0.5f) {
        kk = cell - (w - 1) / 2 + 1;
        de = fx - 0.5f;
    } else {
        kk = cell - (w - 1) / 2;
        de = fx + 0.5f;
    }
    const int64_t o = (int64_t)g * n + s;
    key[o] = kk;
    dlt[o] = de;
    if (kind == 2) {
        const float q = wq32[s];
        cs[o] = (g < H) ? mk<float>(q, wp32[s]) : (((g - H) & 1) ? mk<float>(0.f, q)
                                                                  : mk<float>(q, 0.f));
        return;
    }
    const uint64_t th = (uint64_t)k * A[s] + (uint64_t)(N / 2) * uk;
    float sn, cn;
    sincospif((float)(int32_t)(th >> 32) * 4.656612873077393e-10f, &sn, &cn);  // 2^-31
    float amp = kind == 1 ? wp32[s] : wq32[s];
    if (kind == 3) {
        const float u = (float)((tau[s] - tc) * is);
        for (int q = 0; q < pw; ++q) amp *= u;
    }
    cs[o] = mk<float>(amp * cn, amp * sn);
}

// Keys of a wrapping transform are sorted with their payload by a stable
// radix sort on the key (ties keep time order).
__global__ void k_key_init(const int32_t* __restrict__ key, int64_t n, int32_t off,
                           uint64_t* __restrict__ k64, int32_t* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { k64[i] = (uint64_t)(uint32_t)(key[i] + off); v[i] = (int32_t)i; }
}

template <typename T>
__global__ void k_key_apply(const int32_t* __restrict__ perm, int64_t n,
                            const int32_t* __restrict__ key_in, const T* __restrict__ d_in,
                            const cpx<T>* __restrict__ c_in, int32_t* __restrict__ key_out,
                            T* __restrict__ d_out, cpx<T>* __restrict__ c_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = perm[i];
    key_out[i] = key_in[s];
    d_out[i] = d_in[s];
    c_out[i] = c_in[s];
}

template <typename T>
static cudaError_t sort_keys_of(fc2_plan_s* p, int g, cudaStream_t s) {
    // Scratch: grids are free at this point of the pipeline.
    const bool per_slot = !p->h_slot_n.empty();
    const int64_t n = per_slot ? p->h_slot_n[g] : p->n;
    const int64_t so = per_slot ? p->h_slot_soff[g] : (int64_t)g * p->n;
    int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
    char* base = (char*)p->d_grid[1];
    uint64_t* k0 = (uint64_t*)base;
    uint64_t* k1 = k0 + n;
    int32_t* v0 = (int32_t*)(k1 + n);
    int32_t* v1 = v0 + n;
    int32_t* key2 = v1 + n;
    T* d2 = (T*)(((uintptr_t)(key2 + n) + 255) & ~(uintptr_t)255);
    cpx<T>* c2 = (cpx<T>*)(((uintptr_t)(d2 + n) + 255) & ~(uintptr_t)255);
    uint32_t* hist = (uint32_t*)(((uintptr_t)(c2 + n) + 255) & ~(uintptr_t)255);
    int32_t* key = p->d_key + so;
    T* dl = (T*)p->d_dlt + so;
    cpx<T>* cs = (cpx<T>*)p->d_cs + so;
    const int wmax = std::max(p->w, p->w_p);
    const int32_t off = wmax;  // keys >= 1 - w/2 -> shifted keys are positive
    k_key_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(key, n, off, k0, v0);
    int bits = 0;
    while ((1ll << bits) < p->M + 2 * wmax + 2) ++bits;
    int npass = (bits + 7) / 8;
    for (int pass = 0; pass < npass; ++pass) {
        k_rs_hist<<<(unsigned)nblk, RS_NT, 0, s>>>(k0, n, pass * 8, hist, (int)nblk);
        k_rs_scan<<<1, 1024, 0, s>>>(hist, nblk * 256);
        k_rs_scatter<<<(unsigned)nblk, RS_NT, 0, s>>>(k0, v0, k1, v1, n, pass * 8, hist,
                                                       (int)nblk);
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        int32_t* tv = v0; v0 = v1; v1 = tv;
    }
    k_key_apply<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v0, n, key, dl, cs, key2, d2, c2);
    cudaMemcpyAsync(key, key2, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(dl, d2, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(cs, c2, (size_t)n * sizeof(cpx<T>), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t phase_impl(fc2_plan_s* p, cudaStream_t s) {
    const int nsrc = p->nsrc ? p->nsrc : p->G;
    dim3 grid((unsigned)((p->n + 255) / 256), (unsigned)nsrc);
    if constexpr (sizeof(T) == 4)
        k_phase_fx32<<<grid, 256, 0, s>>>(p->d_phA, p->d_phB, p->d_wq32, p->d_wp32, p->n, p->H,
                                          p->N, p->logM, p->w, p->npk, p->w_p, p->d_tau,
                                          p->jt_tc, p->jt_is, p->d_key, (float*)p->d_dlt,
                                          (cpx<float>*)p->d_cs);
    else
        k_phase<T><<<grid, 256, 0, s>>>(p->d_tau, p->d_wq, p->d_wp, p->n, p->H, p->f_min, p->df,
                                        p->N, p->M, p->w, p->jt_tc, p->jt_is, p->d_key,
                                        (T*)p->d_dlt, (cpx<T>*)p->d_cs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int g = 0; g < nsrc; ++g)
        if (p->geom[g].wraps) {
            e = sort_keys_of<T>(p, g, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t sort_wrapping_keys(fc2_plan_s* p, cudaStream_t s) {
    for (int g = 0; g < (int)p->geom.size(); ++g)
        if (p->geom[g].wraps) {
            cudaError_t e = p->fp64 ? sort_keys_of<double>(p, g, s) : sort_keys_of<float>(p, g, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t launch_phase(fc2_plan_s* p, cudaStream_t s) {
    return p->fp64 ? phase_impl<double>(p, s) : phase_impl<float>(p, s);
}

// ----------------------------------------------------------------- spreading
// Gather formulation: CTA (g, tile) computes cells [a, a + TILE) of grid g as
//   G[l] = sum over samples s with key_s <= l < key_s + w (mod M) of cs_s phi(l - X_s),
// summing each cell's contributions in the samples' sorted order, so the grid
// is bitwise reproducible (no floating-point atomics).
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double re, im;
    FC2_D void init() { re = 0; im = 0; }
    FC2_D void add(double a, double b) { re += a; im += b; }
    FC2_D cpx<double> val() const { return mk(re, im); }
};
template <>
struct Acc<float> {  // compensated (two-sum) accumulation in the mixed path
    CompSum<float> re, im;
    FC2_D void init() { re.init(); im.init(); }
    FC2_D void add(float a, float b) { re.add(a); im.add(b); }
    FC2_D cpx<float> val() const { return mk(re.val(), im.val()); }
};

__device__ __forceinline__ int64_t lower_bound_key(const int32_t* __restrict__ k, int64_t n,
                                                   int64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)k[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Key ranges of every (grid, tile), found before spreading by one thread per
// (grid, tile, bound): for each sample set si of the grid (one, or two for a
// packed grid) and each shift of the keys by -M, 0, +M, the lower bounds in
// the set's sorted keys of a - w + 1 and a + TILE (a = tile start), i.e. the
// samples whose windows meet the tile.  rng[((g ntile + tile) 2 + si) 6 + q]:
// q = 0..5 the bounds for the shifts -M (lo, hi), 0, +M.
// The occupied tiles of every grid as one list: tfirst[g] = first list entry
// of grid g (its tiles cover [0, L_g)), tfirst[G] = the entry count (one CTA,
// a block scan over the grids); then tgrid[t] = the grid of entry t
// (k_tile_fill, a search of tfirst per entry).
template <int TILE>
__global__ void __launch_bounds__(1024) k_tile_list(const int64_t* __restrict__ Lg, int G,
                                                    int64_t* __restrict__ tfirst) {
    __shared__ int64_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
    const int per = (G + 1023) / 1024;
    const int g0 = tid * per, g1 = min(G, g0 + per);
    int64_t v = 0;
    for (int g = g0; g < g1; ++g) v += (Lg[g] + TILE - 1) / TILE;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wi] = incl;
    __syncthreads();
    int64_t base = incl - v;
    for (int k = 0; k < wi; ++k) base += wsum[k];
    for (int g = g0; g < g1; ++g) {
        tfirst[g] = base;
        base += (Lg[g] + TILE - 1) / TILE;
    }
    if (g0 < G && g1 == G) tfirst[G] = base;
}

__global__ void k_tile_fill(const int64_t* __restrict__ tfirst, int G, int64_t ntile,
                            int32_t* __restrict__ tgrid) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntile) return;
    int lo = 0, hi = G;  // the last g with tfirst[g] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tfirst[mid] <= t) lo = mid; else hi = mid;
    }
    tgrid[t] = lo;
}

template <int TILE>
__global__ void __launch_bounds__(128) k_tile_ranges(const int32_t* __restrict__ key,
                                                     int64_t n_all, int64_t M, int w, int npk,
                                                     int pH, int w_p,
                                                     const int64_t* __restrict__ tfirst,
                                                     const int32_t* __restrict__ tgrid,
                                                     const int64_t* __restrict__ slot_soff,
                                                     const int64_t* __restrict__ slot_n,
                                                     int64_t ntile, int64_t* __restrict__ rng) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t et = idx / 12;  // list entry
    const int sq = (int)(idx - et * 12), si = sq / 6, q = sq - si * 6;
    if (et >= ntile) return;
    const int g = tgrid[et];
    const int64_t tile = et - tfirst[g];
    const int64_t a = tile * TILE;
    int t0 = g, nset = 1;
    if (npk > 0) {
        w = w_p;
        if (g >= pH) {
            t0 = pH + 2 * (g - pH);
            nset = (t0 + 1 < 2 * pH) ? 2 : 1;
        }
    }
    if (si >= nset) return;
    const int t = t0 + si;
    const int64_t so = slot_soff ? slot_soff[t] : (int64_t)t * n_all;
    const int64_t n = slot_n ? slot_n[t] : n_all;
    const int64_t shv = (q >> 1) == 0 ? M : ((q >> 1) == 1 ? 0 : -M);
    const int64_t v = (q & 1) ? a + TILE + shv : a - w + 1 + shv;
    rng[et * 12 + sq] = lower_bound_key(key + so, n, v);
}

template <typename T, int TILE, int NT, int CAP>
__global__ void __launch_bounds__(NT) k_spread(const int32_t* __restrict__ key,
                                               const T* __restrict__ dlt,
                                               const cpx<T>* __restrict__ cs, int64_t n_all,
                                               int64_t M, int w, T beta, int npk, int pH,
                                               int w_p, T beta_p,
                                               const int64_t* __restrict__ tfirst,
                                               const int32_t* __restrict__ tgrid,
                                               cpx<T>* __restrict__ grid, int64_t gstride,
                                               const int64_t* __restrict__ slot_soff,
                                               const int64_t* __restrict__ slot_n,
                                               const int64_t* __restrict__ rngtab,
                                               const int32_t* __restrict__ tlist,
                                               const int32_t* __restrict__ tlist_count) {
    constexpr int PER = TILE / NT;
    // cumulative key counts of the staged samples: cum[i] = samples with
    // tile-relative key <= i - w (keys lie in [-w + 1, TILE)), so the samples of
    // cell l (l - w + 1 <= key <= l, contiguous in sorted order) are
    // [cum[l], cum[l + w]); PCUM consecutive entries per thread for the scan
    constexpr int PCUM = (TILE + 32 + NT - 1) / NT;
    __shared__ int32_t sk[CAP];
    __shared__ T sd[CAP];
    __shared__ cpx<T> sc[CAP];
    __shared__ int32_t cum[PCUM * NT];
    __shared__ int32_t wtot[NT / 32];
    // every occupied tile (one per CTA), or the tiles listed by the single-batch
    // kernel (CTAs walk the list)
    const int64_t nlist = tlist ? (int64_t)*tlist_count : 1;
    for (int64_t li = tlist ? blockIdx.x : 0; li < nlist; li += gridDim.x) {
    const int64_t et = tlist ? (int64_t)tlist[li] : (int64_t)blockIdx.x;
    const int g = tgrid[et];
    const int64_t a = (et - tfirst[g]) * TILE;
    const int64_t* rt = rngtab + et * 12;
    // sample sets of grid g: one, or (packed grids g >= H) two
    int t0 = g, nset = 1;
    if (npk > 0) {
        w = w_p;
        beta = beta_p;
        if (g >= pH) {
            t0 = pH + 2 * (g - pH);
            nset = (t0 + 1 < 2 * pH) ? 2 : 1;
        }
    }
    const T ihw = (T)2 / (T)w;
    const T hw = (T)0.5 * (T)w;
    Acc<T> acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q].init();
    for (int si = 0; si < nset; ++si) {
        const int t = t0 + si;
        // samples of set t: from t n_all or, for a batch, from the slot's offset
        const int64_t so = slot_soff ? slot_soff[t] : (int64_t)t * n_all;
        const int32_t* kg = key + so;
        const T* dg = dlt + so;
        const cpx<T>* cg = cs + so;
        int64_t rng[6];  // key ranges of the shifts -M, 0, +M (k_tile_ranges)
#pragma unroll
        for (int q = 0; q < 6; ++q) rng[q] = rt[si * 6 + q];
        const int64_t c0 = rng[1] - rng[0], c1 = rng[3] - rng[2], c2 = rng[5] - rng[4];
        const int64_t total = c0 + c1 + c2;
        for (int64_t cb = 0; cb < total; cb += CAP) {
            const int cnt = (int)min((int64_t)CAP, total - cb);
#pragma unroll
            for (int i = 0; i < PCUM; ++i) cum[threadIdx.x * PCUM + i] = 0;
            for (int e = threadIdx.x; e < cnt; e += NT) {
                int64_t v = cb + e;
                int64_t src;
                int64_t shv;
                if (v < c0) { src = rng[0] + v; shv = -M; }
                else if (v < c0 + c1) { src = rng[2] + (v - c0); shv = 0; }
                else { src = rng[4] + (v - c0 - c1); shv = M; }
                sk[e] = (int32_t)((int64_t)kg[src] + shv - a);  // tile-relative key
                sd[e] = dg[src];
                sc[e] = cg[src];
            }
            __syncthreads();
            // key histogram (exact counts), then an inclusive block scan
            for (int e = threadIdx.x; e < cnt; e += NT) atomicAdd(&cum[sk[e] + w], 1);
            __syncthreads();
            {
                int32_t run[PCUM];
                int32_t t = 0;
#pragma unroll
                for (int i = 0; i < PCUM; ++i) {
                    t += cum[threadIdx.x * PCUM + i];
                    run[i] = t;
                }
                const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
                int32_t incl = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) wtot[wi] = incl;
                __syncthreads();
                int32_t before = incl - t;
                for (int k = 0; k < wi; ++k) before += wtot[k];
#pragma unroll
                for (int i = 0; i < PCUM; ++i) cum[threadIdx.x * PCUM + i] = before + run[i];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int l = threadIdx.x + q * NT;  // tile-relative cell
                // samples with l - w + 1 <= key <= l, in sorted order
                const int e1 = cum[l + w];
                for (int e = cum[l]; e < e1; ++e) {
                    T z = (T)(l - sk[e]) + (T)1 - sd[e] - hw;
                    T ph = es_kernel<T>(z, ihw, beta);
                    acc[q].add(sc[e].x * ph, sc[e].y * ph);
                }
            }
            __syncthreads();
        }
    }
    cpx<T>* gg = grid + (int64_t)g * gstride + a;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int l = threadIdx.x + q * NT;
        gg[l] = acc[q].val();
    }
    }
}

// The same sums for a tile of one sample set whose samples fit one staging
// batch (all tiles of an unpacked grid but the densest): each cell is summed
// and stored in turn, so a thread holds one running sum instead of one per
// cell, and with fewer registers and a smaller staging buffer more CTAs fit
// an SM (the kernel waits mostly on its loads and barriers).  Other tiles are
// appended to `tlist` for the general kernel.  A cell's samples and their
// order, and the arithmetic, are the general kernel's.
template <typename T, int TILE, int NT, int CAP>
__global__ void __launch_bounds__(NT, 2048 / NT) k_spread1(const int32_t* __restrict__ key,
                                                           const T* __restrict__ dlt,
                                                           const cpx<T>* __restrict__ cs,
                                                           int64_t n_all, int64_t M, int w, T beta,
                                                           const int64_t* __restrict__ tfirst,
                                                           const int32_t* __restrict__ tgrid,
                                                           cpx<T>* __restrict__ grid,
                                                           int64_t gstride,
                                                           const int64_t* __restrict__ slot_soff,
                                                           const int64_t* __restrict__ rngtab,
                                                           int32_t* __restrict__ tlist,
                                                           int32_t* __restrict__ tlist_count) {
    constexpr int PER = TILE / NT;
    constexpr int PCUM = (TILE + 32 + NT - 1) / NT;
    __shared__ int32_t sk[CAP];
    __shared__ T sd[CAP];
    __shared__ cpx<T> sc[CAP];
    __shared__ int32_t cum[PCUM * NT];
    __shared__ int32_t wtot[NT / 32];
    const int64_t et = blockIdx.x;
    const int g = tgrid[et];
    const int64_t a = (et - tfirst[g]) * TILE;
    const int64_t* rt = rngtab + et * 12;
    int64_t rng[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) rng[q] = rt[q];
    const int64_t c0 = rng[1] - rng[0], c1 = rng[3] - rng[2], c2 = rng[5] - rng[4];
    const int64_t total = c0 + c1 + c2;
    if (total > CAP) {
        if (threadIdx.x == 0) tlist[atomicAdd(tlist_count, 1)] = (int32_t)et;
        return;
    }
    const int cnt = (int)total;
    const int64_t so = slot_soff ? slot_soff[g] : (int64_t)g * n_all;
    const int32_t* kg = key + so;
    const T* dg = dlt + so;
    const cpx<T>* cg = cs + so;
#pragma unroll
    for (int i = 0; i < PCUM; ++i) cum[threadIdx.x * PCUM + i] = 0;
    for (int e = threadIdx.x; e < cnt; e += NT) {
        int64_t src, shv;
        if (e < c0) { src = rng[0] + e; shv = -M; }
        else if (e < c0 + c1) { src = rng[2] + (e - c0); shv = 0; }
        else { src = rng[4] + (e - c0 - c1); shv = M; }
        sk[e] = (int32_t)((int64_t)kg[src] + shv - a);
        sd[e] = dg[src];
        sc[e] = cg[src];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += NT) atomicAdd(&cum[sk[e] + w], 1);
    __syncthreads();
    {
        int32_t run[PCUM];
        int32_t t = 0;
#pragma unroll
        for (int i = 0; i < PCUM; ++i) {
            t += cum[threadIdx.x * PCUM + i];
            run[i] = t;
        }
        const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
        int32_t incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wtot[wi] = incl;
        __syncthreads();
        int32_t before = incl - t;
        for (int k = 0; k < wi; ++k) before += wtot[k];
#pragma unroll
        for (int i = 0; i < PCUM; ++i) cum[threadIdx.x * PCUM + i] = before + run[i];
    }
    __syncthreads();
    const T ihw = (T)2 / (T)w;
    const T hw = (T)0.5 * (T)w;
    cpx<T>* gg = grid + (int64_t)g * gstride + a;
    for (int q = 0; q < PER; ++q) {
        const int l = threadIdx.x + q * NT;
        Acc<T> acc;
        acc.init();
        const int e1 = cum[l + w];
        for (int e = cum[l]; e < e1; ++e) {
            T z = (T)(l - sk[e]) + (T)1 - sd[e] - hw;
            T ph = es_kernel<T>(z, ihw, beta);
            acc.add(sc[e].x * ph, sc[e].y * ph);
        }
        gg[l] = acc.val();
    }
}

// Tests may send every tile to the general kernel (a comparison of the two).
static int g_spread_general_only = 0;

template <typename T, int TILE, int NT, int CAP, int CAP1>
static cudaError_t spread_tiles(fc2_plan_s* p, cudaStream_t s) {
    // only the occupied tiles are launched: the list of (grid, tile) entries
    // covering [0, L_g) of every grid, built on the device from the same L the
    // host counts here
    int64_t tiles = 0;
    if ((int)p->h_L.size() != p->G) return cudaErrorInvalidValue;
    for (int64_t L : p->h_L) {
        if (L < 1 || L > p->M) return cudaErrorInvalidValue;
        tiles += (L + TILE - 1) / TILE;
    }
    if (tiles < 1 || tiles > INT32_MAX) return cudaErrorInvalidValue;
    // the tile table (12 int64 bounds per entry, at most 96 M / TILE bytes per
    // grid), the list's grid starts and entries live in the second grid
    // buffer, which is free until the transform
    static_assert(96 / TILE < 8, "the tile table must fit the second grid buffer");
    const size_t need = (size_t)tiles * 96 + (size_t)(p->G + 1) * 8 + (size_t)tiles * 8 + 16;
    if (need > (size_t)p->G * (size_t)p->M * sizeof(cpx<T>)) return cudaErrorInvalidValue;
    int64_t* rngtab = reinterpret_cast<int64_t*>(p->d_grid[1]);
    int64_t* tfirst = rngtab + tiles * 12;
    int32_t* tgrid = reinterpret_cast<int32_t*>(tfirst + p->G + 1);
    k_tile_list<TILE><<<1, 1024, 0, s>>>(p->d_L, p->G, tfirst);
    k_tile_fill<<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(tfirst, p->G, tiles, tgrid);
    const unsigned gt = (unsigned)((tiles * 12 + 127) / 128);
    k_tile_ranges<TILE><<<gt, 128, 0, s>>>(p->d_key, p->n, p->M, p->w, p->npk, p->H, p->w_p, tfirst,
                                           tgrid, p->d_slot_soff, p->d_slot_n, tiles, rngtab);
    if (p->npk == 0 && !g_spread_general_only) {
        // one sample set per grid: tiles that fit one batch in the single-batch
        // kernel, the rest listed (after the tile grids) for the general kernel
        int32_t* tlist = tgrid + tiles;
        int32_t* tcount = tlist + tiles;
        cudaError_t e = cudaMemsetAsync(tcount, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        k_spread1<T, TILE, NT, CAP1><<<(unsigned)tiles, NT, 0, s>>>(
            p->d_key, (const T*)p->d_dlt, (const cpx<T>*)p->d_cs, p->n, p->M, p->w, (T)p->beta,
            tfirst, tgrid, (cpx<T>*)p->d_grid[0], p->M, p->d_slot_soff, rngtab, tlist, tcount);
        const unsigned gb = (unsigned)std::min<int64_t>(tiles, (int64_t)device_sm_count() * 2);
        k_spread<T, TILE, NT, CAP><<<gb, NT, 0, s>>>(
            p->d_key, (const T*)p->d_dlt, (const cpx<T>*)p->d_cs, p->n, p->M, p->w, (T)p->beta,
            p->npk, p->H, p->w_p, (T)p->beta_p, tfirst, tgrid, (cpx<T>*)p->d_grid[0], p->M,
            p->d_slot_soff, p->d_slot_n, rngtab, tlist, tcount);
        return cudaGetLastError();
    }
    k_spread<T, TILE, NT, CAP><<<(unsigned)tiles, NT, 0, s>>>(
        p->d_key, (const T*)p->d_dlt, (const cpx<T>*)p->d_cs, p->n, p->M, p->w, (T)p->beta,
        p->npk, p->H, p->w_p, (T)p->beta_p, tfirst, tgrid, (cpx<T>*)p->d_grid[0], p->M,
        p->d_slot_soff, p->d_slot_n, rngtab, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t spread_impl(fc2_plan_s* p, cudaStream_t s) {
    // a tile must be at most half the grid so the three key ranges are disjoint;
    // the batched path may choose another tile width (its autotuner)
    const int tile = spread_tile_of(p->M, p->spread_tile);
    switch (tile) {
        case 2048: return spread_tiles<T, 2048, 256, 2048, 1024>(p, s);
        case 1024: return spread_tiles<T, 1024, 256, 2048, 1024>(p, s);
        case 512: return spread_tiles<T, 512, 128, 2048, 512>(p, s);
        default: return spread_tiles<T, 128, 128, 1024, 256>(p, s);
    }
}

// ------------------------------------------------------- the paper's gridding
// Nearest-lower-cell binning (Sec. 3b): sample i (time order) lands in cell
// floor(frac(df tau_i) M) = B_i >> (64 - logM) of the one zero-padded array,
// which takes q + i p, the weight and the weighted data (Kronecker delta, no
// spreading).  The first sample of each run of equal cells sums the run in
// sample order.  Without a wrap of the fold (df * max tau < 1) the cells grow
// with time, runs are disjoint and the result is reproducible; with a wrap,
// runs from different turns of the fold meet in one cell and are added with
// atomics.
template <typename T>
__global__ void k_bin(const uint64_t* __restrict__ B, const double* __restrict__ wq,
                      const double* __restrict__ wp, int64_t n, int logM,
                      cpx<T>* __restrict__ grid, int atomic) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sh = 64 - logM;
    const uint64_t c = B[i] >> sh;
    if (i > 0 && (B[i - 1] >> sh) == c) return;
    double q = 0.0, v = 0.0;
    for (int64_t k = i; k < n && (B[k] >> sh) == c; ++k) {
        q += wq[k];
        v += wp[k];
    }
    if (atomic) {
        atomicAdd(&grid[c].x, (T)q);
        atomicAdd(&grid[c].y, (T)v);
    } else {
        grid[c] = mk<T>((T)q, (T)v);
    }
}

cudaError_t launch_bin(fc2_plan_s* p, cudaStream_t s) {
    const size_t csz = p->fp64 ? 16 : 8;
    cudaError_t e = cudaMemsetAsync(p->d_grid[0], 0, (size_t)p->M * csz, s);
    if (e != cudaSuccess) return e;
    const int atomic = (p->df * p->scal[SC_TAUMAX] >= 1.0) ? 1 : 0;
    const unsigned blocks = (unsigned)((p->n + 255) / 256);
    if (p->fp64)
        k_bin<double><<<blocks, 256, 0, s>>>(p->d_phB, p->d_wq, p->d_wp, p->n, p->logM,
                                             (cpx<double>*)p->d_grid[0], atomic);
    else
        k_bin<float><<<blocks, 256, 0, s>>>(p->d_phB, p->d_wq, p->d_wp, p->n, p->logM,
                                            (cpx<float>*)p->d_grid[0], atomic);
    return cudaGetLastError();
}

cudaError_t launch_spread(fc2_plan_s* p, cudaStream_t s) {
    return p->fp64 ? spread_impl<double>(p, s) : spread_impl<float>(p, s);
}

void force_spread_general(int on) { g_spread_general_only = on ? 1 : 0; }

}  // namespace fc2
