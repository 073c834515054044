// k_signif.cu -- significance of the trial frequencies (Sec. 3d).
//
// The paper ranks frequencies by the probability, under the constant-source
// null hypothesis, of a chi^2 decrease this large at this frequency or below:
//     p(f) = fhat * P_{2H', >= Delta chi^2}(Delta chi^2_{H'}(f)),
// P the chi^2 survival function with 2H' degrees of freedom and fhat the trial
// count so far, f / df (taken as at least 1).  For an even number of degrees of
// freedom the survival function is a finite Poisson sum,
//     P = e^{-y} S(y),  S(y) = sum_{i < H'} y^i / i!,  y = Delta chi^2 / 2,
// so ln p = ln fhat - y + ln S(y).  The large term -y stays double (it carries
// Delta chi^2's own precision); ln fhat + ln S is evaluated in float, whose
// rounding (a few 1e-5 absolute) is far below the error of Delta chi^2.  The
// kernels write ln p for every (H', j) when asked, find the minimum of each
// row (ties to the lowest j), and evaluate the adjusted-Delta chi^2 factor
//     s_{H'} = (n - 2H' - 1) / (chi2_0 - Delta chi^2_best(H')),
// Delta chi^2_adj = s_{H'} Delta chi^2 (Sec. 3d's definition with the best
// fit's residual chi^2 per degree of freedom as the denominator).
#include <cuda_runtime.h>

#include <algorithm>

#include "fc2_common.cuh"
#include "fc2_internal.h"
#include "fc2_solve.cuh"

namespace fc2 {

namespace {

constexpr int SG_NT = 256;
constexpr int SG_PER = 8;
constexpr int SG_B = SG_NT * SG_PER;
constexpr int SG_NW = SG_NT / 32;

// ln S(y) = ln sum_{i < Hp} y^i / i! in float: a Horner sum for small y, and for
// y >= 16 the form (Hp - 1) ln y - ln (Hp - 1)! + ln T with
// T = sum_m (Hp - 1)! / (Hp - 1 - m)! y^{-m}, whose terms all stay bounded.
FC2_D float log_poisson_sum(float y, int Hp) {
    if (y < 16.0f) {
        float S = 1.0f;
        for (int i = Hp - 1; i >= 1; --i) S = fmaf(S, y / (float)i, 1.0f);
        return logf(S);
    }
    float T = 1.0f, lnfact = 0.0f;
    const float iy = 1.0f / y;
    for (int k = 1; k < Hp; ++k) {
        T = fmaf(T, (float)k * iy, 1.0f);
        lnfact += logf((float)k);
    }
    return (float)(Hp - 1) * logf(y) - lnfact + logf(T);
}

// ln p of one value: d = Delta chi^2_{Hp}(f_j), lf = ln fhat_j (float).
FC2_D double log_p_of(double d, int Hp, float lf) {
    // y = d / 2 by an exponent decrement (integer pipes); d <= 0 or tiny -> 0
    const int64_t b = __double_as_longlong(d);
    const double y = (b > (int64_t)(2ll << 52)) ? __longlong_as_double(b - (1ll << 52)) : 0.0;
    const float small = lf + log_poisson_sum(d2f_trunc(y), Hp);
    return f2d_exact(small) - y;
}

// ln fhat_j = ln max(f_min / df + j, 1), in float.
FC2_D float log_fhat(double f0, int64_t j) {
    const float fh = d2f_trunc(f0 + (double)j);
    return logf(fmaxf(fh, 1.0f));
}

// Stage 1: per (row, block of SG_B bins) the minimum of ln p (as the maximum of
// the integer key of -ln p, ties to the lowest j); ln p written if logp != 0.
__global__ void __launch_bounds__(SG_NT) k_logp1(const double* __restrict__ d, int64_t N, int H,
                                                 double f0, double* __restrict__ logp,
                                                 Cand* __restrict__ bmin, int nblk) {
    __shared__ Cand wres[SG_NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SG_B;
    float lf[SG_PER];
#pragma unroll
    for (int q = 0; q < SG_PER; ++q) lf[q] = log_fhat(f0, base + threadIdx.x + (int64_t)q * SG_NT);
    for (int h = 0; h < H; ++h) {
        const double* row = d + (int64_t)h * N;
        int64_t v = KEY_NONE, jb = INT64_MAX;
#pragma unroll
        for (int q = 0; q < SG_PER; ++q) {
            const int64_t j = base + threadIdx.x + (int64_t)q * SG_NT;
            if (j < N) {
                const double lp = log_p_of(row[j], h + 1, lf[q]);
                if (logp) logp[(int64_t)h * N + j] = lp;
                const int64_t k = okey(-lp);
                if (better(k, j, v, jb)) { v = k; jb = j; }
            }
        }
        warp_best(v, jb);
        if (lane == 0) wres[w] = Cand{v, jb};
        __syncthreads();
        if (w == 0) {
            v = lane < SG_NW ? wres[lane].k : KEY_NONE;
            jb = lane < SG_NW ? wres[lane].j : INT64_MAX;
            warp_best(v, jb);
            if (lane == 0) bmin[(int64_t)h * nblk + blockIdx.x] = Cand{v, jb};
        }
        __syncthreads();
    }
}

// Stage 2: one warp per row reduces the block minima; lane 0 writes the bin,
// its ln p and the adjusted-Delta chi^2 factor of the row.
__global__ void k_logp2(const Cand* __restrict__ bmin, int nblk, const double* __restrict__ d,
                        int64_t N, int H, double f0, const fc2_best* __restrict__ best,
                        const double* __restrict__ scal, int64_t n, int extra,
                        int64_t* __restrict__ jmin, double* __restrict__ lpmin,
                        double* __restrict__ adj) {
    const int h = blockIdx.x;
    const int lane = threadIdx.x;
    if (h >= H) return;
    int64_t v = KEY_NONE, jb = INT64_MAX;
    for (int b = lane; b < nblk; b += 32) {
        const Cand c = bmin[(int64_t)h * nblk + b];
        if (better(c.k, c.j, v, jb)) { v = c.k; jb = c.j; }
    }
    warp_best(v, jb);
    if (lane != 0) return;
    const bool found = jb >= 0 && jb < N;
    jmin[h] = found ? jb : -1;
    lpmin[h] = found ? log_p_of(d[(int64_t)h * N + jb], h + 1, log_fhat(f0, jb)) : 0.0;
    const double chi0 = scal[SC_CHI0];
    const double resid = chi0 - best[h].dchi2;
    const double dof = (double)(n - 2 * (h + 1) - 1 - extra);  // extra: a jointly fitted trend
    adj[h] = (resid > 0.0 && dof > 0.0) ? dof / resid : 0.0;
}

}  // namespace

// Significance of the plan's last execute: logp [H][N] on the device (or
// nullptr), and per row jmin, lpmin, adj into device arrays of H entries.
cudaError_t launch_significance(fc2_plan_s* p, double* logp, int64_t* jmin, double* lpmin,
                                double* adj, cudaStream_t s) {
    const int64_t N = p->N;
    const int H = p->H;
    const int nblk = (int)((N + SG_B - 1) / SG_B);
    const double f0 = p->f_min / p->df;
    Cand* bmin = nullptr;
    cudaError_t e = pool_alloc((void**)&bmin, (size_t)H * nblk * sizeof(Cand), s);
    if (e != cudaSuccess) return e;
    k_logp1<<<(unsigned)nblk, SG_NT, 0, s>>>(p->d_dchi2, N, H, f0, logp, bmin, nblk);
    k_logp2<<<(unsigned)H, 32, 0, s>>>(bmin, nblk, p->d_dchi2, N, H, f0, p->d_best, p->d_scal,
                                       p->n, p->joint ? p->D : 0, jmin, lpmin, adj);
    e = cudaGetLastError();
    cudaFreeAsync(bmin, s);
    return e;
}

}  // namespace fc2
