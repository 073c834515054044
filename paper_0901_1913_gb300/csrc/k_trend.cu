// k_trend.cu -- a polynomial trend fitted together with the harmonics.
//
// Sec. 4 reports detrending "with a polynomial fit" up to t^3.  With
// fc2_options.trend_fit the trend is part of the least-squares model: the null
// model is the weighted polynomial of degree D in u = (t - t_c) / s, and at
// every trial frequency the model is that polynomial plus the H' harmonics of
// Eq. "eqtrunc", all coefficients fitted together, so
//     Delta chi^2_{H'}(f) = chi^2(polynomial) - chi^2(polynomial + H' harmonics).
// The normal equations (Sec. 2) gain D + 1 polynomial columns u^p.  Their
// block G = sum w u^(p+q) does not depend on f, so it is factored once
// (G = L_G L_G^T, on the host) and eliminated: with C the polynomial-harmonic
// cross terms (sum w u^p sin/cos(2 pi h f t), i.e. Q_h for p = 0 and the extra
// transforms T_{p,h} = sum w u^p e^{2 pi i h f t} for p >= 1) and Y = L_G^-1 C,
// the harmonic block becomes alpha_HH - Y^T Y and its right-hand side
// beta_H - Y^T y_P (y_P = L_G^-1 beta_P), and a nested Cholesky factorisation
// of that (2H)-square system gives every H' at once (Sec. 1).  Everything is
// normalised by W and sqrt(W chi2_poly), so Delta chi^2' lies in [0, 1].
//
// One warp per trial frequency in double: lane l holds harmonic column l + 1.
// The gridded pass flags bins whose estimated error is too large; those, and
// the records, are recomputed from exact double sums over the samples (the Q
// and P sums of the double fix-up tier plus the trend sums T).
#include <cuda_runtime.h>

#include <algorithm>

#include "fc2_common.cuh"
#include "fc2_df.cuh"
#include "fc2_internal.h"
#include "fc2_solve.cuh"

namespace fc2 {

struct JointParams {
    int64_t N;
    double tau;      // rank-drop threshold on the relative pivot
    double eps;      // error of the normalised gridded entries (error estimate)
    double err_fix;  // bins whose estimated normalised error exceeds this are recomputed
    double sq;       // 1 / W
    double jsp;      // 1 / sqrt(W chi2_poly)
    double chi0;     // chi2_poly
    double LG[16];   // normalised polynomial Gram factor, lower triangle, row-major 4 x 4
    double yP[4];    // L_G^-1 beta_P (normalised)
};

// Harmonic-column solve of the projected system for one bin.  S holds the
// normalised Q (qr/qi, k = 0..2H) and P (pr/pi, k = 1..H) sums, T the
// normalised trend sums T_{p,h} at [(p - 1) H + h - 1] (re, im).  Every lane
// returns out[H' - 1] = Delta chi^2'_{H'} and the smallest relative pivot.
// With COEF, *anorm2 = max over H' <= H of the harmonic coefficient norm
// |A_H'|^2 (float, for the error estimate); with coef != nullptr, coef[0..2Hc)
// gets the Hc-harmonic coefficients and poly[0..D] the polynomial ones
// (normalised units).
template <int H, int D, bool COEF>
FC2_D double warp_joint_solve(const Sys<double, H>& S, const double* Tre, const double* Tim,
                              const JointParams& jp, double* out, double* anorm2,
                              double* coef = nullptr, int Hc = 0, double* poly = nullptr) {
    constexpr int m = 2 * H;
    static_assert(m <= 32, "one column per lane");
    constexpr unsigned FULL = 0xffffffffu;
    const int l = threadIdx.x & 31;
    const bool act = l < m;
    const int c = l + 1;             // column of the unprojected system
    const int h = (c + 1) >> 1;      // its harmonic
    const bool sn = (c & 1) != 0;    // sine column
    // this lane's cross terms C[p][c] and their projection Y = L_G^-1 C
    double Y[D + 1];
#pragma unroll
    for (int p = 0; p <= D; ++p) {
        double v = 0.0;
        if (act) {
            if (p == 0) v = S.alpha(c, 0);
            else v = sn ? Tim[(p - 1) * H + h - 1] : Tre[(p - 1) * H + h - 1];
        }
#pragma unroll
        for (int q = 0; q < p; ++q) v = fma(-jp.LG[p * 4 + q], Y[q], v);
        Y[p] = v / jp.LG[p * 4 + p];
    }
    // row l of the projected harmonic block (entries k <= l) and its rhs
    double a[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        double v = (act && k <= l) ? S.alpha(c, k + 1) : 0.0;
#pragma unroll
        for (int p = 0; p <= D; ++p) {
            const double yk = __shfl_sync(FULL, Y[p], k);
            v = fma(-Y[p], yk, v);
        }
        a[k] = (act && k <= l) ? v : 0.0;
    }
    double all = act ? S.alpha(c, c) : 0.0;
    double b = act ? S.beta(c) : 0.0;
#pragma unroll
    for (int p = 0; p <= D; ++p) {
        all = fma(-Y[p], Y[p], all);
        b = fma(-Y[p], jp.yP[p], b);
    }
    if (!act) all = 0.0;
    // right-looking Cholesky, lane l holding row l
    double Lr[m], z[m], dinv[m];
    double acc = 0.0;
    float dmin = 1.0f;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        const double dk = __shfl_sync(FULL, a[k], k);
        const double allk = __shfl_sync(FULL, all, k);
        const double bk = __shfl_sync(FULL, b, k);
        const bool keep = allk > 0.0 && dk > jp.tau * allk;
        const double di = keep ? rsqrt(dk) : 0.0;
        dinv[k] = di;
        const double zk = bk * di;
        z[k] = zk;
        const double Llk = (act && l > k) ? a[k] * di : 0.0;
        Lr[k] = Llk;
#pragma unroll
        for (int j = k + 1; j < m; ++j) {
            const double Ljk = __shfl_sync(FULL, Llk, j);
            if (j <= l) a[j] = fma(-Llk, Ljk, a[j]);
        }
        b = fma(-Llk, zk, b);
        const float rc = allk > 0.0 ? fmaxf((float)dk / (float)allk, 0.0f) : 0.0f;
        dmin = fminf(dmin, rc);
        acc = fma(zk, zk, acc);
        if ((k & 1) == 1) out[k >> 1] = acc;
    }
    if constexpr (COEF) {
        float amax = 0.0f;
#pragma unroll
        for (int hp = 1; hp <= H; ++hp) {
            const int mp = 2 * hp;
            float mine = 0.0f, nrm = 0.0f;
#pragma unroll
            for (int k = m - 1; k >= 0; --k) {
                if (k < mp) {
                    float t = (l > k && l < mp) ? (float)Lr[k] * mine : 0.0f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
                    const float A = ((float)z[k] - t) * (float)dinv[k];
                    if (l == k) mine = A;
                    nrm = fmaf(A, A, nrm);
                }
            }
            amax = fmaxf(amax, nrm);
        }
        *anorm2 = (double)amax;
    }
    if (coef) {
        const int mp = 2 * Hc;
        double mine = 0.0;
#pragma unroll
        for (int k = m - 1; k >= 0; --k) {
            if (k < mp) {
                double t = (l > k && l < mp) ? Lr[k] * mine : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
                const double A = (z[k] - t) * dinv[k];
                if (l == k) mine = A;
                coef[k] = A;
            } else {
                coef[k] = 0.0;
            }
        }
        // polynomial coefficients: L_G^T c = y_P - Y A (Y of the first 2 Hc columns)
        double r[D + 1];
#pragma unroll
        for (int p = 0; p <= D; ++p) {
            double v = (l < mp) ? Y[p] * mine : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            r[p] = jp.yP[p] - v;
        }
#pragma unroll
        for (int p = D; p >= 0; --p) {
            double v = r[p];
#pragma unroll
            for (int q = p + 1; q <= D; ++q) v = fma(-jp.LG[q * 4 + p], poly[q], v);
            poly[p] = v / jp.LG[p * 4 + p];
        }
    }
    return (double)dmin;
}

// ---------------------------------------------------------- gridded pass
// Warp per bin.  Spectra rows: Q_1..Q_2H, P_1..P_H, then T_{p,1..H} for
// p = 1..D (all deconvolved by dec[j]).  Bins whose error estimate is too
// large, or whose smallest relative pivot is below what these sums resolve,
// go to the exact list.
template <typename TS, int H, int D>
__global__ void __launch_bounds__(128) k_assemble_joint(const cpx<TS>* __restrict__ spec,
                                                        const TS* __restrict__ dec,
                                                        double* __restrict__ dchi2,
                                                        JointParams jp, double dmin_exact,
                                                        int32_t* __restrict__ list,
                                                        int32_t* __restrict__ list_count,
                                                        int64_t cap) {
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t j = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); j < jp.N;
         j += (int64_t)gridDim.x * wpb) {
        const double d = (double)dec[j];
        const double dq = d * jp.sq, dp = d * jp.jsp;
        Sys<double, H> S;
        S.qr[0] = 1.0; S.qi[0] = 0.0; S.pr[0] = 0.0; S.pi[0] = 0.0;
#pragma unroll
        for (int k = 1; k <= 2 * H; ++k) {
            const cpx<TS> v = spec[(int64_t)(k - 1) * jp.N + j];
            S.qr[k] = (double)v.x * dq;
            S.qi[k] = (double)v.y * dq;
        }
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const cpx<TS> v = spec[(int64_t)(2 * H + k - 1) * jp.N + j];
            S.pr[k] = (double)v.x * dp;
            S.pi[k] = (double)v.y * dp;
        }
        double Tre[D * H], Tim[D * H];
#pragma unroll
        for (int q = 0; q < D * H; ++q) {
            const cpx<TS> v = spec[(int64_t)(3 * H + q) * jp.N + j];
            Tre[q] = (double)v.x * dq;
            Tim[q] = (double)v.y * dq;
        }
        double out[H], an2 = 0.0;
        const double dmin = warp_joint_solve<H, D, true>(S, Tre, Tim, jp, out, &an2);
        if ((threadIdx.x & 31) == 0) {
            if (!(est_err<double>(an2, 2 * H + 1 + D, jp.eps) <= jp.err_fix) || dmin < dmin_exact) {
                const int32_t pos = atomicAdd(list_count, 1);
                if (pos < cap) list[pos] = (int32_t)j;
            }
#pragma unroll
            for (int hh = 0; hh < H; ++hh) dchi2[(int64_t)hh * jp.N + j] = out[hh] * jp.chi0;
        }
    }
}

// ------------------------------------------------------ exact trend sums
// T_{p,k} = sum_i w_i u_i^p e^{2 pi i k f tau_i} (p = 1..D, k = 1..H) in double,
// u_i = (tau_i - tc) is, for work items (bin, chunk of samples) laid out as the
// double tier's (exact_geometry), so both partial arrays share the chunking.
template <int H, int D>
__global__ void __launch_bounds__(256) k_exact_trend_partial(
    const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
    const double* __restrict__ tau, const double* __restrict__ wq,
    const dfc* __restrict__ dftab, int64_t n, double tc, double is,
    const int32_t* __restrict__ bins32, const int64_t* __restrict__ bins64,
    const int32_t* __restrict__ count_dev, int64_t count, int64_t base, int64_t cap,
    double* __restrict__ part_t) {
    constexpr int NV = 2 * D * H;
    constexpr int NT = 256;
    __shared__ double red[NT / 32][NV];
    __shared__ double2 stab64[512];
    int64_t cnt = count_dev ? (int64_t)(*count_dev) - base : count;
    if (cnt > cap) cnt = cap;
    if (cnt <= 0) return;
    int64_t chunk;
    int nch;
    exact_geometry(n, cnt, &chunk, &nch);
    const int64_t items = cnt * nch;
    const int lane = threadIdx.x & 31, wpi = threadIdx.x >> 5;
    {
        const double2* t64 = reinterpret_cast<const double2*>(dftab + 512);
        for (int i = threadIdx.x; i < 512; i += NT) stab64[i] = t64[i];
        __syncthreads();
    }
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t b = it / nch;
        const int ch = (int)(it % nch);
        const int64_t j = bins32 ? (int64_t)bins32[base + b] : bins64[base + b];
        const uint64_t ju = (uint64_t)(j >= 0 ? j : 0);
        const int64_t i0 = (int64_t)ch * chunk;
        const int64_t i1 = (j >= 0) ? min(n, i0 + chunk) : i0;
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += NT) {
            const double2 z1 = d_phasor(Aph[i] + ju * Bph[i], stab64, stab64 + 256);
            const double u = (tau[i] - tc) * is;
            double wu[D];
            double up = wq[i];
#pragma unroll
            for (int p = 0; p < D; ++p) { up *= u; wu[p] = up; }
            double cr = z1.x, ci = z1.y;
#pragma unroll
            for (int k = 0; k < H; ++k) {
#pragma unroll
                for (int p = 0; p < D; ++p) {
                    acc[2 * (p * H + k)] = fma(wu[p], cr, acc[2 * (p * H + k)]);
                    acc[2 * (p * H + k) + 1] = fma(wu[p], ci, acc[2 * (p * H + k) + 1]);
                }
                const double nr = cr * z1.x - ci * z1.y, ni = cr * z1.y + ci * z1.x;
                cr = nr;
                ci = ni;
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double x = acc[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) red[wpi][v] = x;
        }
        __syncthreads();
        for (int v = threadIdx.x; v < NV; v += NT) {
            double x = 0.0;
#pragma unroll
            for (int q = 0; q < NT / 32; ++q) x += red[q][v];
            part_t[((b * nch) + ch) * NV + v] = x;
        }
        __syncthreads();
    }
}

// Exact sums of one bin (warp w of the CTA): the Q / P partials of the double
// tier and the trend partials, each added in chunk order, normalised.
template <int H, int D>
FC2_D void joint_exact_sys(const double* __restrict__ part, const double* __restrict__ part_t,
                           int64_t b, int nch, const double* __restrict__ scal, double* sh,
                           double* sht, Sys<double, H>& S, double* Tre, double* Tim) {
    constexpr int NT2 = 2 * D * H;
    const int lane = threadIdx.x & 31;
    warp_sum_chunks<H>(part, b, nch, sh);
    for (int v = lane; v < NT2; v += 32) {
        double a = 0.0;
        for (int c = 0; c < nch; ++c) a += part_t[((b * nch) + c) * NT2 + v];
        sht[v] = a;
    }
    __syncwarp();
    exact_sys_from_sums<H>(sh, H, scal, S);  // scal's chi2_0 is the polynomial's chi^2
    const double iw = 1.0 / scal[SC_W];
#pragma unroll
    for (int q = 0; q < D * H; ++q) {
        Tre[q] = sht[2 * q] * iw;
        Tim[q] = sht[2 * q + 1] * iw;
    }
}

template <int H, int D>
__global__ void __launch_bounds__(128) k_exact_joint_dchi2(
    const double* __restrict__ part, const double* __restrict__ part_t, int64_t n,
    const int32_t* __restrict__ list, const int32_t* __restrict__ count_dev, int64_t base,
    int64_t cap, const double* __restrict__ scal, JointParams jp, double* __restrict__ dchi2) {
    __shared__ double sh[4][6 * H];
    __shared__ double sht[4][2 * D * H];
    int64_t cnt = (int64_t)(*count_dev) - base;
    if (cnt > cap) cnt = cap;
    const int w = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= cnt) return;
    int64_t chunk;
    int nch;
    exact_geometry(n, cnt, &chunk, &nch);
    Sys<double, H> S;
    double Tre[D * H], Tim[D * H];
    joint_exact_sys<H, D>(part, part_t, b, nch, scal, sh[w], sht[w], S, Tre, Tim);
    double out[H], an2 = 0.0;
    warp_joint_solve<H, D, false>(S, Tre, Tim, jp, out, &an2);
    if ((threadIdx.x & 31) != 0) return;
    const int64_t j = list[base + b];
#pragma unroll
    for (int hh = 0; hh < H; ++hh) dchi2[(int64_t)hh * jp.N + j] = out[hh] * jp.chi0;
}

// Records: Delta chi^2 and coefficients from the exact sums at each record's bin
// (record r < H has r + 1 harmonics, the peaks H).  Coefficients: harmonics in
// the absolute-time frame at A[1..2H'], A[0] = polynomial value at t_c + xbar,
// A[2H' + 1 .. 2H' + D] = the polynomial's higher coefficients in u.
template <int H, int D>
__global__ void __launch_bounds__(128) k_exact_joint_coeffs(
    const double* __restrict__ part, const double* __restrict__ part_t, int nch,
    const int64_t* __restrict__ rec_j, int nrec, const double* __restrict__ scal,
    JointParams jp, double f_min, double df, fc2_best* __restrict__ out) {
    __shared__ double sh[4][6 * H];
    __shared__ double sht[4][2 * D * H];
    const int w = threadIdx.x >> 5;
    const int r = blockIdx.x * (blockDim.x >> 5) + w;
    if (r >= nrec) return;
    const int64_t j = rec_j[r];
    const int Hp = (r < H) ? r + 1 : H;
    fc2_best rec;
    rec.j = j; rec.f = 0; rec.dchi2 = 0; rec.H = Hp; rec.flags = 0;
    for (int q = 0; q < 2 * FC2_MAX_H + 1; ++q) rec.A[q] = 0.0;
    if (j < 0) {
        if ((threadIdx.x & 31) == 0) out[r] = rec;
        return;
    }
    Sys<double, H> S;
    double Tre[D * H], Tim[D * H];
    joint_exact_sys<H, D>(part, part_t, r, nch, scal, sh[w], sht[w], S, Tre, Tim);
    double o[H], an2 = 0.0, coef[2 * H], poly[D + 1];
    warp_joint_solve<H, D, false>(S, Tre, Tim, jp, o, &an2, coef, Hp, poly);
    if ((threadIdx.x & 31) != 0) return;
    const double W = scal[SC_W];
    const double unit = (W > 0.0) ? sqrt(jp.chi0 / W) : 0.0;
    const double f = f_min + (double)j * df;
    rec.f = f;
    rec.dchi2 = o[Hp - 1] * jp.chi0;
    rec.A[0] = poly[0] * unit + scal[SC_XBAR];
    const double fT0 = f * scal[SC_T0];
    for (int hh = 1; hh <= Hp; ++hh) {
        const double ph = (double)hh * (fT0 - floor(fT0));
        double sn, cn;
        sincospi(2.0 * (ph - floor(ph)), &sn, &cn);
        const double as = coef[2 * hh - 2] * unit, ac = coef[2 * hh - 1] * unit;
        rec.A[2 * hh - 1] = as * cn + ac * sn;
        rec.A[2 * hh] = ac * cn - as * sn;
    }
    for (int p = 1; p <= D; ++p) rec.A[2 * Hp + p] = poly[p] * unit;
    out[r] = rec;
}

// ------------------------------------------------------------- launchers
static JointParams joint_params(const fc2_plan_s* p) {
    JointParams jp;
    jp.N = p->N;
    jp.tau = p->tau;
    jp.eps = p->fp64 ? 1e-13 : 1e-7;
    jp.err_fix = 2e-5;
    jp.sq = 1.0 / p->scal[SC_W];
    jp.chi0 = p->jt_chi0;
    jp.jsp = (p->jt_chi0 > 0.0) ? 1.0 / sqrt(p->scal[SC_W] * p->jt_chi0) : 0.0;
    for (int i = 0; i < 16; ++i) jp.LG[i] = p->jt_LG[i];
    for (int i = 0; i < 4; ++i) jp.yP[i] = p->jt_yP[i];
    return jp;
}

template <typename TS>
static cudaError_t assemble_joint_impl(fc2_plan_s* p, cudaStream_t s) {
    const JointParams jp = joint_params(p);
    cudaMemsetAsync(p->d_flag_count, 0, 4 * sizeof(int32_t), s);
    int32_t* list = p->d_flag_list + 3 * p->flag_cap;  // the double tier's list
    int32_t* cnt = p->d_flag_count + 3;
    const cpx<TS>* spec = (const cpx<TS>*)p->d_spec;
    const TS* dec = (const TS*)p->d_dec;
    const unsigned blocks = (unsigned)std::min<int64_t>((p->N + 3) / 4, 152 * 64);
    const double dmin_exact = p->fp64 ? 1e-11 : 1e-7;
#define FC2_JA(HH, DD)                                                                        \
    if (p->H == HH && p->D == DD) {                                                           \
        k_assemble_joint<TS, HH, DD><<<blocks, 128, 0, s>>>(spec, dec, p->d_dchi2, jp,        \
                                                            dmin_exact, list, cnt,            \
                                                            p->flag_cap);                     \
        return cudaGetLastError();                                                            \
    }
#define FC2_JA_H(HH) FC2_JA(HH, 1) FC2_JA(HH, 2) FC2_JA(HH, 3)
    FC2_JA_H(1) FC2_JA_H(2) FC2_JA_H(3) FC2_JA_H(4) FC2_JA_H(5) FC2_JA_H(6) FC2_JA_H(7)
    FC2_JA_H(8)
#undef FC2_JA_H
#undef FC2_JA
    return cudaErrorInvalidValue;
}

cudaError_t launch_assemble_joint(fc2_plan_s* p, cudaStream_t s) {
    return p->fp64 ? assemble_joint_impl<double>(p, s) : assemble_joint_impl<float>(p, s);
}

template <int HH, int DD>
static void trend_partial(fc2_plan_s* p, const int32_t* b32, const int64_t* b64,
                          const int32_t* cnt_dev, int64_t cnt, int64_t base, int64_t cap,
                          cudaStream_t s) {
    k_exact_trend_partial<HH, DD><<<4 * 152, 256, 0, s>>>(
        p->d_phA, p->d_phB, p->d_tau, p->d_wq, (const dfc*)p->d_dftab, p->n, p->jt_tc, p->jt_is,
        b32, b64, cnt_dev, cnt, base, cap, p->d_part_t);
}

// Exact fix-up of the n3 listed bins (rounds of at most exact_cap): the double
// tier's Q / P sums, the trend sums, and the projected solve.
template <int HH, int DD>
static cudaError_t fixup_joint_hd(fc2_plan_s* p, int64_t n3, cudaStream_t s) {
    const JointParams jp = joint_params(p);
    const int64_t cap = p->exact_cap;
    int32_t* list = p->d_flag_list + 3 * p->flag_cap;
    int32_t* cnt = p->d_flag_count + 3;
    for (int64_t base = 0; base < n3; base += cap) {
        launch_exact_partial_tier3(p, HH, list, nullptr, cnt, 0, base, cap, s);
        trend_partial<HH, DD>(p, list, nullptr, cnt, 0, base, cap, s);
        const unsigned blocks = (unsigned)((std::min(cap, n3 - base) + 3) / 4);
        k_exact_joint_dchi2<HH, DD><<<blocks, 128, 0, s>>>(p->d_part, p->d_part_t, p->n, list, cnt,
                                                            base, cap, p->d_scal, jp, p->d_dchi2);
    }
    return cudaGetLastError();
}

cudaError_t launch_fixup_joint(fc2_plan_s* p, int64_t n3, cudaStream_t s) {
#define FC2_JF(HH, DD) \
    if (p->H == HH && p->D == DD) return fixup_joint_hd<HH, DD>(p, n3, s);
#define FC2_JF_H(HH) FC2_JF(HH, 1) FC2_JF(HH, 2) FC2_JF(HH, 3)
    FC2_JF_H(1) FC2_JF_H(2) FC2_JF_H(3) FC2_JF_H(4) FC2_JF_H(5) FC2_JF_H(6) FC2_JF_H(7)
    FC2_JF_H(8)
#undef FC2_JF_H
#undef FC2_JF
    return cudaErrorInvalidValue;
}

template <int HH, int DD>
static cudaError_t records_joint_hd(fc2_plan_s* p, const int64_t* rec_j, int nrec, int nch,
                                    cudaStream_t s) {
    const JointParams jp = joint_params(p);
    launch_exact_partial_tier3(p, HH, nullptr, rec_j, nullptr, nrec, 0, nrec, s);
    trend_partial<HH, DD>(p, nullptr, rec_j, nullptr, nrec, 0, nrec, s);
    k_exact_joint_coeffs<HH, DD><<<(unsigned)((nrec + 3) / 4), 128, 0, s>>>(
        p->d_part, p->d_part_t, nch, rec_j, nrec, p->d_scal, jp, p->f_min, p->df, p->d_best);
    return cudaGetLastError();
}

cudaError_t launch_records_joint(fc2_plan_s* p, const int64_t* rec_j, int nrec, int nch,
                                 cudaStream_t s) {
#define FC2_JR(HH, DD) \
    if (p->H == HH && p->D == DD) return records_joint_hd<HH, DD>(p, rec_j, nrec, nch, s);
#define FC2_JR_H(HH) FC2_JR(HH, 1) FC2_JR(HH, 2) FC2_JR(HH, 3)
    FC2_JR_H(1) FC2_JR_H(2) FC2_JR_H(3) FC2_JR_H(4) FC2_JR_H(5) FC2_JR_H(6) FC2_JR_H(7)
    FC2_JR_H(8)
#undef FC2_JR_H
#undef FC2_JR
    return cudaErrorInvalidValue;
}

size_t trend_part_bytes(int64_t cap, int H, int D) {
    return (size_t)cap * 64 * 2 * D * H * sizeof(double);  // 64 = most chunks per bin
}

}  // namespace fc2
