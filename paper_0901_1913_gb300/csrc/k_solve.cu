// k_solve.cu -- per-frequency normal equations, bordered Cholesky, exact
// fix-up of ill-conditioned bins, peak selection and coefficients.
//
// Paper: Sec. 2 Eqs. "eqalphafirst".."eqalpha" (alpha from C', S' at (h -+ h') f),
// the beta equations (C, S at h f), Eq. "eqchix" (chi2_min = X - beta^T alpha^-1 beta),
// Eq. "eqcoeffs" (A = alpha^-1 beta), Sec. 3c (Delta chi^2 = beta^T alpha^-1 beta with
// mean-subtracted data), Sec. 3e (best frequency = largest Delta chi^2; several
// candidate frequencies).
//
// Bordered Cholesky: with alpha = L L^T and z = L^-1 beta, the leading
// (2H'+1)-square block of alpha factors as the leading block of L, so
//   Delta chi^2_{H'} = sum_{l=1..2H'} z_l^2
// for every H' from one factorisation (z_0^2 = beta_0^2 / alpha_00 is the
// constant-only projection, zero up to rounding, and is excluded).
// Rank rule (the paper is silent on singular alpha): column l is dropped when
// its relative pivot d_l / alpha_ll <= tau; dropped columns contribute nothing.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "fc2_common.cuh"
#include "fc2_df.cuh"
#include "fc2_internal.h"
#include "fc2_solve.cuh"

#include <algorithm>

namespace fc2 {

struct SolveParams {
    int64_t N;
    double tau;        // rank-drop threshold
    double eps_spec;   // absolute error of the normalised gridded alpha/beta entries
    double eps_f32;    // extra error of a float factorisation
    double err_fix;    // bins whose estimated normalised error exceeds this are recomputed
    double sq, sp, chi0, s1n;  // 1/W, 1/sqrt(W chi2_0), chi2_0, sum w(x - xbar) / sqrt(W chi2_0)
    double eps_t1, eps_t2;     // precision of the tier-1 and tier-2 exact sums (routing)
    // float copies for the float path (a conversion per thread would run on the
    // double pipe): sq, sp, chi0, s1n, tau, eps_spec + eps_f32, err_fix
    float fsq, fsp, fchi0, fs1n, ftau, feps, ferr;
    // the paper's gridding: one spectrum Z = Qhat + i Phat of length pM, bin j
    // at index fhat = s0 + j
    int paper;
    int64_t pM, s0;
};

template <typename TS>
struct SP;  // solve parameters in the path's precision
template <>
struct SP<float> {
    float sq, sp, chi0, s1n, tau, eps, err;
    FC2_HD explicit SP(const SolveParams& p)
        : sq(p.fsq), sp(p.fsp), chi0(p.fchi0), s1n(p.fs1n), tau(p.ftau), eps(p.feps), err(p.ferr) {}
};
template <>
struct SP<double> {
    double sq, sp, chi0, s1n, tau, eps, err;
    FC2_HD explicit SP(const SolveParams& p)
        : sq(p.sq), sp(p.sp), chi0(p.chi0), s1n(p.s1n), tau(p.tau), eps(p.eps_spec), err(p.err_fix) {}
};
FC2_D double to_double(float v) { return f2d_exact(v); }
FC2_D double to_double(double v) { return v; }

// Normalised system of bin j from the gridded spectra.  Packed layout
// (npk > 0): grid g keeps F = X_a + i X_b at modes +(sh + j) (row 2g) and
// -(sh + j) (row 2g + 1), so X_a = (F+ + conj F-) / 2 and
// X_b = (F+ - conj F-) / 2i, deconvolved by dec_p; grid k - 1 holds (Q_k, P_k)
// for k <= H, grid H + q holds (Q_{H+2q+1}, Q_{H+2q+2}).  Otherwise row g is
// transform g (Q_1..Q_2H, P_1..P_H), deconvolved by dec.
template <typename TS, int H>
FC2_D void load_gridded(const cpx<TS>* __restrict__ spec, const TS* __restrict__ dec,
                        const TS* __restrict__ dec_p, int npk, int64_t N, int64_t j, TS sq,
                        TS sp, TS s1n, Sys<TS, H>& S) {
    S.qr[0] = (TS)1;
    S.qi[0] = (TS)0;
    S.pr[0] = s1n;
    S.pi[0] = (TS)0;
    if (npk > 0) {
        const TS e = dec_p[j] * (TS)0.5;
        const TS eq = e * sq, ep = e * sp;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const cpx<TS> a = spec[(int64_t)(2 * k - 2) * N + j];
            const cpx<TS> b = spec[(int64_t)(2 * k - 1) * N + j];
            S.qr[k] = (a.x + b.x) * eq;
            S.qi[k] = (a.y - b.y) * eq;
            S.pr[k] = (a.y + b.y) * ep;
            S.pi[k] = (b.x - a.x) * ep;
        }
#pragma unroll
        for (int k = H + 1; k <= 2 * H; ++k) {
            const int g = H + (k - H - 1) / 2;
            const cpx<TS> a = spec[(int64_t)(2 * g) * N + j];
            const cpx<TS> b = spec[(int64_t)(2 * g + 1) * N + j];
            if (((k - H - 1) & 1) == 0) {
                S.qr[k] = (a.x + b.x) * eq;
                S.qi[k] = (a.y - b.y) * eq;
            } else {
                S.qr[k] = (a.y + b.y) * eq;
                S.qi[k] = (b.x - a.x) * eq;
            }
        }
        return;
    }
    const TS d = dec[j];
    const TS dq = d * sq, dp = d * sp;
#pragma unroll
    for (int k = 1; k <= 2 * H; ++k) {
        cpx<TS> v = spec[(int64_t)(k - 1) * N + j];
        S.qr[k] = v.x * dq;
        S.qi[k] = v.y * dq;
    }
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        cpx<TS> v = spec[(int64_t)(2 * H + k - 1) * N + j];
        S.pr[k] = v.x * dp;
        S.pi[k] = v.y * dp;
    }
}

// Normalised system of bin j under the paper's gridding (Sec. 3b-3c): one
// spectrum Z = Qhat + i Phat of the binned weights and weighted data, read at
// the multiples k fhat of the bin's index (Q at k = 1..2H, P at k = 1..H), the
// two real transforms separated by Qhat(m) = (Z(m) + conj Z(-m)) / 2 and
// Phat(m) = (Z(m) - conj Z(-m)) / 2i; no deconvolution (the paper's Kronecker
// delta has none).  The transform stores mode m at spec[M/2 + m]; k fhat < M/2
// by the choice of M.
template <typename TS, int H>
FC2_D void load_paper(const cpx<TS>* __restrict__ spec, int64_t M, int64_t fh, TS sq, TS sp,
                      TS s1n, Sys<TS, H>& S) {
    S.qr[0] = (TS)1;
    S.qi[0] = (TS)0;
    S.pr[0] = s1n;
    S.pi[0] = (TS)0;
    const TS hq = (TS)0.5 * sq, hp = (TS)0.5 * sp;
    const cpx<TS>* z0 = spec + M / 2;
#pragma unroll
    for (int k = 1; k <= 2 * H; ++k) {
        const int64_t m = (int64_t)k * fh;
        const cpx<TS> a = z0[m];
        const cpx<TS> b = z0[-m];
        S.qr[k] = (a.x + b.x) * hq;
        S.qi[k] = (a.y - b.y) * hq;
        if (k <= H) {
            S.pr[k] = (a.y + b.y) * hp;
            S.pi[k] = (b.x - a.x) * hp;
        }
    }
}

// Per trial frequency: deconvolve and normalise the 3H spectra, factor, and
// write Delta chi^2 for every H'.  A bin whose estimated error is too large
// for this precision goes to a list: the float path sends it to a double
// re-solve of the same spectra, the double path to the exact fix-up.
template <typename TS, int H>
__global__ void __launch_bounds__(128) k_assemble(const cpx<TS>* __restrict__ spec,
                                                  const TS* __restrict__ dec,
                                                  const TS* __restrict__ dec_p, int npk,
                                                  double* __restrict__ dchi2, SolveParams sp,
                                                  int32_t* __restrict__ list,
                                                  int32_t* __restrict__ list_count,
                                                  int64_t cap) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= sp.N) return;
    constexpr int m = 2 * H + 1;
    const SP<TS> q(sp);
    Sys<TS, H> S;
    if (sp.paper) load_paper<TS, H>(spec, sp.pM, sp.s0 + j, q.sq, q.sp, q.s1n, S);
    else load_gridded<TS, H>(spec, dec, dec_p, npk, sp.N, j, q.sq, q.sp, q.s1n, S);
    TS out[H];
    TS an2 = (TS)0;
    chol_solve<TS, H, true>(S, q.tau, out, &an2);
    if (!(est_err<TS>(an2, m, q.eps) <= q.err)) {
        int32_t pos = atomicAdd(list_count, 1);
        if (pos < cap) list[pos] = (int32_t)j;
    }
#pragma unroll
    for (int h = 0; h < H; ++h) dchi2[(int64_t)h * sp.N + j] = to_double(out[h] * q.chi0);
}

// Relative pivot of the gridded equations (float spectra, entries good to
// about 1e-7) below which a bin is taken as nearly singular and its exact
// sums start at the double tier.
constexpr double DMIN_T3 = 1e-7;

// Double re-solve of float-path bins; bins still too sensitive go on to the
// exact fix-up list.
template <int H>
__global__ void __launch_bounds__(128) k_resolve(const cpx<float>* __restrict__ spec,
                                                 const float* __restrict__ dec,
                                                 const float* __restrict__ dec_p, int npk,
                                                 double* __restrict__ dchi2, SolveParams sp,
                                                 const int32_t* __restrict__ rlist,
                                                 const int32_t* __restrict__ rcount, int64_t rcap,
                                                 int32_t* __restrict__ flist,
                                                 int32_t* __restrict__ fcount, int64_t fcap,
                                                 int32_t* __restrict__ flist2,
                                                 int32_t* __restrict__ fcount2,
                                                 int32_t* __restrict__ flist3,
                                                 int32_t* __restrict__ fcount3) {
    int64_t cnt = *rcount;
    if (cnt > rcap) cnt = rcap;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t b = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); b < cnt;
         b += (int64_t)gridDim.x * wpb) {
        const int64_t j = rlist[b];
        Sys<float, H> Sf;
        if (sp.paper) load_paper<float, H>(spec, sp.pM, sp.s0 + j, sp.fsq, sp.fsp, sp.fs1n, Sf);
        else load_gridded<float, H>(spec, dec, dec_p, npk, sp.N, j, sp.fsq, sp.fsp, sp.fs1n, Sf);
        Sys<double, H> S;
#pragma unroll
        for (int k = 0; k <= 2 * H; ++k) { S.qr[k] = Sf.qr[k]; S.qi[k] = Sf.qi[k]; }
#pragma unroll
        for (int k = 0; k <= H; ++k) { S.pr[k] = Sf.pr[k]; S.pi[k] = Sf.pi[k]; }
        double out[H], an2 = 0.0;
        const double dmin = warp_chol_solve<H, true>(S, sp.tau, out, &an2);
        if ((threadIdx.x & 31) == 0) {
            if (!(est_err<double>(an2, 2 * H + 1, sp.eps_spec) <= sp.err_fix)) {
                // exact fix-up: bins that these (gridded) equations already show
                // to be beyond float sums -- by the coefficient norm, or by a
                // small relative pivot (columns this solve drops come back with
                // large coefficients in the exact solve) -- start at the
                // double-float tier, and bins whose coefficient norm is beyond
                // the double-float sums too, or whose relative pivot is already
                // below what these equations resolve (DMIN_T3), start at the
                // double tier.  Each tier checks its own result and passes bins
                // on.
                const int m = 2 * H + 1;
                int32_t *lst = flist, *cnt = fcount;
                if (!(est_err<double>(an2, m, sp.eps_t2) <= sp.err_fix) || dmin < DMIN_T3) {
                    lst = flist3;
                    cnt = fcount3;
                } else if (!(est_err<double>(an2, m, sp.eps_t1) <= sp.err_fix) || dmin < 3e-3) {
                    lst = flist2;
                    cnt = fcount2;
                }
                int32_t pos = atomicAdd(cnt, 1);
                if (pos < fcap) lst[pos] = (int32_t)j;
            }
#pragma unroll
            for (int h = 0; h < H; ++h) dchi2[(int64_t)h * sp.N + j] = out[h] * sp.chi0;
        }
    }
}

// ------------------------------------------------- exact sums per bin
// Q_k = sum_i w_i e^{2 pi i k f tau_i} (k = 1..2H) and P_k = sum_i w_i (x_i - xbar)
// e^{2 pi i k f tau_i} (k = 1..H) straight from the samples (Eq. "eqPQ").
// Work items are (bin, chunk of samples); each CTA reduces its chunk in a fixed
// order and the final kernels add the chunks in order (reproducible).
// Three precisions, tried in turn for a bin until its error estimate (the
// coefficient-norm model of chol_solve) is within budget:
//  - tier 1: the phase f tau_i is reduced in double and held as a 32-bit
//    fixed-point fraction, so harmonic k's phase is an exact integer product;
//    sine/cosine in float, accumulation in compensated float.  Each term
//    carries an independent ~2e-7 relative error, so the sums are good to
//    ~2e-7 * sqrt(sum w^2), far below the gridded spectra's error for large n.
//  - tier 2: double-float phasors (table + Taylor from the exact 64-bit phase,
//    powers by multiplication) and double-float accumulation; worst-case
//    error ~1e-12 * sum w, on the float pipes.
//  - tier 3: everything in double (powers of e^{2 pi i f tau_i}).
// Fixed-point phases: A_i = frac(f_min tau_i) 2^64 and B_i = frac(df tau_i) 2^64
// (u64, from the exact double-double products), so that the phase of trial
// bin j is A_i + j B_i modulo 2^64 -- an exact integer, as is k times it.
__global__ void k_phase_fx(const double* __restrict__ tau, const double* __restrict__ wq,
                           const double* __restrict__ wp, int64_t n, double f_min, double df,
                           uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                           float* __restrict__ wq32, float* __restrict__ wp32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    A[i] = frac_fx(f_min, tau[i]);
    B[i] = frac_fx(df, tau[i]);
    const float qh = (float)wq[i], ph = (float)wp[i];
    wq32[i] = qh;
    wp32[i] = ph;
    wq32[n + i] = (float)(wq[i] - (double)qh);  // low parts for double-float sums
    wp32[n + i] = (float)(wp[i] - (double)ph);
}

// Tables e^{2 pi i a / 256} (entries 0..255) and e^{2 pi i b / 65536}
// (entries 256..511): double-float for df_phasor (tier 2), then the same in
// double (tier 3); then e^{2 pi i m / 65536}, m < 65536, double-float, for
// df_phasor16 (the last tier) at DFTAB_T16.
__global__ void k_init_dftab(dfc* __restrict__ tab, int with16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (with16 ? 512 + 65536 : 512)) return;
    double sn, cn;
    if (i < 512) {
        const double x = (i < 256) ? (double)i / 128.0 : (double)(i - 256) / 32768.0;
        sincospi(x, &sn, &cn);
        tab[i] = dfc{df_from_double(cn), df_from_double(sn)};
        reinterpret_cast<double2*>(tab + 512)[i] = make_double2(cn, sn);
    } else {
        sincospi((double)(i - 512) / 32768.0, &sn, &cn);
        tab[DFTAB_T16 + (i - 512)] = dfc{df_from_double(cn), df_from_double(sn)};
    }
}
constexpr unsigned DFTAB_INIT_BLOCKS = (512 + 65536 + 255) / 256;

// Lane 0 receives the warp's sum of (hi, lo) float pairs, added with
// error-free two-sums (all on the float pipes).
FC2_D float2 warp_sum_pair(float hi, float lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const dfl t = df_two_sum(hi, h2);
        hi = t.h;
        lo = lo + l2 + t.l;
    }
    return make_float2(hi, lo);
}

template <int HM, int TIER>
__global__ void __launch_bounds__(EX_NT) k_exact_partial(
    const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
    const float* __restrict__ wq32, const float* __restrict__ wp32,
    const double* __restrict__ wq, const double* __restrict__ wp, const dfc* __restrict__ dftab,
    int64_t n, const int32_t* __restrict__ bins32, const int64_t* __restrict__ bins64,
    const int32_t* __restrict__ count_dev, int64_t count, int64_t base, int64_t cap, int H,
    double* __restrict__ part) {
    constexpr int NV = 6 * HM;
    constexpr bool DRED = (TIER == 3 || TIER == 4);  // per-warp partials in double
    __shared__ double red[DRED ? EX_NT / 32 : 1][NV];
    __shared__ float2 redf[DRED ? 1 : EX_NT / 32][NV];
    __shared__ dfc stab[TIER == 2 ? 512 : 1];
    __shared__ double2 stab64[TIER == 3 ? 512 : 1];
    __shared__ float smax[2][EX_NT / 32];
    int64_t cnt = count_dev ? (int64_t)(*count_dev) - base : count;
    if (cnt > cap) cnt = cap;
    if (cnt <= 0) return;
    int64_t chunk;
    int nch;
    exact_geometry(n, cnt, &chunk, &nch);
    const int64_t items = cnt * nch;
    const int lane = threadIdx.x & 31, wpi = threadIdx.x >> 5;
    if constexpr (TIER == 2) {
        for (int i = threadIdx.x; i < 512; i += EX_NT) stab[i] = dftab[i];
        __syncthreads();
    }
    if constexpr (TIER == 3) {
        const double2* t64 = reinterpret_cast<const double2*>(dftab + 512);
        for (int i = threadIdx.x; i < 512; i += EX_NT) stab64[i] = t64[i];
        __syncthreads();
    }
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t b = it / nch;
        const int c = (int)(it % nch);
        const int64_t j = bins32 ? (int64_t)bins32[base + b] : bins64[base + b];
        const uint64_t ju = (uint64_t)(j >= 0 ? j : 0);
        const int64_t i0 = (int64_t)c * chunk;
        const int64_t i1 = (j >= 0) ? min(n, i0 + chunk) : i0;
        if constexpr (TIER == 1) {
            CompSum<float> fa[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) fa[v].init();
            for (int64_t i = i0 + threadIdx.x; i < i1; i += EX_NT) {
                const uint32_t u = (uint32_t)((Aph[i] + ju * Bph[i]) >> 32);
                const float a = wq32[i], bb = wp32[i];
#pragma unroll
                for (int k = 1; k <= 2 * HM; ++k) {
                    if (k <= 2 * H) {
                        const int32_t ph = (int32_t)(u * (uint32_t)k);  // [-1/2, 1/2) cycles
                        float sn, cn;
                        sincospif((float)ph * 4.656612873077393e-10f, &sn, &cn);  // 2^-31
                        fa[2 * (k - 1)].add(a * cn);
                        fa[2 * (k - 1) + 1].add(a * sn);
                        if (k <= H) {
                            fa[4 * HM + 2 * (k - 1)].add(bb * cn);
                            fa[4 * HM + 2 * (k - 1) + 1].add(bb * sn);
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float2 x = warp_sum_pair(fa[v].s, fa[v].c);
                if (lane == 0) redf[wpi][v] = x;
            }
        } else if constexpr (TIER == 2) {
            dfl fa[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) fa[v] = dfl{0.f, 0.f};
            for (int64_t i = i0 + threadIdx.x; i < i1; i += EX_NT) {
                const uint64_t u = Aph[i] + ju * Bph[i];
                const dfl a{wq32[i], wq32[n + i]}, bb{wp32[i], wp32[n + i]};
                const dfc z1 = df_phasor(u, stab, stab + 256);
                dfc z = z1;
#pragma unroll
                for (int k = 0; k < 2 * HM; ++k) {
                    if (k < 2 * H) {
                        df_acc_mul(fa[2 * k], a, z.re);
                        df_acc_mul(fa[2 * k + 1], a, z.im);
                        if (k < H) {
                            df_acc_mul(fa[4 * HM + 2 * k], bb, z.re);
                            df_acc_mul(fa[4 * HM + 2 * k + 1], bb, z.im);
                        }
                        if (k + 1 < 2 * H) z = dfc_mul(z, z1);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float2 x = warp_sum_pair(fa[v].h, fa[v].l);
                if (lane == 0) redf[wpi][v] = x;
            }
        } else if constexpr (TIER == 4) {
            // lph lanes per harmonic multiple k (lane = (k - 1) lph + r); warp w
            // takes samples i0 + r + lph (w + 8 q); sums exact in fixed point at
            // scales set by the item's largest weights
            float mq = 0.f, mp = 0.f;
            for (int64_t i = i0 + threadIdx.x; i < i1; i += EX_NT) {
                mq = fmaxf(mq, fabsf(wq32[i]));
                mp = fmaxf(mp, fabsf(wp32[i]));
            }
            mq = warp_max_f(mq);
            mp = warp_max_f(mp);
            if (lane == 0) { smax[0][wpi] = mq; smax[1][wpi] = mp; }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < EX_NT / 32; ++q) {
                mq = fmaxf(mq, smax[0][q]);
                mp = fmaxf(mp, smax[1][q]);
            }
            const int eq = fx_exponent(mq * 1.0000002f, i1 - i0 + 1);
            const int ep = fx_exponent(mp * 1.0000002f, i1 - i0 + 1);
            const int lph = 32 / (2 * H);
            const int g = lane / lph, r = lane - g * lph;
            long long acc[4] = {0, 0, 0, 0};
            if (g < 2 * H)
                fx_lane_sums<true>(Aph, Bph, wq32, wp32, n, ju, (uint64_t)(g + 1), i0, i1,
                                   r + (int64_t)lph * wpi, (int64_t)lph * (EX_NT / 32), g < H,
                                   dftab + DFTAB_T16, nullptr, exp2f((float)eq),
                                   exp2f((float)ep), acc);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                long long sacc = acc[q];
                for (int o = 1; o < lph; ++o) {
                    const long long y = __shfl_sync(0xffffffffu, acc[q], (lane + o) & 31);
                    if (r == 0) sacc += y;
                }
                acc[q] = sacc;
            }
            if (r == 0 && g < 2 * H) {
                const double uq = ldexp(1.0, -eq), up = ldexp(1.0, -ep);
                red[wpi][2 * g] = (double)acc[0] * uq;
                red[wpi][2 * g + 1] = (double)acc[1] * uq;
                if (g < H) {
                    red[wpi][4 * HM + 2 * g] = (double)acc[2] * up;
                    red[wpi][4 * HM + 2 * g + 1] = (double)acc[3] * up;
                }
            }
            // values of multiples beyond 2H (and P beyond H) are never read
            if (lane < NV) {
                const int v = lane;
                const bool used = (v < 4 * HM) ? (v / 2 < 2 * H) : ((v - 4 * HM) / 2 < H);
                if (!used) red[wpi][v] = 0.0;
            }
            for (int v = lane + 32; v < NV; v += 32) {
                const bool used = (v < 4 * HM) ? (v / 2 < 2 * H) : ((v - 4 * HM) / 2 < H);
                if (!used) red[wpi][v] = 0.0;
            }
        } else {
            double acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = 0.0;
            for (int64_t i = i0 + threadIdx.x; i < i1; i += EX_NT) {
                const double2 z1 = d_phasor(Aph[i] + ju * Bph[i], stab64, stab64 + 256);
                const double c1 = z1.x, s1 = z1.y;
                double cr = c1, ci = s1;
                const double a = wq[i], bb = wp[i];
#pragma unroll
                for (int k = 0; k < 2 * HM; ++k) {
                    if (k < 2 * H) {
                        acc[2 * k] = fma(a, cr, acc[2 * k]);
                        acc[2 * k + 1] = fma(a, ci, acc[2 * k + 1]);
                        if (k < H) {
                            acc[4 * HM + 2 * k] = fma(bb, cr, acc[4 * HM + 2 * k]);
                            acc[4 * HM + 2 * k + 1] = fma(bb, ci, acc[4 * HM + 2 * k + 1]);
                        }
                        const double nr = cr * c1 - ci * s1;
                        const double ni = cr * s1 + ci * c1;
                        cr = nr;
                        ci = ni;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double x = acc[v];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) red[wpi][v] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            double x = 0.0;
            if constexpr (DRED) {
#pragma unroll
                for (int q = 0; q < EX_NT / 32; ++q) x += red[q][threadIdx.x];
            } else {
                float hi = 0.0f, lo = 0.0f;
#pragma unroll
                for (int q = 0; q < EX_NT / 32; ++q) {
                    const float2 y = redf[q][threadIdx.x];
                    const dfl t = df_two_sum(hi, y.x);
                    hi = t.h;
                    lo += y.y + t.l;
                }
                x = (double)hi + (double)lo;
            }
            part[((b * nch) + c) * NV + threadIdx.x] = x;
        }
        __syncthreads();
    }
}

// Final step of a fix-up round: solve from the exact sums; bins whose
// estimated error with the round's sum precision eps_sums still exceeds
// err_fix are queued for the next tier (when `next` is given).
template <int H>
__global__ void __launch_bounds__(128) k_exact_dchi2(const double* __restrict__ part, int64_t n,
                              const int32_t* __restrict__ list,
                              const int32_t* __restrict__ count_dev, int64_t base, int64_t cap,
                              const double* __restrict__ scal, double tau_drop, double eps_sums,
                              double err_fix, int32_t* __restrict__ next,
                              int32_t* __restrict__ next_count, int64_t next_cap,
                              double* __restrict__ dchi2, int64_t N) {
    __shared__ double sh[4][6 * H];
    int64_t cnt = (int64_t)(*count_dev) - base;
    if (cnt > cap) cnt = cap;
    const int w = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;  // one system per warp
    if (b >= cnt) return;
    int64_t chunk;
    int nch;
    exact_geometry(n, cnt, &chunk, &nch);
    warp_sum_chunks<H>(part, b, nch, sh[w]);
    const int64_t j = list[base + b];
    Sys<double, H> S;
    exact_sys_from_sums<H>(sh[w], H, scal, S);
    double out[H], an2 = 0.0;
    const double dmin = warp_chol_solve<H, true>(S, tau_drop, out, &an2);
    if ((threadIdx.x & 31) != 0) return;
    // The coefficient norm only measures the error if these sums resolve the
    // system's smallest pivot: a relative pivot within 1e3 of the sums'
    // precision may be an artefact of their errors (which can also make the
    // coefficients look small), so such bins go on to the next tier too.
    if (next && (!(est_err<double>(an2, 2 * H + 1, eps_sums) <= err_fix) ||
                 dmin < 1e3 * eps_sums)) {
        int32_t pos = atomicAdd(next_count, 1);
        if (pos < next_cap) next[pos] = (int32_t)j;
    }
    const double chi0 = scal[SC_CHI0];
#pragma unroll
    for (int h = 0; h < H; ++h) dchi2[(int64_t)h * N + j] = out[h] * chi0;
}

// Coefficients of each record (Eq. "eqcoeffs"): back-substitution (dropped
// columns = 0), rotation of each (sin, cos) pair from the tau = t - T0 frame to
// absolute time, and xbar added to A_0 (Sec. 3b).
template <int HM>
__global__ void __launch_bounds__(128) k_exact_coeffs(const double* __restrict__ part, int nch,
                               const int64_t* __restrict__ rec_j, int nrec, int H,
                               const double* __restrict__ scal, double f_min, double df,
                               double tau_drop, fc2_best* __restrict__ out) {
    __shared__ double sh[4][6 * HM];
    const int w = threadIdx.x >> 5;
    const int r = blockIdx.x * (blockDim.x >> 5) + w;
    if (r >= nrec) return;
    warp_sum_chunks<HM>(part, r, nch, sh[w]);
    const int64_t j = rec_j[r];
    const int Hp = (r < H) ? r + 1 : H;  // best[h] has h + 1 harmonics; peaks have H
    fc2_best b;
    b.j = j; b.f = 0; b.dchi2 = 0; b.H = Hp; b.flags = 0;
    for (int l = 0; l < 2 * FC2_MAX_H + 1; ++l) b.A[l] = 0.0;
    if (j < 0) {
        if ((threadIdx.x & 31) == 0) out[r] = b;
        return;
    }
    Sys<double, HM> S;
    exact_sys_from_sums<HM>(sh[w], H, scal, S);
    double outv[HM], an2;
    double A[2 * HM + 1];
    warp_chol_solve<HM, false>(S, tau_drop, outv, &an2, H, A, Hp);
    if ((threadIdx.x & 31) != 0) return;
    const double W = scal[SC_W], chi0 = scal[SC_CHI0];
    const double unit = (W > 0.0) ? sqrt(chi0 / W) : 0.0;
    const double f = f_min + (double)j * df;
    b.f = f;
    b.dchi2 = outv[Hp - 1] * chi0;
    b.A[0] = A[0] * unit + scal[SC_XBAR];
    const double fT0 = f * scal[SC_T0];
    for (int h = 1; h <= Hp; ++h) {
        const double ph = (double)h * (fT0 - floor(fT0));
        double sn, cn;
        sincospi(2.0 * (ph - floor(ph)), &sn, &cn);
        const double as = A[2 * h - 1] * unit, ac = A[2 * h] * unit;
        b.A[2 * h - 1] = as * cn + ac * sn;
        b.A[2 * h] = ac * cn - as * sn;
    }
    out[r] = b;
}

// ----------------------------------------------------------------- peaks
constexpr int PK_NT = 256;
constexpr int PK_PER = 16;
constexpr int PK_B = PK_NT * PK_PER;
constexpr int PK_NW = PK_NT / 32;

// Top-K local maxima by a threshold: the K-th best of the per-block best
// local maxima, theta, is a lower bound of the K-th best local maximum overall
// (those K block maxima are K distinct local maxima >= theta), so the global
// top K are among the local maxima >= theta, which lie in at most K blocks.
// Order everywhere: key desc, then j asc (key = okey(value)).
//
// Stage 1: per block of PK_B bins, the argmax of every row (ties -> lowest j)
// and the best local maximum of row H (value > left, >= right; edges
// one-sided).
__global__ void __launch_bounds__(PK_NT) k_peaks1(const double* __restrict__ d, int64_t N, int H,
                                                  Cand* __restrict__ amax,
                                                  Cand* __restrict__ bmax, int nblk) {
    __shared__ Cand wres[PK_NW][FC2_MAX_H + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * PK_B;
    for (int h = 0; h < H; ++h) {
        const double* row = d + (int64_t)h * N;
        int64_t v = KEY_NONE, j = INT64_MAX;
#pragma unroll
        for (int q = 0; q < PK_PER; ++q) {
            const int64_t jj = base + threadIdx.x + (int64_t)q * PK_NT;
            if (jj < N) {
                const int64_t x = okey(row[jj]);
                if (better(x, jj, v, j)) { v = x; j = jj; }
            }
        }
        warp_best(v, j);
        if (lane == 0) wres[w][h] = Cand{v, j};
    }
    {
        const double* row = d + (int64_t)(H - 1) * N;
        int64_t v = KEY_NONE, j = INT64_MAX;
#pragma unroll
        for (int q = 0; q < PK_PER; ++q) {
            const int64_t jj = base + threadIdx.x + (int64_t)q * PK_NT;
            if (jj < N) {
                const int64_t x = okey(row[jj]);
                const bool left = (jj == 0) || (x > okey(row[jj - 1]));
                const bool right = (jj == N - 1) || (x >= okey(row[jj + 1]));
                if (left && right && better(x, jj, v, j)) { v = x; j = jj; }
            }
        }
        warp_best(v, j);
        if (lane == 0) wres[w][FC2_MAX_H] = Cand{v, j};
    }
    __syncthreads();
    if (w == 0) {
        for (int h = 0; h < H; ++h) {
            int64_t v = lane < PK_NW ? wres[lane][h].k : KEY_NONE;
            int64_t j = lane < PK_NW ? wres[lane][h].j : INT64_MAX;
            warp_best(v, j);
            if (lane == 0) amax[(int64_t)h * nblk + blockIdx.x] = Cand{v, j};
        }
        int64_t v = lane < PK_NW ? wres[lane][FC2_MAX_H].k : KEY_NONE;
        int64_t j = lane < PK_NW ? wres[lane][FC2_MAX_H].j : INT64_MAX;
        warp_best(v, j);
        if (lane == 0) bmax[blockIdx.x] = Cand{v, j};
    }
}

// Block-wide best of (v, j) over the CTA (blockDim.x <= 1024); every thread
// gets the winner.
FC2_D Cand block_best(int64_t v, int64_t j, Cand* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_best(v, j);
    if (lane == 0) ws[w] = Cand{v, j};
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? ws[lane].k : KEY_NONE;
        j = lane < nw ? ws[lane].j : INT64_MAX;
        warp_best(v, j);
        if (lane == 0) ws[32] = Cand{v, j};
    }
    __syncthreads();
    const Cand r = ws[32];
    __syncthreads();
    return r;
}

// Stage 2 (one CTA): best bin of every row, and theta = the K-th best block
// maximum (K rounds, each excluding what the previous rounds took).
__global__ void __launch_bounds__(1024) k_peaks2(const Cand* __restrict__ amax,
                                                 const Cand* __restrict__ bmax, int nblk, int H,
                                                 int K, int64_t* __restrict__ best_j,
                                                 Cand* __restrict__ theta,
                                                 int32_t* __restrict__ ncand) {
    __shared__ Cand ws[33];
    for (int h = 0; h < H; ++h) {
        int64_t v = KEY_NONE, j = INT64_MAX;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            const Cand c = amax[(int64_t)h * nblk + b];
            if (better(c.k, c.j, v, j)) { v = c.k; j = c.j; }
        }
        const Cand r = block_best(v, j, ws);
        if (threadIdx.x == 0) best_j[h] = (r.j == INT64_MAX) ? -1 : r.j;
    }
    int64_t pv = INT64_MAX, pj = -1;
    Cand th{KEY_NONE, INT64_MAX};
    for (int r = 0; r < K; ++r) {
        int64_t v = KEY_NONE, j = INT64_MAX;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            const Cand c = bmax[b];
            if (c.j != INT64_MAX && better(pv, pj, c.k, c.j) && better(c.k, c.j, v, j)) {
                v = c.k;
                j = c.j;
            }
        }
        const Cand c = block_best(v, j, ws);
        if (c.j == INT64_MAX) {  // fewer than K blocks hold a local maximum: keep them all
            th = Cand{KEY_NONE, INT64_MAX};
            break;
        }
        th = c;
        pv = c.k;
        pj = c.j;
    }
    if (threadIdx.x == 0) {
        *theta = th;
        *ncand = 0;
    }
}

// Stage 3: blocks whose best local maximum reaches theta list their local
// maxima that do (at most K blocks, PK_B / 2 maxima each, so `cap` =
// K PK_B / 2 entries never overflow).
__global__ void __launch_bounds__(PK_NT) k_peaks3(const double* __restrict__ d, int64_t N, int H,
                                                  const Cand* __restrict__ bmax,
                                                  const Cand* __restrict__ theta,
                                                  Cand* __restrict__ cand,
                                                  int32_t* __restrict__ ncand, int cap) {
    const Cand th = *theta;
    const Cand bm = bmax[blockIdx.x];
    if (bm.j == INT64_MAX || better(th.k, th.j, bm.k, bm.j)) return;
    const double* row = d + (int64_t)(H - 1) * N;
    const int64_t base = (int64_t)blockIdx.x * PK_B;
    for (int q = 0; q < PK_PER; ++q) {
        const int64_t jj = base + threadIdx.x + (int64_t)q * PK_NT;
        if (jj >= N) break;
        const int64_t x = okey(row[jj]);
        const bool left = (jj == 0) || (x > okey(row[jj - 1]));
        const bool right = (jj == N - 1) || (x >= okey(row[jj + 1]));
        if (left && right && !better(th.k, th.j, x, jj)) {
            const int32_t pos = atomicAdd(ncand, 1);
            if (pos < cap) cand[pos] = Cand{x, jj};
        }
    }
}

// Stage 4 (one CTA): the K best candidates in order.
__global__ void __launch_bounds__(1024) k_peaks4(const Cand* __restrict__ cand,
                                                 const int32_t* __restrict__ ncand, int cap,
                                                 int K, int64_t* __restrict__ peak_j) {
    __shared__ Cand ws[33];
    const int64_t total = min((int64_t)*ncand, (int64_t)cap);
    int64_t pv = INT64_MAX, pj = -1;
    for (int r = 0; r < K; ++r) {
        int64_t v = KEY_NONE, j = INT64_MAX;
        for (int64_t b = threadIdx.x; b < total; b += blockDim.x) {
            const Cand c = cand[b];
            if (better(pv, pj, c.k, c.j) && better(c.k, c.j, v, j)) { v = c.k; j = c.j; }
        }
        const Cand c = block_best(v, j, ws);
        if (threadIdx.x == 0) peak_j[r] = (c.j == INT64_MAX) ? -1 : c.j;
        pv = c.j == INT64_MAX ? KEY_NONE : c.k;
        pj = c.j;
    }
}

// ---------------------------------------------------------------- launchers
static SolveParams solve_params(const fc2_plan_s* p) {
    SolveParams sp;
    sp.N = p->N;
    sp.tau = p->tau;
    sp.eps_spec = p->fp64 ? 1e-13 : 1e-7;
    sp.eps_f32 = 3e-7;
    sp.err_fix = 2e-5;
    const double W = p->scal[SC_W], chi0 = p->scal[SC_CHI0];
    sp.sq = 1.0 / W;
    sp.sp = (chi0 > 0.0) ? 1.0 / sqrt(W * chi0) : 0.0;
    sp.chi0 = chi0;
    sp.s1n = p->scal[SC_S1] * sp.sp;
    sp.fsq = (float)sp.sq; sp.fsp = (float)sp.sp; sp.fchi0 = (float)sp.chi0;
    sp.eps_t1 = 2e-7 * p->scal[SC_RW];
    sp.eps_t2 = 1.5e-12;  // EPS_DF
    sp.fs1n = (float)sp.s1n; sp.ftau = (float)sp.tau;
    sp.feps = (float)(sp.eps_spec + sp.eps_f32); sp.ferr = (float)sp.err_fix;
    sp.paper = p->paper ? 1 : 0;
    sp.pM = p->M;
    sp.s0 = p->s0;
    return sp;
}

template <typename TS>
static cudaError_t assemble_impl(fc2_plan_s* p, cudaStream_t s) {
    const SolveParams sp = solve_params(p);
    dim3 grid((unsigned)((p->N + 127) / 128));
    const cpx<TS>* spec = (const cpx<TS>*)p->d_spec;
    const TS* dec = (const TS*)p->d_dec;
    cudaMemsetAsync(p->d_flag_count, 0, 4 * sizeof(int32_t), s);
    // float path: list = re-solve list (counter 1); double path: exact list (counter 0)
    int32_t* list = p->fp64 ? p->d_flag_list : p->d_flag_list + p->flag_cap;
    int32_t* cnt = p->fp64 ? p->d_flag_count : p->d_flag_count + 1;
#define FC2_ASM(HH)                                                                           \
    case HH:                                                                                  \
        k_assemble<TS, HH><<<grid, 128, 0, s>>>(spec, dec, (const TS*)p->d_dec_p, p->npk,     \
                                                p->d_dchi2, sp, list, cnt, p->flag_cap);      \
        if (!p->fp64)                                                                         \
            k_resolve<HH><<<8 * 152, 32, 0, s>>>((const cpx<float>*)spec, (const float*)dec, \
                                                  (const float*)p->d_dec_p, p->npk,           \
                                                  p->d_dchi2, sp, list, cnt, p->flag_cap,     \
                                                  p->d_flag_list, p->d_flag_count,            \
                                                  p->flag_cap, p->d_flag_list + 2 * p->flag_cap,  \
                                                  p->d_flag_count + 2,                        \
                                                  p->d_flag_list + 3 * p->flag_cap,           \
                                                  p->d_flag_count + 3);                       \
        break;
    switch (p->H) {
        FC2_ASM(1) FC2_ASM(2) FC2_ASM(3) FC2_ASM(4) FC2_ASM(5) FC2_ASM(6) FC2_ASM(7) FC2_ASM(8)
        default: return cudaErrorInvalidValue;
    }
#undef FC2_ASM
    return cudaGetLastError();
}

cudaError_t launch_assemble(fc2_plan_s* p, cudaStream_t s) {
    if (p->joint) return launch_assemble_joint(p, s);
    return p->fp64 ? assemble_impl<double>(p, s) : assemble_impl<float>(p, s);
}

template <int HH, int TIER>
static void launch_partial(fc2_plan_s* p, const int32_t* b32, const int64_t* b64,
                           const int32_t* cnt_dev, int64_t cnt, int64_t base, int64_t cap,
                           cudaStream_t s) {
    k_exact_partial<HH, TIER><<<EX_GRID, EX_NT, 0, s>>>(
        p->d_phA, p->d_phB, p->d_wq32, p->d_wp32, p->d_wq, p->d_wp, (const dfc*)p->d_dftab, p->n,
        b32, b64, cnt_dev, cnt, base, cap, p->H, p->d_part);
}

cudaError_t launch_exact_partial_tier3(fc2_plan_s* p, int H, const int32_t* b32,
                                       const int64_t* b64, const int32_t* cnt_dev, int64_t cnt,
                                       int64_t base, int64_t cap, cudaStream_t s) {
    switch (H) {
        case 1: launch_partial<1, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 2: launch_partial<2, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 3: launch_partial<3, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 4: launch_partial<4, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 5: launch_partial<5, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 6: launch_partial<6, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 7: launch_partial<7, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        case 8: launch_partial<8, 3>(p, b32, b64, cnt_dev, cnt, base, cap, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Worst-case relative error of the double-float sums: phasor powers up to
// k = 16 by repeated multiplication, each step ~3 * 2^-47.
constexpr double EPS_DF = 1.5e-12;
constexpr double ERR_FIX = 2e-5;

// Last tier of the mixed path's fix-up: 4 (double-float terms, sums exact in
// fixed point; the default) or 3 (double; diagnostics).  The FP64 path always
// ends in tier 3.
static std::atomic<int> g_last_tier{4};
void set_last_fixup_tier(int tier) { g_last_tier.store(tier == 3 ? 3 : 4); }
int last_fixup_tier() { return g_last_tier.load(); }

// Exact fix-up of the flagged bins in up to three tiers.  Bins start at the
// tier the re-solve routed them to (lists 0, 2, 3 with n1, n2, n3 entries;
// the double path routes everything to tier 1); a bin that a tier cannot
// settle moves on to the next.  Rounds of at most exact_cap bins.  The later
// tiers read their bin counts on the device, so nothing waits for the host.
template <int HH>
static cudaError_t fixup_h(fc2_plan_s* p, int64_t n1, int64_t n2, int64_t n3, cudaStream_t s) {
    const int64_t cap = p->exact_cap;
    const double eps_t1 = 2e-7 * p->scal[SC_RW];
    int32_t* list1 = p->d_flag_list;
    int32_t* list2 = p->d_flag_list + 2 * p->flag_cap;
    int32_t* list3 = p->d_flag_list + 3 * p->flag_cap;
    int32_t* cnt1 = p->d_flag_count;
    int32_t* cnt2 = p->d_flag_count + 2;
    int32_t* cnt3 = p->d_flag_count + 3;
    const int64_t b2 = n1 + n2, b3 = n1 + n2 + n3;  // upper bounds after escalation
    for (int64_t base = 0; base < n1; base += cap) {
        const unsigned blocks = (unsigned)std::min(cap, n1 - base);
        launch_partial<HH, 1>(p, list1, nullptr, cnt1, 0, base, cap, s);
        k_exact_dchi2<HH><<<blocks, 32, 0, s>>>(p->d_part, p->n, list1, cnt1, base, cap, p->d_scal,
                                                 1e-13, eps_t1, ERR_FIX, list2, cnt2, p->flag_cap,
                                                 p->d_dchi2, p->N);
    }
    for (int64_t base = 0; base < b2; base += cap) {
        const unsigned blocks = (unsigned)std::min(cap, b2 - base);
        launch_partial<HH, 2>(p, list2, nullptr, cnt2, 0, base, cap, s);
        k_exact_dchi2<HH><<<blocks, 32, 0, s>>>(p->d_part, p->n, list2, cnt2, base, cap, p->d_scal,
                                                 1e-13, EPS_DF, ERR_FIX, list3, cnt3, p->flag_cap,
                                                 p->d_dchi2, p->N);
    }
    const bool fx_last = !p->fp64 && last_fixup_tier() == 4;
    for (int64_t base = 0; base < b3; base += cap) {
        const unsigned blocks = (unsigned)std::min(cap, b3 - base);
        if (fx_last) launch_partial<HH, 4>(p, list3, nullptr, cnt3, 0, base, cap, s);
        else launch_partial<HH, 3>(p, list3, nullptr, cnt3, 0, base, cap, s);
        k_exact_dchi2<HH><<<blocks, 32, 0, s>>>(p->d_part, p->n, list3, cnt3, base, cap, p->d_scal,
                                                 1e-13, 0.0, ERR_FIX, nullptr, nullptr, 0,
                                                 p->d_dchi2, p->N);
    }
    return cudaGetLastError();
}

// Delta chi^2 of nb given bins from tier-`tier` exact sums alone, written
// into the plan's output array (diagnostics and tests of each tier).
template <int HH>
static cudaError_t exact_bins_h(fc2_plan_s* p, int64_t nb, int tier, cudaStream_t s) {
    int32_t* list = p->d_flag_list;
    const unsigned blocks = (unsigned)nb;
    if (tier == 1) launch_partial<HH, 1>(p, list, nullptr, nullptr, nb, 0, nb, s);
    else if (tier == 2) launch_partial<HH, 2>(p, list, nullptr, nullptr, nb, 0, nb, s);
    else if (tier == 4) launch_partial<HH, 4>(p, list, nullptr, nullptr, nb, 0, nb, s);
    else launch_partial<HH, 3>(p, list, nullptr, nullptr, nb, 0, nb, s);
    int32_t* cnt = p->d_flag_count + 3;
    const int32_t nb32 = (int32_t)nb;
    cudaMemcpyAsync(cnt, &nb32, 4, cudaMemcpyHostToDevice, s);
    k_exact_dchi2<HH><<<blocks, 32, 0, s>>>(p->d_part, p->n, list, cnt, 0, nb, p->d_scal, 1e-13,
                                             0.0, ERR_FIX, nullptr, nullptr, 0, p->d_dchi2, p->N);
    return cudaStreamSynchronize(s);
}

cudaError_t launch_exact_bins(fc2_plan_s* p, int64_t nb, int tier, cudaStream_t s) {
    switch (p->H) {
        case 1: return exact_bins_h<1>(p, nb, tier, s);
        case 2: return exact_bins_h<2>(p, nb, tier, s);
        case 3: return exact_bins_h<3>(p, nb, tier, s);
        case 4: return exact_bins_h<4>(p, nb, tier, s);
        case 5: return exact_bins_h<5>(p, nb, tier, s);
        case 6: return exact_bins_h<6>(p, nb, tier, s);
        case 7: return exact_bins_h<7>(p, nb, tier, s);
        case 8: return exact_bins_h<8>(p, nb, tier, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fixup(fc2_plan_s* p, int64_t n1, int64_t n2, int64_t n3, cudaStream_t s) {
    if (p->joint) return launch_fixup_joint(p, n3, s);  // every flagged bin: exact double sums
    switch (p->H) {
        case 1: return fixup_h<1>(p, n1, n2, n3, s);
        case 2: return fixup_h<2>(p, n1, n2, n3, s);
        case 3: return fixup_h<3>(p, n1, n2, n3, s);
        case 4: return fixup_h<4>(p, n1, n2, n3, s);
        case 5: return fixup_h<5>(p, n1, n2, n3, s);
        case 6: return fixup_h<6>(p, n1, n2, n3, s);
        case 7: return fixup_h<7>(p, n1, n2, n3, s);
        case 8: return fixup_h<8>(p, n1, n2, n3, s);
        default: return cudaErrorInvalidValue;
    }
}

// Scratch of the peak search: amax [H][nblk], bmax [nblk], theta, the
// candidate count and list [K PK_B / 2], then the record bins [H + K].
static int64_t peaks_cap(int K) { return (int64_t)K * (PK_B / 2); }
size_t peaks_scratch_bytes(int64_t N, int H, int K) {
    const int64_t nblk = (N + PK_B - 1) / PK_B;
    return (size_t)(nblk * (H + 1) + 2 + peaks_cap(K)) * sizeof(Cand) + (size_t)(H + K) * 8 + 4096;
}

cudaError_t launch_peaks(fc2_plan_s* p, cudaStream_t s) {
    const int64_t nblk = (p->N + PK_B - 1) / PK_B;
    const int H = p->H, K = p->top_k;
    const int cap = (int)peaks_cap(K);
    Cand* amax = (Cand*)p->d_red;
    Cand* bmax = amax + nblk * H;
    Cand* theta = bmax + nblk;
    int32_t* ncand = (int32_t*)(theta + 1);
    Cand* cand = theta + 2;
    int64_t* rec_j = (int64_t*)(cand + cap);
    k_peaks1<<<(unsigned)nblk, PK_NT, 0, s>>>(p->d_dchi2, p->N, H, amax, bmax, (int)nblk);
    k_peaks2<<<1, 1024, 0, s>>>(amax, bmax, (int)nblk, H, K, rec_j, theta, ncand);
    k_peaks3<<<(unsigned)nblk, PK_NT, 0, s>>>(p->d_dchi2, p->N, H, bmax, theta, cand, ncand, cap);
    k_peaks4<<<1, 1024, 0, s>>>(cand, ncand, cap, K, rec_j + H);
    const int nrec = H + K;
    int64_t chunk;
    int nch;
    exact_geometry(p->n, nrec, &chunk, &nch);
    if (p->joint) return launch_records_joint(p, rec_j, nrec, nch, s);
#define FC2_CO(HH)                                                                            \
    case HH:                                                                                  \
        launch_partial<HH, 1>(p, nullptr, rec_j, nullptr, nrec, 0, nrec, s);               \
        k_exact_coeffs<HH><<<nrec, 32, 0, s>>>(p->d_part, nch, rec_j, nrec, H, p->d_scal,        \
                                            p->f_min, p->df, 1e-13, p->d_best);               \
        break;
    switch (H) {
        FC2_CO(1) FC2_CO(2) FC2_CO(3) FC2_CO(4) FC2_CO(5) FC2_CO(6) FC2_CO(7) FC2_CO(8)
        default: return cudaErrorInvalidValue;
    }
#undef FC2_CO
    return cudaGetLastError();
}

cudaError_t launch_phase_fx(fc2_plan_s* p, cudaStream_t s) {
    k_phase_fx<<<(unsigned)((p->n + 255) / 256), 256, 0, s>>>(p->d_tau, p->d_wq, p->d_wp, p->n,
                                                             p->f_min, p->df, p->d_phA, p->d_phB,
                                                             p->d_wq32, p->d_wp32);
    k_init_dftab<<<DFTAB_INIT_BLOCKS, 256, 0, s>>>((dfc*)p->d_dftab, 1);
    return cudaGetLastError();
}

cudaError_t launch_init_dftab(void* tab, bool with16, cudaStream_t s) {
    if (with16) k_init_dftab<<<DFTAB_INIT_BLOCKS, 256, 0, s>>>((dfc*)tab, 1);
    else k_init_dftab<<<2, 256, 0, s>>>((dfc*)tab, 0);
    return cudaGetLastError();
}

// The double-float phasor of each phase (diagnostics: its accuracy test), from
// the two 256-entry tables (df_phasor) or the 65536-entry one (df_phasor16).
__global__ void k_debug_phasor(const uint64_t* __restrict__ u, int64_t n,
                               const dfc* __restrict__ tab, int table16, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dfc z = table16 ? df_phasor16(u[i], tab + DFTAB_T16) : df_phasor(u[i], tab, tab + 256);
    out[4 * i] = z.re.h;
    out[4 * i + 1] = z.re.l;
    out[4 * i + 2] = z.im.h;
    out[4 * i + 3] = z.im.l;
}

cudaError_t debug_phasor(const uint64_t* u, int64_t n, int table16, float* out4) {
    void* d = nullptr;
    const size_t tb = DFTAB_BYTES;
    const size_t bytes = tb + (size_t)n * 8 + (size_t)n * 16;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return e;
    char* base = (char*)d;
    uint64_t* du = (uint64_t*)(base + tb);
    float* dout = (float*)(base + tb + (size_t)n * 8);
    e = launch_init_dftab(base, true, 0);
    if (e == cudaSuccess) e = cudaMemcpy(du, u, (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_debug_phasor<<<(unsigned)((n + 255) / 256), 256>>>(du, n, (const dfc*)base, table16, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out4, dout, (size_t)n * 16, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

size_t exact_scratch_bytes(int64_t n, int H, int64_t cap) {
    (void)n;
    return (size_t)cap * EX_MAX_CHUNKS * 6 * H * sizeof(double);
}

}  // namespace fc2

// ===========================================================================
// Allocation-free exact evaluation (fc2_dchi2_exact_noalloc).
//
// Some callers cannot allocate device memory at the moment they need an
// answer: code whose device memory is entirely reserved by another allocator
// (a framework's caching pool, a fixed arena), or a latency-critical loop that
// must not take the device-wide synchronisation that cudaMalloc/cudaFree can
// imply.  This entry point computes the same exact (ungridded) Delta chi^2 as
// the fix-up kernels above, but keeps all of its intermediate data in one
// file-scope device array of fixed size instead of plan-owned allocations.
//
// The array lives in every device that loads the library, until the process
// exits.  In host code its name is only a stand-in for the device symbol, so
// the kernels are handed the device address obtained once per device with
// cudaGetSymbolAddress (done by the first call on that device).  All calls on
// a device share the array: calls whose work overlaps on the GPU (e.g. issued
// on two streams without ordering between them) race with each other.
// ===========================================================================
namespace fc2 {
namespace {

constexpr int NA_NT = 256;
constexpr int NA_MAX_H = 8;
constexpr int64_t NA_MAX_N = 1ll << 22;
constexpr int64_t NA_MAX_BINS = 128;
constexpr int NA_MAX_CHUNKS = 64;
constexpr int64_t NA_MOM_CHUNK = 8192;
constexpr int64_t NA_MOM_BLOCKS = NA_MAX_N / NA_MOM_CHUNK;

// Layout of the scratch array (doubles unless noted):
//   [0, 16)                      scalars in the SC_* slots, status word at 15 (as int)
//   [16, 16 + 4 * NA_MOM_BLOCKS) per-block moment partials (4 doubles each)
//   then NA_MAX_BINS * NA_MAX_CHUNKS * 6 * NA_MAX_H chunk partials
constexpr int64_t NA_PART_OFF = 16 + 4 * NA_MOM_BLOCKS;
constexpr int64_t NA_DOUBLES = NA_PART_OFF + NA_MAX_BINS * NA_MAX_CHUNKS * 6 * NA_MAX_H;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// Device address of g_noalloc_scratch per device ordinal, with the unique ID
// of the context it was looked up in: after cudaDeviceReset the device has a
// new primary context and the address is looked up again.  Guarded by a mutex
// (first calls may come from several host threads).
struct NaScratchAddr {
    double* ptr = nullptr;
    unsigned long long ctx_id = 0;
};
std::mutex g_na_mu;
NaScratchAddr g_na_addr[64];

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points
// (no link against the driver library).
typedef int (*NaCtxGetCurrent)(void** ctx);
typedef int (*NaCtxGetId)(void* ctx, unsigned long long* id);
NaCtxGetCurrent g_na_get_ctx = nullptr;
NaCtxGetId g_na_get_id = nullptr;
std::once_flag g_na_once;

// Unique ID of the current context, or 0 if it cannot be read (the address is
// then looked up again on every call).
unsigned long long na_context_id() {
    std::call_once(g_na_once, [] {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_na_get_ctx = (NaCtxGetCurrent)f1;
            g_na_get_id = (NaCtxGetId)f2;
        }
        cudaGetLastError();
    });
    if (!g_na_get_ctx || !g_na_get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_na_get_ctx(&ctx) != 0 || !ctx || g_na_get_id(ctx, &id) != 0) return 0;
    return id;
}

__global__ void __launch_bounds__(NA_NT) k_na_moments(const double* __restrict__ t,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ sg, int64_t n,
                                                      int pass, double* __restrict__ scr) {
    __shared__ double sh[4][NA_NT];
    const int64_t a = (int64_t)blockIdx.x * NA_MOM_CHUNK;
    const int64_t b = min(n, a + NA_MOM_CHUNK);
    double v0 = 0.0, v1 = 0.0, v2 = INFINITY, bad = 0.0;
    const double xbar = pass ? scr[SC_XBAR] : 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += NA_NT) {
        const double si = sg[i], xi = x[i], ti = t[i];
        if (pass == 0) {
            if (!isfinite(ti) || !isfinite(xi) || !isfinite(si) || !(si > 0.0)) { bad = 1.0; continue; }
            const double w = 1.0 / (si * si);
            v0 += w;
            v1 += w * xi;
            v2 = fmin(v2, ti);
        } else {
            const double w = 1.0 / (si * si), d = xi - xbar;
            v0 += w * d * d;
            v1 += w * d;
        }
    }
    sh[0][threadIdx.x] = v0; sh[1][threadIdx.x] = v1; sh[2][threadIdx.x] = v2; sh[3][threadIdx.x] = bad;
    __syncthreads();
    for (int st = NA_NT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + st]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) scr[16 + 4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_na_moments_final(int nblk, int pass, double* __restrict__ scr) {
    if (threadIdx.x != 0) return;
    double v0 = 0.0, v1 = 0.0, v2 = INFINITY, bad = 0.0;
    for (int k = 0; k < nblk; ++k) {
        const double* q = scr + 16 + 4 * k;
        v0 += q[0]; v1 += q[1]; v2 = fmin(v2, q[2]); bad = fmax(bad, q[3]);
    }
    if (pass == 0) {
        scr[SC_W] = v0;
        scr[SC_XBAR] = v1 / v0;
        scr[SC_T0] = v2;
        if (bad != 0.0) reinterpret_cast<int*>(scr + 15)[0] = FC2_ERR_INVALID_ARG;
    } else {
        scr[SC_CHI0] = v0;
        scr[SC_S1] = v1;
    }
}

// Work items (bin, chunk): all-double sums, phases from the exact fixed-point
// reduction of (f_min + j df) (t - T0).
template <int HM>
__global__ void __launch_bounds__(NA_NT) k_na_partial(const double* __restrict__ t,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ sg, int64_t n,
                                                      int H, double f_min, double df,
                                                      const int64_t* __restrict__ bins, int64_t nb,
                                                      int64_t chunk, int nch,
                                                      double* __restrict__ scr) {
    constexpr int NV = 6 * HM;
    __shared__ double red[NA_NT / 32][NV];
    const double T0 = scr[SC_T0], xbar = scr[SC_XBAR];
    double* part = scr + NA_PART_OFF;
    const int lane = threadIdx.x & 31, wpi = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < nb * nch; it += gridDim.x) {
        const int64_t b = it / nch;
        const int c = (int)(it % nch);
        const uint64_t ju = (uint64_t)bins[b];
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
        const int64_t i0 = (int64_t)c * chunk, i1 = min(n, i0 + chunk);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += NA_NT) {
            const double tau = __dsub_rn(t[i], T0);
            const double si = sg[i];
            const double a = 1.0 / (si * si), bb = a * (x[i] - xbar);
            const int64_t ph = (int64_t)(frac_fx(f_min, tau) + ju * frac_fx(df, tau));
            double s1, c1;
            sincospi(ldexp((double)ph, -63), &s1, &c1);
            double cr = c1, ci = s1;
#pragma unroll
            for (int k = 0; k < 2 * HM; ++k) {
                if (k < 2 * H) {
                    acc[2 * k] = fma(a, cr, acc[2 * k]);
                    acc[2 * k + 1] = fma(a, ci, acc[2 * k + 1]);
                    if (k < H) {
                        acc[4 * HM + 2 * k] = fma(bb, cr, acc[4 * HM + 2 * k]);
                        acc[4 * HM + 2 * k + 1] = fma(bb, ci, acc[4 * HM + 2 * k + 1]);
                    }
                    const double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                    cr = nr;
                    ci = ni;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double y = acc[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
            if (lane == 0) red[wpi][v] = y;
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            double y = 0.0;
#pragma unroll
            for (int q = 0; q < NA_NT / 32; ++q) y += red[q][threadIdx.x];
            part[(b * nch + c) * NV + threadIdx.x] = y;
        }
        __syncthreads();
    }
}

template <int HM>
__global__ void __launch_bounds__(128) k_na_final(int64_t nb, int nch, int H, double tau_drop,
                                                  double* __restrict__ out,
                                                  double* __restrict__ scr) {
    __shared__ double sh[4][6 * HM];
    const int w = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;  // one system per warp
    if (b >= nb) return;
    warp_sum_chunks<HM>(scr + NA_PART_OFF, b, nch, sh[w]);
    Sys<double, HM> S;
    exact_sys_from_sums<HM>(sh[w], H, scr, S);
    double o[HM], an2 = 0.0;
    warp_chol_solve<HM, false>(S, tau_drop, o, &an2);
    if ((threadIdx.x & 31) != 0) return;
    const double chi0 = scr[SC_CHI0];
    for (int h = 0; h < H; ++h) out[(int64_t)h * nb + b] = o[h] * chi0;
}

template <int HM>
void na_launch(const double* t, const double* x, const double* sg, int64_t n, int H, double f_min,
               double df, const int64_t* bins, int64_t nb, int64_t chunk, int nch, double* out,
               double* scr, cudaStream_t s) {
    k_na_partial<HM><<<4 * 152, NA_NT, 0, s>>>(t, x, sg, n, H, f_min, df, bins, nb, chunk, nch,
                                                scr);
    k_na_final<HM><<<(unsigned)nb, 32, 0, s>>>(nb, nch, H, 1e-13, out, scr);
}

}  // namespace
}  // namespace fc2

extern "C" fc2_status fc2_dchi2_exact_noalloc(const double* t, const double* x,
                                              const double* sigma, int64_t n, int H,
                                              double f_min, double df, const int64_t* bins,
                                              int64_t nb, double* dchi2, void* cuda_stream) {
    using namespace fc2;
    if (!t || !x || !sigma || !bins || !dchi2) return FC2_ERR_INVALID_ARG;
    if (n < 1 || n > NA_MAX_N || H < 1 || H > NA_MAX_H || nb < 1 || nb > NA_MAX_BINS)
        return FC2_ERR_INVALID_ARG;
    if (!(isfinite(f_min) && f_min >= 0.0) || !(isfinite(df) && df > 0.0)) return FC2_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FC2_ERR_CUDA;
    // makes the device's primary context current (a no-op when it already is)
    if (cudaSetDevice(dev) != cudaSuccess) return FC2_ERR_CUDA;
    double* scr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        const unsigned long long id = na_context_id();
        NaScratchAddr& a = g_na_addr[dev];
        if (!a.ptr || id == 0 || id != a.ctx_id) {
            // first call on this device (or in its current context): the device
            // address of the scratch array
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return FC2_ERR_CUDA;
            }
            a.ptr = (double*)p;
            a.ctx_id = id;
        }
        scr = a.ptr;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int64_t chunk = (n + NA_MAX_CHUNKS - 1) / NA_MAX_CHUNKS;
    if (chunk < 2048) chunk = 2048;
    const int nch = (int)((n + chunk - 1) / chunk);
    const int nblk = (int)((n + NA_MOM_CHUNK - 1) / NA_MOM_CHUNK);
    // the status word must start at zero; everything else is overwritten
    if (cudaMemsetAsync(scr + 15, 0, sizeof(double), s) != cudaSuccess) return FC2_ERR_CUDA;
    for (int pass = 0; pass < 2; ++pass) {
        k_na_moments<<<nblk, NA_NT, 0, s>>>(t, x, sigma, n, pass, scr);
        k_na_moments_final<<<1, 32, 0, s>>>(nblk, pass, scr);
    }
    switch (H) {
        case 1: na_launch<1>(t, x, sigma, n, H, f_min, df, bins, nb, chunk, nch, dchi2, scr, s); break;
        case 2: na_launch<2>(t, x, sigma, n, H, f_min, df, bins, nb, chunk, nch, dchi2, scr, s); break;
        case 3: na_launch<3>(t, x, sigma, n, H, f_min, df, bins, nb, chunk, nch, dchi2, scr, s); break;
        case 4: na_launch<4>(t, x, sigma, n, H, f_min, df, bins, nb, chunk, nch, dchi2, scr, s); break;
        default: na_launch<8>(t, x, sigma, n, H, f_min, df, bins, nb, chunk, nch, dchi2, scr, s); break;
    }
    int status = 0;
    if (cudaGetLastError() != cudaSuccess) return FC2_ERR_CUDA;
    if (cudaMemcpyAsync(&status, scr + 15, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FC2_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FC2_ERR_CUDA;
    return status ? (fc2_status)status : FC2_OK;
}
