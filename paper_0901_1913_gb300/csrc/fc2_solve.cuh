// fc2_solve.cuh -- per-frequency normal equations and their bordered Cholesky
// solve, shared by the single-curve and batched kernels.  Not part of the ABI.
//
// Paper: Sec. 2 Eqs. "eqalphafirst".."eqalpha" (alpha from C', S' at (h -+ h') f),
// the beta equations (C, S at h f), Eq. "eqchix" (chi2_min = X - beta^T alpha^-1 beta),
// Eq. "eqcoeffs" (A = alpha^-1 beta), Sec. 3c (Delta chi^2 with mean-subtracted data).
#pragma once
#include "fc2_common.cuh"
#include "fc2_internal.h"

namespace fc2 {

// Normalised system: alpha' = alpha / W, beta' = beta / sqrt(W chi2_0), so
// Delta chi^2' = Delta chi^2 / chi2_0 lies in [0, 1].
template <typename TC, int H>
struct Sys {
    TC qr[2 * H + 1], qi[2 * H + 1], pr[H + 1], pi[H + 1];

    FC2_HD TC alpha(int l, int k) const {
        if (l < k) { int t = l; l = k; k = t; }
        if (l == 0) return qr[0];
        const int hl = (l + 1) >> 1;
        const bool sl = (l & 1);
        if (k == 0) return sl ? qi[hl] : qr[hl];
        const int hk = (k + 1) >> 1;
        const bool sk = (k & 1);
        const int d = hl > hk ? hl - hk : hk - hl;
        const TC sg = hl > hk ? (TC)1 : (hl < hk ? (TC)-1 : (TC)0);
        const int s = hl + hk;
        const TC h = (TC)0.5;
        if (sl && sk) return h * (qr[d] - qr[s]);
        if (!sl && !sk) return h * (qr[d] + qr[s]);
        if (sl && !sk) return h * (qi[s] + sg * qi[d]);   // sin(hl) cos(hk)
        return h * (qi[s] - sg * qi[d]);                  // cos(hl) sin(hk)
    }
    FC2_HD TC beta(int l) const {
        if (l == 0) return pr[0];
        const int h = (l + 1) >> 1;
        return (l & 1) ? pi[h] : pr[h];
    }
};

// 1 / sqrt(d): one reciprocal square root in float (its rounding is far
// inside the float solve's error budget), the exact quotient in double.
FC2_D float inv_sqrt(float d) { return rsqrtf(d); }
FC2_D double inv_sqrt(double d) { return 1.0 / sqrt(d); }

// Factor and solve; out[H'-1] = Delta chi^2'_{H'}.  Returns the minimum
// relative pivot over all columns (clamped at 0).  With COEF, *anorm2 receives
// max over H' of |A^{(H')}|^2 (A^{(H')} = the H'-harmonic coefficients, by
// back-substitution L^T A = z on the leading block), the sensitivity of the
// result to errors in alpha and beta.  Optionally keeps L and z.
template <typename TC, int H, bool COEF>
FC2_D TC chol_solve(const Sys<TC, H>& S, TC tau, TC* out, TC* anorm2,
                    TC (*Lkeep)[2 * H + 1] = nullptr, TC* zkeep = nullptr, int Hrun = H) {
    constexpr int m = 2 * H + 1;
    TC L[m][m];
    TC z[m], dinv[m];
    TC acc = (TC)0, dmin = (TC)1;
#pragma unroll
    for (int l = 0; l < m; ++l) {
#pragma unroll
        for (int k = 0; k < l; ++k) {
            TC a = S.alpha(l, k);
#pragma unroll
            for (int p = 0; p < k; ++p) a = fma(-L[l][p], L[k][p], a);
            L[l][k] = a * dinv[k];
        }
        const TC all = S.alpha(l, l);
        TC d = all;
#pragma unroll
        for (int p = 0; p < l; ++p) d = fma(-L[l][p], L[l][p], d);
        TC b = S.beta(l);
#pragma unroll
        for (int p = 0; p < l; ++p) b = fma(-L[l][p], z[p], b);
        // keep the column when its relative pivot d / alpha_ll exceeds tau; the
        // quotient itself only feeds the returned minimum (and is dropped by
        // the compiler when a caller ignores it)
        if (all > (TC)0 && d > tau * all) {
            const TC di = inv_sqrt(d);
            L[l][l] = d * di;
            dinv[l] = di;
            z[l] = b * di;
        } else {
            L[l][l] = (TC)0;
            dinv[l] = (TC)0;
            z[l] = (TC)0;
        }
        const TC ratio = (all > (TC)0) ? d / all : (TC)0;
        const TC rc = ratio > (TC)0 ? ratio : (TC)0;
        dmin = rc < dmin ? rc : dmin;
        if (l > 0) acc = fma(z[l], z[l], acc);
        if (l > 0 && (l & 1) == 0) out[(l >> 1) - 1] = acc;
    }
    if constexpr (COEF) {
        TC amax = (TC)0;
#pragma unroll
        for (int hp = 1; hp <= H; ++hp) {
            if (hp > Hrun) break;  // harmonics beyond the curve's own H are padding
            const int mp = 2 * hp + 1;
            TC A[m];
            TC nrm = (TC)0;
#pragma unroll
            for (int l = m - 1; l >= 0; --l) {
                if (l < mp) {
                    TC a = z[l];
#pragma unroll
                    for (int k = l + 1; k < m; ++k)
                        if (k < mp) a = fma(-L[k][l], A[k], a);
                    A[l] = a * dinv[l];
                    nrm = fma(A[l], A[l], nrm);
                }
            }
            amax = nrm > amax ? nrm : amax;
        }
        *anorm2 = amax;
    }
    if (Lkeep) {
#pragma unroll
        for (int l = 0; l < m; ++l)
#pragma unroll
            for (int k = 0; k <= l; ++k) Lkeep[l][k] = L[l][k];
#pragma unroll
        for (int l = 0; l < m; ++l) zkeep[l] = z[l];
    }
    return dmin;
}

// Warp-cooperative chol_solve<double> for one system per warp (all 32 lanes
// call it with the same S): lane l holds row l of [alpha | beta] and the
// factorisation is right-looking, so each double instruction of the warp does
// up to m lanes of work (double instructions are expensive on this part
// whatever the number of active lanes).  Every lane returns the same out[]
// and minimum relative pivot.  With COEF, *anorm2 gets max over H' <= Hrun of
// |A^{(H')}|^2 computed in float (it only feeds the error estimate).  With
// coef != nullptr, coef[0..2Hc] gets the Hc-harmonic coefficients in double.
template <int H, bool COEF>
FC2_D double warp_chol_solve(const Sys<double, H>& S, double tau, double* out, double* anorm2,
                             int Hrun = H, double* coef = nullptr, int Hc = 0) {
    constexpr int m = 2 * H + 1;
    static_assert(m <= 32, "one row per lane");
    constexpr unsigned FULL = 0xffffffffu;
    const int l = threadIdx.x & 31;
    const bool act = l < m;
    double a[m];
#pragma unroll
    for (int k = 0; k < m; ++k) a[k] = (act && k <= l) ? S.alpha(l, k) : 0.0;
    const double all = act ? S.alpha(l, l) : 0.0;
    double b = act ? S.beta(l) : 0.0;
    double Lr[m], z[m], dinv[m];
    double acc = 0.0;
    float dmin = 1.0f;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        const double dk = __shfl_sync(FULL, a[k], k);
        const double allk = __shfl_sync(FULL, all, k);
        const double bk = __shfl_sync(FULL, b, k);
        const bool keep = allk > 0.0 && dk > tau * allk;
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
        if (k > 0) acc = fma(zk, zk, acc);
        if (k > 0 && (k & 1) == 0) out[(k >> 1) - 1] = acc;
    }
    if constexpr (COEF) {
        float Lf[m], zf[m], df[m];
#pragma unroll
        for (int k = 0; k < m; ++k) { Lf[k] = (float)Lr[k]; zf[k] = (float)z[k]; df[k] = (float)dinv[k]; }
        float amax = 0.0f;
#pragma unroll
        for (int hp = 1; hp <= H; ++hp) {
            if (hp > Hrun) break;
            const int mp = 2 * hp + 1;
            float mine = 0.0f, nrm = 0.0f;
#pragma unroll
            for (int k = m - 1; k >= 0; --k) {
                if (k < mp) {
                    float t = (l > k && l < mp) ? Lf[k] * mine : 0.0f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
                    const float A = (zf[k] - t) * df[k];
                    if (l == k) mine = A;
                    nrm = fmaf(A, A, nrm);
                }
            }
            amax = fmaxf(amax, nrm);
        }
        *anorm2 = (double)amax;
    }
    if (coef) {
        const int mp = 2 * Hc + 1;
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
    }
    return (double)dmin;
}

// Error model of a result computed from an alpha and beta whose entries carry
// absolute errors ~eps (normalised units): with A the coefficient vector,
// dDelta = 2 A^T dbeta - A^T dalpha A, so |dDelta| <~ eps (m |A|^2 + 2 sqrt(m) |A|).
template <typename TC>
FC2_HD TC est_err(TC anorm2, int m, TC eps) {
    return eps * ((TC)m * anorm2 + (TC)2 * sqrt((TC)m * anorm2));
}

// Fixed-point phase frac(a b) 2^64 from the exact double-double product a b.
FC2_D uint64_t frac_fx(double a, double b) {
    const double p = __dmul_rn(a, b);
    const double e = fma(a, b, -p);  // a b = p + e exactly
    const double fl = floor(p);
    const double r = __dsub_rn(p, fl);  // exact
    const uint64_t hi = (uint64_t)ldexp(r, 64 - 1) * 2ull + (uint64_t)0;  // r 2^64 (r < 1)
    const int64_t lo = (int64_t)ldexp(e, 63) * 2;                          // e 2^64
    return hi + (uint64_t)lo;
}

// ------------------------------------------------------------ exact sums
// Geometry of the exact sums' work items (bin, chunk of samples).
constexpr int EX_NT = 256;
constexpr int EX_GRID = 4 * 152;
constexpr int EX_MAX_CHUNKS = 64;

// Chunks of the sample range of each bin (at least 16 samples per thread, at
// most EX_MAX_CHUNKS).  While the bins do not outnumber the EX_GRID CTAs, the
// chunk count is rounded down so that no CTA gets more than two items (a
// third item on a few CTAs stretches the launch by one item time); with more
// bins than CTAs, each bin is cut as finely as allowed, so that the
// grid-stride loop hands every SM about the same share of small items.
// Evaluated identically on host and device, so kernels that read the bin
// count from device memory derive the same geometry.
FC2_HD void exact_geometry(int64_t n, int64_t count, int64_t* chunk, int* nch) {
    if (count < 1) count = 1;
    int64_t want = count <= EX_GRID ? (2 * EX_GRID) / count : EX_MAX_CHUNKS;
    if (want > EX_MAX_CHUNKS) want = EX_MAX_CHUNKS;
    int64_t c = (n + want - 1) / want;
    if (c < 16 * EX_NT) c = 16 * EX_NT;
    c = ((c + EX_NT - 1) / EX_NT) * EX_NT;
    *chunk = c;
    *nch = (int)((n + c - 1) / c);
}


// Warp w of the CTA owns record b: lanes add the chunk partials of values
// v = lane, lane + 32, ... in chunk order into sh[], then every lane of the
// warp can read the full sums.
template <int HM>
FC2_D void warp_sum_chunks(const double* __restrict__ part, int64_t b, int nch, double* sh) {
    constexpr int NV = 6 * HM;
    const int lane = threadIdx.x & 31;
    for (int v = lane; v < NV; v += 32) {
        double a = 0.0;
        for (int c = 0; c < nch; ++c) a += part[((b * nch) + c) * NV + v];
        sh[v] = a;
    }
    __syncwarp();
}


// Normalised system from exact sums acc = [Q_1..Q_2H (re, im) | P_1..P_H (re, im)]
// laid out with stride 4 HM between the Q and P parts.
template <int HM>
FC2_D void exact_sys_from_sums(const double* acc, int H, const double* __restrict__ scal,
                               Sys<double, HM>& S) {
    const double W = scal[SC_W], chi0 = scal[SC_CHI0];
    const double sq = (chi0 > 0.0) ? rsqrt(W * chi0) : 0.0;
    const double iw = 1.0 / W;
#pragma unroll
    for (int k = 0; k <= 2 * HM; ++k) { S.qr[k] = 0.0; S.qi[k] = 0.0; }
#pragma unroll
    for (int k = 0; k <= HM; ++k) { S.pr[k] = 0.0; S.pi[k] = 0.0; }
    S.qr[0] = 1.0;
    S.pr[0] = scal[SC_S1] * sq;
#pragma unroll
    for (int k = 1; k <= 2 * HM; ++k)
        if (k <= 2 * H) { S.qr[k] = acc[2 * (k - 1)] * iw; S.qi[k] = acc[2 * (k - 1) + 1] * iw; }
#pragma unroll
    for (int k = 1; k <= HM; ++k)
        if (k <= H) { S.pr[k] = acc[4 * HM + 2 * (k - 1)] * sq; S.pi[k] = acc[4 * HM + 2 * (k - 1) + 1] * sq; }
}

// Peak candidates ordered by (value desc, index asc).
// Candidates for arg-max / top-K searches carry an integer sort key instead of
// the value: comparisons then run on the integer pipes (double compares are
// slow on this part).  okey() maps a double to an int64 with the same order
// (-0 just below +0, NaN below everything); KEY_NONE marks an empty slot.
constexpr int64_t KEY_NONE = INT64_MIN;
FC2_D int64_t okey(double v) {
    const int64_t b = __double_as_longlong(v);
    if ((b & 0x7fffffffffffffffll) > 0x7ff0000000000000ll) return KEY_NONE;  // NaN
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
FC2_D int64_t okey(float v) {
    const int32_t b = __float_as_int(v);
    if ((b & 0x7fffffff) > 0x7f800000) return KEY_NONE;
    return (int64_t)(b ^ ((b >> 31) & 0x7fffffff));
}
struct Cand { int64_t k; int64_t j; };
FC2_D bool better(int64_t k1, int64_t j1, int64_t k2, int64_t j2) {
    return k1 > k2 || (k1 == k2 && j1 < j2);
}
FC2_D void warp_best(int64_t& k, int64_t& j) {  // all lanes get the winner
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int64_t j2 = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(k2, j2, k, j)) { k = k2; j = j2; }
    }
}

}  // namespace fc2
