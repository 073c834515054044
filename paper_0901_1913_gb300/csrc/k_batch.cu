// k_batch.cu -- many independent light curves through one launch per stage.
//
// The "many sources" case of Sec. 4: each curve is its own Fchi2 search (its own
// moments, H, trial grid), but all curves of a chunk share the grid length M, so
// every stage covers the whole chunk in one launch: transforms are indexed by a
// slot table (curve, multiple k, P or Q), curves by a curve table.  The spread
// and FFT kernels are the single-curve ones driven by those tables; the kernels
// here are the batch forms of the per-frequency solve, the exact fix-up and the
// peak search.  Output Delta chi^2 is float, packed curve after curve.
#include <cuda_runtime.h>

#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <tuple>
#include <type_traits>
#include <vector>

#include "fc2_common.cuh"
#include "fc2_df.cuh"
#include "fc2_internal.h"
#include "fc2_solve.cuh"

namespace fc2 {

// Per-curve constants (device arrays) used by the kernels below.
struct CurveTab {
    const int64_t* off;     // [C+1] sample offsets (chunk-local)
    const int* H;           // [C]
    const double* fmin;     // [C]
    const double* df;       // [C]
    const double* scal;     // [C][SC_COUNT]
    const int* slot0;       // [C] first transform slot of the curve
    const int64_t* out_off; // [C] first output element of the curve
    const float* sq;        // [C] 1/W
    const float* sp;        // [C] 1/sqrt(W chi2_0)
    const float* s1n;       // [C] sum w(x - xbar) / sqrt(W chi2_0)
    const float* chi0f;     // [C] chi2_0
    const int* qown;        // [C] curve whose Q transforms (weights only) this curve reads
    const int* pslot0;      // [C] first P transform slot of the curve
    int bx_ch;              // samples per exact-sum work item
};

// ------------------------------------------------------------------ gather
// Sample i of the chunk: its curve by binary search of the offsets; perm (if
// given) is a chunk-level permutation that sorts every curve by time.
__global__ void k_bgather(const double* __restrict__ t, const double* __restrict__ x,
                          const double* __restrict__ sg, const int32_t* __restrict__ perm,
                          int64_t ntot, const int64_t* __restrict__ off, int C,
                          const double* __restrict__ scal, const double* __restrict__ fmin,
                          const double* __restrict__ df, double* __restrict__ tau,
                          double* __restrict__ wq, double* __restrict__ wp,
                          uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                          float* __restrict__ wq32, float* __restrict__ wp32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int lo = 0, hi = C;  // largest c with off[c] <= i
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    const int c = lo;
    const int64_t src = perm ? perm[i] : i;
    const double* sc = scal + (int64_t)c * SC_COUNT;
    const double si = sg[src];
    const double w = 1.0 / (si * si);
    const double ta = __dsub_rn(t[src], sc[SC_T0]);
    const double v = __dmul_rn(w, __dsub_rn(x[src], sc[SC_XBAR]));
    tau[i] = ta;
    wq[i] = w;
    wp[i] = v;
    A[i] = frac_fx(fmin[c], ta);
    B[i] = frac_fx(df[c], ta);
    const float qh = (float)w, ph = (float)v;
    wq32[i] = qh;
    wp32[i] = ph;
    wq32[ntot + i] = (float)(w - (double)qh);  // low parts for double-float sums
    wp32[ntot + i] = (float)(v - (double)ph);
}

// ----------------------------------------------------------- phase reduction
// As the single-curve k_phase, per slot: the slot's curve, multiple k and
// kind select the samples and the strengths.  The band-centre modulation
// e^{2 pi i k f_c tau}, f_c = f_min + (N/2) df, has the exact fixed-point
// phase k (A + (N/2) B) mod 2^64 (A, B the sample's phases of f_min and df);
// in the float path its phasor comes from the double-float tables on the
// float pipes (well below float rounding), in the double path from sincospi.
template <typename T>
__global__ void k_bphase(const double* __restrict__ tau, const double* __restrict__ wq,
                         const double* __restrict__ wp, const uint64_t* __restrict__ Aph,
                         const uint64_t* __restrict__ Bph, const dfc* __restrict__ dftab,
                         const int64_t* __restrict__ off,
                         const double* __restrict__ fmin, const double* __restrict__ df,
                         int64_t N, int64_t M, int w, const int* __restrict__ slot_cur,
                         const int* __restrict__ slot_k, const int* __restrict__ slot_kind,
                         const int64_t* __restrict__ slot_soff, int32_t* __restrict__ key,
                         T* __restrict__ dlt, cpx<T>* __restrict__ cs) {
    const int g = blockIdx.y;
    const int c = slot_cur[g];
    const int64_t a = off[c], n = off[c + 1] - a;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int k = slot_k[g], kind = slot_kind[g];
    double sn, cn;
    int64_t fl;
    T de;
    if constexpr (sizeof(T) == 4) {
        // the cell position from the exact fixed-point phase B = frac(df tau) 2^64:
        // X - w/2 = M frac(k df tau) - w/2 in fixed point with 63 - log2 M
        // fraction bits (integer arithmetic, no double instruction)
        const uint64_t kk = (uint64_t)k;
        const uint64_t kb = kk * Bph[a + s];  // frac(k df tau) 2^64
        const int fb = 63 - (63 - __clzll((long long)M));
        const int64_t xs = (int64_t)(kb >> 1) - ((int64_t)w << (fb - 1));
        fl = xs >> fb;  // floor
        const uint64_t fr = (uint64_t)xs & ((1ull << fb) - 1);
        de = __fmul_rn(__ull2float_rn(fr), __int_as_float((127 - fb) << 23));  // fr 2^-fb
        const uint64_t th = kk * Aph[a + s] + (uint64_t)(N / 2) * kb;
        const dfc z = df_phasor(th, dftab, dftab + 256);
        cn = (double)z.re.h + (double)z.re.l;
        sn = (double)z.im.h + (double)z.im.l;
    } else {
        const double ts = tau[a + s];
        const double cc = __dmul_rn((double)k, df[c]);
        const double p = __dmul_rn(cc, ts);
        const double u = __dsub_rn(p, floor(p));
        const double X = __dmul_rn((double)M, u);
        const double Xs = __dsub_rn(X, 0.5 * (double)w);
        const double flo = floor(Xs);
        fl = (int64_t)flo;
        de = (T)__dsub_rn(Xs, flo);
        const double q1 = __dmul_rn(__dmul_rn((double)k, fmin[c]), ts);
        const double q2 = __dmul_rn((double)(N / 2), u);
        const double th = __dadd_rn(__dsub_rn(q1, floor(q1)), __dsub_rn(q2, floor(q2)));
        sincospi(2.0 * th, &sn, &cn);
    }
    const double amp = kind == 0 ? wq[a + s] : wp[a + s];
    const int64_t o = slot_soff[g] + s;
    key[o] = (int32_t)fl + 1;
    dlt[o] = de;
    cs[o] = mk<T>((T)(amp * cn), (T)(amp * sn));
}

// --------------------------------------------------------------- assemble
// One thread per (trial frequency, curve) for the curves of one H; Delta
// chi^2 written as float.  Bins whose estimated error is too large go to
// `list` as (curve << 32 | j).
template <typename TS, int H, int NT>
__global__ void __launch_bounds__(NT) k_bassemble(const cpx<TS>* __restrict__ spec,
                                                   const TS* __restrict__ dec, int64_t N,
                                                   const int* __restrict__ curves, CurveTab ct,
                                                   TS tau, TS eps, TS err_fix,
                                                   float* __restrict__ out,
                                                   int64_t* __restrict__ list,
                                                   int32_t* __restrict__ list_count,
                                                   int64_t cap) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int c = curves[blockIdx.y];
    const int qo = ct.qown[c];
    const int gq = ct.slot0[qo], gp = ct.pslot0[c];
    const TS d = dec[j];
    const TS dq = d * (TS)ct.sq[qo], dp = d * (TS)ct.sp[c];
    Sys<TS, H> S;
    S.qr[0] = (TS)1;
    S.qi[0] = (TS)0;
    S.pr[0] = (TS)ct.s1n[c];
    S.pi[0] = (TS)0;
#pragma unroll
    for (int k = 1; k <= 2 * H; ++k) {
        const cpx<TS> v = spec[(int64_t)(gq + k - 1) * N + j];
        S.qr[k] = v.x * dq;
        S.qi[k] = v.y * dq;
    }
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        const cpx<TS> v = spec[(int64_t)(gp + k - 1) * N + j];
        S.pr[k] = v.x * dp;
        S.pi[k] = v.y * dp;
    }
    TS o[H], an2 = (TS)0;
    chol_solve<TS, H, true>(S, tau, o, &an2);
    if (!(est_err<TS>(an2, 2 * H + 1, eps) <= err_fix)) {
        const int32_t pos = atomicAdd(list_count, 1);
        if (pos < cap) list[pos] = ((int64_t)c << 32) | j;
    }
    float* oc = out + ct.out_off[c];
    const float c0 = ct.chi0f[c];
#pragma unroll
    for (int h = 0; h < H; ++h) oc[(int64_t)h * N + j] = (float)o[h] * c0;
}

constexpr double BX_EPS_DF = 1.5e-12;  // relative precision of the tier-2 (double-float) sums
// relative pivot of the gridded equations below which an entry is taken as
// nearly singular and starts at the double tier
constexpr double BX_DMIN_T3 = 1e-7;

// Double re-solve of listed (curve, bin) entries of the float path.  Entries
// still too sensitive go on to the exact sums: to the float tier, straight to
// the double-float tier when the float sums could not settle them either
// (error estimate at the float sums' precision above the bar, or a small
// relative pivot), or straight to the double tier when the coefficient norm
// is beyond the double-float sums as well or the pivot is below what the
// gridded equations resolve.
template <int HM>
__global__ void __launch_bounds__(128) k_bresolve(const cpx<float>* __restrict__ spec,
                                                  const float* __restrict__ dec, int64_t N,
                                                  CurveTab ct, double tau, double eps,
                                                  double err_fix, float* __restrict__ out,
                                                  const int64_t* __restrict__ rlist,
                                                  const int32_t* __restrict__ rcount,
                                                  int64_t rcap, int64_t* __restrict__ flist,
                                                  int32_t* __restrict__ fcount, int64_t fcap,
                                                  int64_t* __restrict__ flist2,
                                                  int32_t* __restrict__ fcount2, int64_t fcap2,
                                                  int64_t* __restrict__ flist3,
                                                  int32_t* __restrict__ fcount3, int64_t fcap3) {
    int64_t cnt = *rcount;
    if (cnt > rcap) cnt = rcap;
    const int64_t wpb = blockDim.x >> 5;  // one entry per warp (warp-cooperative solve)
    for (int64_t b = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); b < cnt;
         b += (int64_t)gridDim.x * wpb) {
        const int c = (int)(rlist[b] >> 32);
        const int64_t j = rlist[b] & 0xffffffffll;
        const int H = ct.H[c];
        const int qo = ct.qown[c];
        const int gq = ct.slot0[qo], gp = ct.pslot0[c];
        const double* sc = ct.scal + (int64_t)c * SC_COUNT;
        const double W = sc[SC_W], chi0 = sc[SC_CHI0];
        const double sp = (chi0 > 0.0) ? rsqrt(W * chi0) : 0.0;
        const double d = (double)dec[j];
        const double dw = d / ct.scal[(int64_t)qo * SC_COUNT + SC_W];
        Sys<double, HM> S;
#pragma unroll
        for (int k = 0; k <= 2 * HM; ++k) { S.qr[k] = 0.0; S.qi[k] = 0.0; }
#pragma unroll
        for (int k = 0; k <= HM; ++k) { S.pr[k] = 0.0; S.pi[k] = 0.0; }
        S.qr[0] = 1.0;
        S.pr[0] = sc[SC_S1] * sp;
        for (int k = 1; k <= 2 * H; ++k) {
            const cpx<float> v = spec[(int64_t)(gq + k - 1) * N + j];
            S.qr[k] = (double)v.x * dw;
            S.qi[k] = (double)v.y * dw;
        }
        for (int k = 1; k <= H; ++k) {
            const cpx<float> v = spec[(int64_t)(gp + k - 1) * N + j];
            S.pr[k] = (double)v.x * d * sp;
            S.pi[k] = (double)v.y * d * sp;
        }
        double o[HM], an2 = 0.0;
        const double dmin = warp_chol_solve<HM, true>(S, tau, o, &an2, H);
        if ((threadIdx.x & 31) == 0) {
            const int m = 2 * H + 1;
            if (!(est_err<double>(an2, m, eps) <= err_fix)) {
                if (!(est_err<double>(an2, m, BX_EPS_DF) <= err_fix) || dmin < BX_DMIN_T3) {
                    const int32_t pos = atomicAdd(fcount3, 1);
                    if (pos < fcap3) flist3[pos] = rlist[b];
                } else if (!(est_err<double>(an2, m, 2e-7 * sc[SC_RW]) <= err_fix) || dmin < 3e-3) {
                    const int32_t pos = atomicAdd(fcount2, 1);
                    if (pos < fcap2) flist2[pos] = rlist[b];
                } else {
                    const int32_t pos = atomicAdd(fcount, 1);
                    if (pos < fcap) flist[pos] = rlist[b];
                }
            }
            float* oc = out + ct.out_off[c];
            for (int h = 0; h < H; ++h) oc[(int64_t)h * N + j] = (float)(o[h] * chi0);
        }
    }
}

// ------------------------------------------------------------ exact sums
// Entries (curve << 32 | j).  Precision tiers of the sums over the exact
// integer phases (Sec. 3's moments, Eqs. for Q and P):
//   1: float sine / cosine, compensated float sums;
//   2: double-float phasors, products and sums (about 48 bits);
//   3: double phasors and sums.
// An entry's samples are cut into work items of about bx_ch samples (at most
// BX_QMAX per entry) so that the long curves of a batch spread over all SMs:
// k_bx_split numbers the items in entry order, k_bx_part sums each item with
// one warp (lanes at stride 32, then a butterfly) into a row of partial sums,
// and k_bexact adds an entry's rows in item order, solves and routes.  Entries
// beyond the item capacity are summed whole by k_bexact.  An entry's items and
// their summation order depend only on its curve, so its result does not
// depend on where the entry sits in the (atomically filled) list -- unless the
// list overflows the item capacity, when which entries are summed whole does.
// MODE 0 writes Delta chi^2 (float) and passes on to `next` the entries whose
// error estimate from the coefficient norm, or whose smallest relative pivot,
// is beyond what the tier's sums can vouch for.  MODE 1 writes coefficient
// records.  Weights: wq32 / wp32 hold the float high parts at [i] and the low
// parts at [ntot + i].
constexpr int BX_NT = 256;
constexpr int BX_W = BX_NT / 32;
constexpr int BX_CH = 2048;           // samples per work item by default (autotuned)
constexpr int BX_QMAX = 64;           // work items per entry at most
constexpr int BX_ITEMS = 1 << 18;     // work items per launch at most
constexpr int BX_SPLIT_NT = 1024;     // threads of the (single-CTA) item numbering

FC2_HD int bx_items_of(int64_t n, int ch) {
    const int64_t q = (n + ch - 1) / ch;
    return (int)(q < 1 ? 1 : (q > BX_QMAX ? BX_QMAX : q));
}

// The phasor tables of tiers 2 and 3, staged in shared memory by every CTA.
template <int TIER>
struct BxTables {
    dfc t2[(TIER == 2 || TIER == 4) ? 512 : 1];
    double2 t3[TIER == 3 ? 512 : 1];
    FC2_D void load(const dfc* __restrict__ dftab) {
        if constexpr (TIER == 2 || TIER == 4)
            for (int i = threadIdx.x; i < 512; i += blockDim.x) t2[i] = dftab[i];
        if constexpr (TIER == 3) {
            const double2* t64 = reinterpret_cast<const double2*>(dftab + 512);
            for (int i = threadIdx.x; i < 512; i += blockDim.x) t3[i] = t64[i];
        }
        __syncthreads();
    }
};

// Sums of samples [i0, i1) of one entry (bin ju, H harmonics) by one warp;
// every lane returns the same totals tot[6 HM]: Q_k (k = 1..2H) re/im at
// [2(k-1)], [2(k-1)+1], P_k (k = 1..H) at [4 HM + 2(k-1)], [4 HM + 2(k-1)+1].
template <int HM, int TIER>
FC2_D void bx_sums(const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
                   const float* __restrict__ wq32, const float* __restrict__ wp32,
                   const double* __restrict__ wq, const double* __restrict__ wp,
                   const BxTables<TIER>& tb, int64_t ntot, uint64_t ju, int H, int64_t i0,
                   int64_t i1, int lane, double* tot) {
    constexpr int NV = 6 * HM;
    if constexpr (TIER == 1) {
        CompSum<float> fa[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) fa[v].init();
        for (int64_t i = i0 + lane; i < i1; i += 32) {
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
            const float2 x = warp_allsum_pair(fa[v].s, fa[v].c);
            tot[v] = (double)x.x + (double)x.y;
        }
    } else if constexpr (TIER == 2) {
        dfl fa[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) fa[v] = dfl{0.f, 0.f};
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const uint64_t u = Aph[i] + ju * Bph[i];
            const dfl a{wq32[i], wq32[ntot + i]}, bb{wp32[i], wp32[ntot + i]};
            const dfc z1 = df_phasor(u, tb.t2, tb.t2 + 256);
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
            const float2 x = warp_allsum_pair(fa[v].h, fa[v].l);
            tot[v] = (double)x.x + (double)x.y;
        }
    } else if constexpr (TIER == 4) {
        // lph lanes per harmonic multiple k = 1..2H (lane = (k - 1) lph + r),
        // each over the samples i0 + r, + lph, ..; sums exact in fixed point
        const int lph = 32 / (2 * H);
        const int g = lane / lph, r = lane - g * lph;
        float mq = 0.f, mp = 0.f;  // the item's largest weights set the scales
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            mq = fmaxf(mq, fabsf(wq32[i]));
            mp = fmaxf(mp, fabsf(wp32[i]));
        }
        mq = warp_max_f(mq);
        mp = warp_max_f(mp);
        // a harmonic's terms over the item (|w e^{..}| <= |w| (1 + 2^-23))
        const int eq = fx_exponent(mq * 1.0000002f, i1 - i0 + 1);
        const int ep = fx_exponent(mp * 1.0000002f, i1 - i0 + 1);
        long long acc[4] = {0, 0, 0, 0};
        if (g < 2 * H)
            fx_lane_sums<false>(Aph, Bph, wq32, wp32, ntot, ju, (uint64_t)(g + 1), i0, i1, r, lph,
                                g < H, tb.t2, tb.t2 + 256, exp2f((float)eq), exp2f((float)ep), acc);
        // group sums, exact: the group's first lane adds its lanes' values in order
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long s = acc[q];
            for (int o = 1; o < lph; ++o) {
                const long long y = __shfl_sync(0xffffffffu, acc[q], (lane + o) & 31);
                if (r == 0) s += y;
            }
            acc[q] = s;
        }
        const double uq = ldexp(1.0, -eq), up = ldexp(1.0, -ep);
#pragma unroll
        for (int k = 0; k < 2 * HM; ++k) {
            const int src = (k < 2 * H) ? k * lph : 0;
            const double v0 = (double)__shfl_sync(0xffffffffu, acc[0], src) * uq;
            const double v1 = (double)__shfl_sync(0xffffffffu, acc[1], src) * uq;
            const double v2 = (double)__shfl_sync(0xffffffffu, acc[2], src) * up;
            const double v3 = (double)__shfl_sync(0xffffffffu, acc[3], src) * up;
            tot[2 * k] = (k < 2 * H) ? v0 : 0.0;
            tot[2 * k + 1] = (k < 2 * H) ? v1 : 0.0;
            if (k < HM) {
                tot[4 * HM + 2 * k] = (k < H) ? v2 : 0.0;
                tot[4 * HM + 2 * k + 1] = (k < H) ? v3 : 0.0;
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) tot[v] = 0.0;
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const double2 z1 = d_phasor(Aph[i] + ju * Bph[i], tb.t3, tb.t3 + 256);
            const double c1 = z1.x, s1 = z1.y;
            double cr = c1, ci = s1;
            const double a = wq[i], bb = wp[i];
#pragma unroll
            for (int k = 0; k < 2 * HM; ++k) {
                if (k < 2 * H) {
                    tot[2 * k] = fma(a, cr, tot[2 * k]);
                    tot[2 * k + 1] = fma(a, ci, tot[2 * k + 1]);
                    if (k < H) {
                        tot[4 * HM + 2 * k] = fma(bb, cr, tot[4 * HM + 2 * k]);
                        tot[4 * HM + 2 * k + 1] = fma(bb, ci, tot[4 * HM + 2 * k + 1]);
                    }
                    const double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                    cr = nr;
                    ci = ni;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot[v] += __shfl_xor_sync(0xffffffffu, tot[v], o);
        }
    }
}

// Work items of the listed entries, numbered in entry order by one CTA (each
// thread a run of entries, then a block scan): qbase[e] = first item of entry
// e (items qbase[e] .. + bx_items_of(n) - 1), or -1 when the entry is summed
// whole (an empty peak slot, or past the item capacity; the entries that fit
// form a prefix); items[w] = e * BX_QMAX + q; *nitems = items placed.
__global__ void __launch_bounds__(BX_SPLIT_NT) k_bx_split(CurveTab ct,
                                                          const int64_t* __restrict__ list,
                                                          const int32_t* __restrict__ count,
                                                          int64_t cap, int32_t* __restrict__ qbase,
                                                          int32_t* __restrict__ items,
                                                          int32_t* __restrict__ nitems) {
    __shared__ int32_t wsum[BX_SPLIT_NT / 32];
    __shared__ int32_t placed;
    int64_t cnt = *count;
    if (cnt > cap) cnt = cap;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) placed = 0;
    const int64_t per = (cnt + BX_SPLIT_NT - 1) / BX_SPLIT_NT;
    const int64_t e0 = (int64_t)tid * per;
    const int64_t e1 = (e0 + per < cnt) ? e0 + per : cnt;
    auto items_of = [&](int64_t e) -> int {
        const int64_t ent = list[e];
        if ((ent & 0xffffffffll) == 0xffffffffll) return 0;  // empty peak slot
        const int c = (int)(ent >> 32);
        return bx_items_of(ct.off[c + 1] - ct.off[c], ct.bx_ch);
    };
    // item counts: at most (2^22 entries) x BX_QMAX in all, so int32 sums are exact
    int32_t v = 0;
    for (int64_t e = e0; e < e1; ++e) v += items_of(e);
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t x = lane < BX_SPLIT_NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < BX_SPLIT_NT / 32) wsum[lane] = x;
    }
    __syncthreads();
    // entries in order: those whose items fit below the capacity form a prefix
    int32_t base = (w > 0 ? wsum[w - 1] : 0) + (incl - v);
    int32_t end = 0;
    for (int64_t e = e0; e < e1; ++e) {
        const int nq = items_of(e);
        if (nq > 0 && base + nq <= BX_ITEMS) {
            qbase[e] = base;
            for (int q = 0; q < nq; ++q) items[base + q] = (int32_t)(e * BX_QMAX + q);
            end = base + nq;
        } else {
            qbase[e] = -1;
        }
        base += nq;
    }
    atomicMax(&placed, end);
    __syncthreads();
    if (tid == 0) *nitems = placed;
}

// One warp per work item: the item's share of its entry's samples, summed
// into row w of part (6 BHM doubles per row).
template <int HM, int TIER>
__global__ void __launch_bounds__(BX_NT) k_bx_part(
    const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
    const float* __restrict__ wq32, const float* __restrict__ wp32,
    const double* __restrict__ wq, const double* __restrict__ wp, const dfc* __restrict__ dftab,
    int64_t ntot, CurveTab ct, const int64_t* __restrict__ list,
    const int32_t* __restrict__ items, const int32_t* __restrict__ nitems,
    double* __restrict__ part) {
    constexpr int NV = 6 * HM;
    __shared__ BxTables<TIER> tb;
    tb.load(dftab);
    const int nw = *nitems;
    const int lane = threadIdx.x & 31;
    for (int w = blockIdx.x * BX_W + (threadIdx.x >> 5); w < nw; w += gridDim.x * BX_W) {
        const int it = items[w];
        const int64_t e = it / BX_QMAX;
        const int q = it % BX_QMAX;
        const int64_t ent = list[e];
        const int c = (int)(ent >> 32);
        const uint64_t ju = (uint64_t)(ent & 0xffffffffll);
        const int64_t a0 = ct.off[c], n = ct.off[c + 1] - a0;
        const int nq = bx_items_of(n, ct.bx_ch);
        const int64_t i0 = a0 + n * q / nq, i1 = a0 + n * (q + 1) / nq;
        double tot[NV];
        bx_sums<HM, TIER>(Aph, Bph, wq32, wp32, wq, wp, tb, ntot, ju, ct.H[c], i0, i1, lane, tot);
        double* row = part + (int64_t)w * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if ((v & 31) == lane) row[v] = tot[v];
    }
}

// Entry totals in every lane: the entry's partial rows added in item order
// (lanes own values v = lane, lane + 32), or the whole sum when it has none.
template <int HM, int TIER, int MODE>
__global__ void __launch_bounds__(BX_NT) k_bexact(
    const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
    const float* __restrict__ wq32, const float* __restrict__ wp32,
    const double* __restrict__ wq, const double* __restrict__ wp, const dfc* __restrict__ dftab,
    int64_t ntot, CurveTab ct, int64_t N, const int64_t* __restrict__ list,
    const int32_t* __restrict__ count, int64_t cap, const int32_t* __restrict__ qbase,
    const double* __restrict__ part, double tau_drop, double err_fix, float* __restrict__ out,
    int64_t* __restrict__ next, int32_t* __restrict__ next_count, int64_t next_cap,
    fc2_best* __restrict__ recs) {
    constexpr int NV = 6 * HM;
    static_assert(NV <= 64, "two values per lane");
    __shared__ BxTables<TIER> tb;
    tb.load(dftab);
    int64_t cnt = *count;
    if (cnt > cap) cnt = cap;
    const int lane = threadIdx.x & 31;
    for (int64_t e = (int64_t)blockIdx.x * BX_W + (threadIdx.x >> 5); e < cnt;
         e += (int64_t)gridDim.x * BX_W) {
        const int64_t ent = list[e];
        const int c = (int)(ent >> 32);
        const int64_t j = ent & 0xffffffffll;
        const int H = ct.H[c];
        if (MODE == 1 && j == 0xffffffffll) {  // empty peak slot
            if (lane == 0) {
                fc2_best b;
                b.j = -1; b.f = 0; b.dchi2 = 0; b.H = H; b.flags = 0;
                for (int l = 0; l < 2 * FC2_MAX_H + 1; ++l) b.A[l] = 0.0;
                recs[e] = b;
            }
            continue;
        }
        const int64_t a0 = ct.off[c], a1 = ct.off[c + 1];
        double tot[NV];
        const int qb = qbase[e];
        if (qb >= 0) {
            const int nq = bx_items_of(a1 - a0, ct.bx_ch);
            double lo = 0.0, hi = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double* row = part + (int64_t)(qb + q) * NV;
                lo += row[lane];
                if (lane + 32 < NV) hi += row[lane + 32];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v)
                tot[v] = __shfl_sync(0xffffffffu, v < 32 ? lo : hi, v & 31);
        } else {
            bx_sums<HM, TIER>(Aph, Bph, wq32, wp32, wq, wp, tb, ntot, (uint64_t)j, H, a0, a1,
                              lane, tot);
        }
        const double* sc = ct.scal + (int64_t)c * SC_COUNT;
        Sys<double, HM> S;
        exact_sys_from_sums<HM>(tot, H, sc, S);
        const double chi0 = sc[SC_CHI0];
        if constexpr (MODE == 0) {
            double o[HM], an2 = 0.0;
            const double dmin = warp_chol_solve<HM, true>(S, tau_drop, o, &an2, H);
            const double eps = TIER == 1 ? 2e-7 * sc[SC_RW] : (TIER == 2 ? BX_EPS_DF : 1e-14);
            // sums cannot vouch for a pivot near their precision (their errors
            // can also make the coefficients look small): such entries go on
            if (lane == 0) {
                if (next && (!(est_err<double>(an2, 2 * H + 1, eps) <= err_fix) ||
                             dmin < 1e3 * eps)) {
                    const int32_t pos = atomicAdd(next_count, 1);
                    if (pos < next_cap) next[pos] = ent;
                }
                float* oc = out + ct.out_off[c];
                for (int h = 0; h < H; ++h) oc[(int64_t)h * N + j] = (float)(o[h] * chi0);
            }
        } else {
            double o[HM], an2;
            double A[2 * HM + 1];
            warp_chol_solve<HM, false>(S, tau_drop, o, &an2, H, A, H);
            if (lane == 0) {
                const double W = sc[SC_W];
                const double unit = (W > 0.0) ? sqrt(chi0 / W) : 0.0;
                const double f = ct.fmin[c] + (double)j * ct.df[c];
                fc2_best b;
                b.j = j; b.f = f; b.dchi2 = o[H - 1] * chi0; b.H = H; b.flags = 0;
                for (int l = 0; l < 2 * FC2_MAX_H + 1; ++l) b.A[l] = 0.0;
                b.A[0] = A[0] * unit + sc[SC_XBAR];
                const double fT0 = f * sc[SC_T0];
                for (int h = 1; h <= H; ++h) {
                    const double ph = (double)h * (fT0 - floor(fT0));
                    double sn, cn;
                    sincospi(2.0 * (ph - floor(ph)), &sn, &cn);
                    const double as = A[2 * h - 1] * unit, ac = A[2 * h] * unit;
                    b.A[2 * h - 1] = as * cn + ac * sn;
                    b.A[2 * h] = ac * cn - as * sn;
                }
                recs[e] = b;
            }
        }
    }
}

// ------------------------------------------------------------------- peaks
// Per curve: top-K local maxima of its Delta chi^2_H row (value > left,
// >= right; edges one-sided), ordered by (value desc, j asc).  A threshold
// first: every block of BP_B bins finds its best local maximum, and the K-th
// best of those over the curve's blocks, theta, bounds the K-th best local
// maximum from below (the K blocks whose best reaches theta hold K local maxima
// at least as large).  Then only the blocks whose best reaches theta rank their
// local maxima >= theta (the rest write empty lists), and one block per curve
// merges the lists.  Writes the peak list as (curve << 32 | j) entries, empty
// slots as (curve << 32 | 0xffffffff).
constexpr int BP_NT = 256;
constexpr int BP_PER = 16;
constexpr int BP_B = BP_NT * BP_PER;
constexpr int BP_NW = BP_NT / 32;
constexpr int BP_KMAX = 64;

// Local maxima of the block's bins held by this thread (key, bin), empty as
// (KEY_NONE, INT64_MAX).
FC2_D void bp_local_maxima(const float* __restrict__ row, int64_t N, int64_t base, int lane, int w,
                           int64_t* cv, int64_t* cj) {
#pragma unroll
    for (int q = 0; q < BP_PER; ++q) {
        const int64_t jj = base + lane + (int64_t)(w * BP_PER + q) * 32;
        cv[q] = KEY_NONE;
        cj[q] = INT64_MAX;
        if (jj < N) {
            const int64_t x = okey(row[jj]);
            const bool left = (jj == 0) || (x > okey(row[jj - 1]));
            const bool right = (jj == N - 1) || (x >= okey(row[jj + 1]));
            if (left && right) { cv[q] = x; cj[q] = jj; }
        }
    }
}

// Each block's best local maximum.
__global__ void __launch_bounds__(BP_NT) k_bpeaks0(const float* __restrict__ out, int64_t N,
                                                   CurveTab ct, int nblk,
                                                   Cand* __restrict__ bbest) {
    __shared__ Cand wb[BP_NW];
    const int c = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float* row = out + ct.out_off[c] + (int64_t)(ct.H[c] - 1) * N;
    // 32-bit order keys (okey's order for floats); neighbours from the adjacent
    // lanes, the run's ends from memory; the running best in (value desc, j asc)
    auto key32 = [](float f) -> int32_t {
        const int32_t b = __float_as_int(f);
        if ((b & 0x7fffffff) > 0x7f800000) return INT32_MIN;  // NaN: below everything
        return b ^ ((b >> 31) & 0x7fffffff);
    };
    int32_t bv = INT32_MIN;
    int64_t bj = INT64_MAX;
    const int64_t base = (int64_t)blockIdx.x * BP_B;
#pragma unroll 4
    for (int q = 0; q < BP_PER; ++q) {
        const int64_t j0 = base + (int64_t)(w * BP_PER + q) * 32;  // the warp's 32 bins
        const int64_t jj = j0 + lane;
        const int32_t x = jj < N ? key32(row[jj]) : INT32_MIN;
        int32_t xl = __shfl_up_sync(0xffffffffu, x, 1);
        int32_t xr = __shfl_down_sync(0xffffffffu, x, 1);
        if (lane == 0 && jj > 0 && jj - 1 < N) xl = key32(row[jj - 1]);
        if (lane == 31 && jj + 1 < N) xr = key32(row[jj + 1]);
        const bool left = (jj == 0) || (x > xl);
        const bool right = (jj == N - 1) || (x >= xr);
        if (jj < N && left && right && (x > bv || (x == bv && jj < bj))) {
            bv = x;
            bj = jj;
        }
    }
    int64_t v = (bv == INT32_MIN) ? KEY_NONE : (int64_t)bv, j = bj;
    warp_best(v, j);
    if (lane == 0) wb[w] = Cand{v, j};
    __syncthreads();
    if (w == 0) {
        v = lane < BP_NW ? wb[lane].k : KEY_NONE;
        j = lane < BP_NW ? wb[lane].j : INT64_MAX;
        warp_best(v, j);
        if (lane == 0) bbest[(int64_t)c * nblk + blockIdx.x] = Cand{v, j};
    }
}

// theta[c]: the K-th best of curve c's block maxima, KEY_NONE when fewer than
// K blocks have a local maximum (one 256-thread block per curve).
__global__ void __launch_bounds__(256) k_bpeaks_theta(const Cand* __restrict__ bbest, int nblk,
                                                      int K, int64_t* __restrict__ theta) {
    __shared__ Cand ws[8];
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Cand* bc = bbest + (int64_t)c * nblk;
    int64_t pv = INT64_MAX, pj = -1, th = KEY_NONE;
    for (int r = 0; r < K; ++r) {
        int64_t v = KEY_NONE, j = INT64_MAX;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            const Cand cd = bc[b];
            if (cd.j != INT64_MAX && better(pv, pj, cd.k, cd.j) && better(cd.k, cd.j, v, j)) {
                v = cd.k;
                j = cd.j;
            }
        }
        warp_best(v, j);
        if (lane == 0) ws[w] = Cand{v, j};
        __syncthreads();
        v = lane < 8 ? ws[lane].k : KEY_NONE;
        j = lane < 8 ? ws[lane].j : INT64_MAX;
        warp_best(v, j);  // every warp: the round's winner
        __syncthreads();  // ws is rewritten by the next round
        if (j == INT64_MAX) {  // fewer than K blocks with a local maximum
            th = KEY_NONE;
            break;
        }
        th = v;
        pv = v;
        pj = j;
    }
    if (threadIdx.x == 0) theta[c] = th;
}

// The top-K local maxima >= theta of the blocks whose best reaches theta.
__global__ void __launch_bounds__(BP_NT) k_bpeaks1(const float* __restrict__ out, int64_t N,
                                                   CurveTab ct, int K, int nblk,
                                                   const Cand* __restrict__ bbest,
                                                   const int64_t* __restrict__ theta,
                                                   Cand* __restrict__ tops) {
    __shared__ Cand wtop[BP_NW][BP_KMAX];
    const int c = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t th = theta[c];
    const Cand bb = bbest[(int64_t)c * nblk + blockIdx.x];
    Cand* tb = tops + ((int64_t)c * nblk + blockIdx.x) * K;
    if (bb.j == INT64_MAX || bb.k < th) {
        for (int r = threadIdx.x; r < K; r += blockDim.x) tb[r] = Cand{KEY_NONE, INT64_MAX};
        return;
    }
    const float* row = out + ct.out_off[c] + (int64_t)(ct.H[c] - 1) * N;
    int64_t cv[BP_PER], cj[BP_PER];
    bp_local_maxima(row, N, (int64_t)blockIdx.x * BP_B, lane, w, cv, cj);
#pragma unroll
    for (int q = 0; q < BP_PER; ++q)
        if (cv[q] < th) { cv[q] = KEY_NONE; cj[q] = INT64_MAX; }
    for (int r = 0; r < K; ++r) {
        int64_t v = KEY_NONE, j = INT64_MAX;
#pragma unroll
        for (int q = 0; q < BP_PER; ++q)
            if (better(cv[q], cj[q], v, j)) { v = cv[q]; j = cj[q]; }
        warp_best(v, j);
#pragma unroll
        for (int q = 0; q < BP_PER; ++q)
            if (cj[q] == j) { cv[q] = KEY_NONE; cj[q] = INT64_MAX; }
        if (lane == 0) wtop[w][r] = Cand{v, j};
    }
    __syncthreads();
    if (w == 0) {
        // merge the warps' sorted lists by their heads
        int head = 0;
        for (int r = 0; r < K; ++r) {
            int64_t v = KEY_NONE, j = INT64_MAX;
            if (lane < BP_NW && head < K) { v = wtop[lane][head].k; j = wtop[lane][head].j; }
            const int64_t mj = j;
            warp_best(v, j);
            if (lane < BP_NW && mj == j && j != INT64_MAX) ++head;
            if (lane == 0) tb[r] = Cand{v, j};
        }
    }
}

__global__ void __launch_bounds__(256) k_bpeaks2(const Cand* __restrict__ tops, int nblk, int K,
                                                 int64_t* __restrict__ peak_ent) {
    __shared__ Cand ws[8];
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Cand* tc = tops + (int64_t)c * nblk * K;
    const int64_t total = (int64_t)nblk * K;
    int64_t pv = INT64_MAX, pj = -1;
    for (int r = 0; r < K; ++r) {
        int64_t v = KEY_NONE, j = INT64_MAX;
        for (int64_t b = threadIdx.x; b < total; b += blockDim.x) {
            const Cand cd = tc[b];
            if (cd.j != INT64_MAX && better(pv, pj, cd.k, cd.j) && better(cd.k, cd.j, v, j)) {
                v = cd.k;
                j = cd.j;
            }
        }
        warp_best(v, j);
        if (lane == 0) ws[w] = Cand{v, j};
        __syncthreads();
        if (w == 0) {
            v = lane < 8 ? ws[lane].k : KEY_NONE;
            j = lane < 8 ? ws[lane].j : INT64_MAX;
            warp_best(v, j);
            if (lane == 0) {
                ws[0] = Cand{v, j};
                peak_ent[(int64_t)c * K + r] =
                    ((int64_t)c << 32) | (j == INT64_MAX ? 0xffffffffll : j);
            }
        }
        __syncthreads();
        pv = ws[0].k;
        pj = ws[0].j;
        __syncthreads();
        if (pj == INT64_MAX) pv = KEY_NONE;
    }
}

// ============================================================ host driver
namespace {

template <typename P>
cudaError_t need(P** ptr, size_t* cap, size_t n, cudaStream_t s) {
    if (n <= *cap && *ptr) return cudaSuccess;
    if (*ptr) cudaFreeAsync(*ptr, s);
    *ptr = nullptr;
    *cap = 0;
    n = std::max<size_t>(n, 64);
    cudaError_t e = pool_alloc((void**)ptr, n * sizeof(P), s);
    if (e == cudaSuccess) *cap = n;
    return e;
}

template <typename P>
void release(P*& ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync((void*)ptr, s);
    ptr = nullptr;
}

__global__ void k_iota_plus(int32_t* v, int64_t n, int64_t base) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)(base + i);
}
__global__ void k_add_base(int32_t* v, int64_t n, int64_t base) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] += (int32_t)base;
}

fc2_status map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return FC2_OK;
    if (e == cudaErrorMemoryAllocation) return FC2_ERR_OOM;
    return FC2_ERR_CUDA;
}

constexpr int BHM = 8;  // harmonic capacity of the batched kernels

}  // namespace

// Pinned host buffers of the batched calls (the chunk tables' staging and the
// mapped moments), kept for the process: pinning host memory costs
// milliseconds per call on this platform.  A call takes a free pair large
// enough or allocates one, and returns it at the end; concurrent calls get
// different pairs.
struct PinnedPair {
    char* stage = nullptr;
    size_t stage_bytes = 0;
    char* map = nullptr;
    size_t map_bytes = 0;
};
static std::mutex g_pin_mu;
static std::vector<PinnedPair> g_pin_free;

static bool pinned_acquire(size_t stage_bytes, size_t map_bytes, PinnedPair* out) {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_pin_free.size(); ++i)
            if (g_pin_free[i].stage_bytes >= stage_bytes && g_pin_free[i].map_bytes >= map_bytes) {
                *out = g_pin_free[i];
                g_pin_free.erase(g_pin_free.begin() + (long)i);
                return true;
            }
    }
    PinnedPair p;
    p.stage_bytes = stage_bytes;
    p.map_bytes = map_bytes;
    if (cudaHostAlloc((void**)&p.stage, stage_bytes, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaHostAlloc((void**)&p.map, map_bytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(p.stage);
        return false;
    }
    *out = p;
    return true;
}

static void pinned_release(const PinnedPair& p) {
    if (!p.stage && !p.map) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
    // keep a few pairs; free the smallest beyond that
    while (g_pin_free.size() > 4) {
        size_t k = 0;
        for (size_t i = 1; i < g_pin_free.size(); ++i)
            if (g_pin_free[i].stage_bytes + g_pin_free[i].map_bytes <
                g_pin_free[k].stage_bytes + g_pin_free[k].map_bytes)
                k = i;
        cudaFreeHost(g_pin_free[k].stage);
        cudaFreeHost(g_pin_free[k].map);
        g_pin_free.erase(g_pin_free.begin() + (long)k);
    }
}

// The launch configuration of a chunk: the transform plan and family, the
// spreading tile, the assembly block and the exact-sum work item.
struct BatchConfig {
    FftChoice fft;
    int spread_tile;
    int asm_nt;
    int bx_ch;
    int fft_group = 0;  // grids taken through both passes at a time (0 = all)
};

struct Batch {
    cudaStream_t s = nullptr;
    bool own_stream = false;
    // chunk plan: drives the shared spread / FFT launchers
    fc2_plan_s cp;
    // device arrays with capacities
    double *t = nullptr, *x = nullptr, *sg = nullptr;
    size_t ct = 0, cx = 0, csg = 0;
    int32_t* perm = nullptr; size_t cperm = 0;
    double *tau = nullptr, *wq = nullptr, *wp = nullptr; size_t ctau = 0, cwq = 0, cwp = 0;
    uint64_t *A = nullptr, *B = nullptr; size_t cA = 0, cB = 0;
    float *wq32 = nullptr, *wp32 = nullptr; size_t cwq32 = 0, cwp32 = 0;
    int64_t* off = nullptr; size_t coff = 0;
    int* H = nullptr; size_t cH = 0;
    int* slot0 = nullptr; size_t cslot0 = 0;
    int *qown = nullptr, *pslot0 = nullptr; size_t cqown = 0, cpslot0 = 0;
    double *fmin = nullptr, *df = nullptr, *scal = nullptr; size_t cfmin = 0, cdf = 0, cscal = 0;
    int64_t* out_off = nullptr; size_t coo = 0;
    float *sq = nullptr, *sp = nullptr, *s1n = nullptr, *chi0f = nullptr;
    size_t csq = 0, csp = 0, cs1n = 0, cchi0f = 0;
    int *slot_cur = nullptr, *slot_k = nullptr, *slot_kind = nullptr;
    size_t cscur = 0, csk = 0, cskind = 0;
    int64_t *slot_soff = nullptr, *slot_n = nullptr, *L = nullptr;
    size_t cssoff = 0, csn = 0, cL = 0;
    int32_t* key = nullptr; size_t ckey = 0;
    char *dlt = nullptr, *cs = nullptr; size_t cdlt = 0, ccs = 0;
    char *grid0 = nullptr, *grid1 = nullptr, *spec = nullptr; size_t cg0 = 0, cg1 = 0, cspec = 0;
    float* out = nullptr; size_t cout = 0;
    float* out2 = nullptr; size_t cout2 = 0;  // second host-bound output buffer
    int64_t *list = nullptr, *list2 = nullptr, *list3 = nullptr, *list4 = nullptr;
    size_t cl1 = 0, cl2 = 0, cl3 = 0, cl4 = 0;
    char* dftab = nullptr; size_t cdftab = 0;  // phasor tables of the exact sums
    int32_t *qbase = nullptr, *items = nullptr; size_t cqbase = 0, citems = 0;  // exact-sum work items
    double* part = nullptr; size_t cpart = 0;  // their partial sums
    int32_t* counts = nullptr; size_t ccnt = 0;
    int* curves = nullptr; size_t ccurves = 0;
    Cand* tops = nullptr; size_t ctops = 0;
    Cand* bbest = nullptr; size_t cbbest = 0;  // best local maximum of each peak block
    int64_t* theta = nullptr; size_t ctheta = 0;  // per curve: the peak threshold
    int64_t* pent = nullptr; size_t cpent = 0;
    fc2_best* recs = nullptr; size_t crecs = 0;  // every curve's peak records [C][K]
    fc2_best* recs_now = nullptr;  // the records of the chunk being launched
    int32_t* cnt_hist = nullptr; size_t chist = 0;  // every chunk's counters, [chunk][16]
    // mapped host memory for the per-chunk moments and status word
    char* hmap = nullptr;
    char* hmap_dev = nullptr;
    // copy-out overlap: the host copies of chunk i run on their own stream while
    // chunk i + 1 computes; chunks alternate between two output buffers, and a
    // chunk waits for the copies of the chunk two before it (same buffers)
    cudaStream_t cs2 = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    bool copied_pending[2] = {false, false};
    char* red = nullptr; size_t cred = 0;
    // two executable graphs used by alternate chunks: a chunk's graph is updated
    // only once the launch of the chunk two before it (same executable) is done
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaEvent_t ev_graph[2] = {nullptr, nullptr};
    bool graph_pending[2] = {false, false};
    // the chunk being launched: its slices of the device inputs
    const double *tc = nullptr, *xc = nullptr, *sgc = nullptr;
    // every curve's moments (one launch for the whole call) and its offsets
    double* scal_all = nullptr; size_t cscal_all = 0;
    int64_t* goff = nullptr; size_t cgoff = 0;
    // pinned staging of the chunk tables, two halves used by alternate chunks
    // (a half is refilled once the copies of the chunk two before are done)
    PinnedPair pins;  // the staging and mapped buffers (returned to the cache at the end)
    char* stage = nullptr;
    size_t stage_half = 0;
    cudaEvent_t ev_tab[2] = {nullptr, nullptr};
    bool tab_pending[2] = {false, false};
    int64_t graphs = 0;  // chunk graphs launched
    // tuned launch parameters (besides the transform plan in cp): threads per
    // assembly block and samples per exact-sum work item
    int asm_nt = 128;
    int bx_ch = BX_CH;
    // the configuration of the last chunk, its source (0 fixed, 1 tuning table,
    // 2 tuned in this call), the tuning time and the configurations timed
    BatchConfig cfg{FftChoice{std::vector<int>(), 0}, 0, 0, 0};
    int cfg_source = 0;
    double tune_ms = 0;
    int tune_timed = 0;
    int64_t launches = 0;
    int64_t stats[4] = {0, 0, 0, 0};
    double phase_ms[7] = {0, 0, 0, 0, 0, 0, 0};  // host wall time of the call's phases
    // stage timing (fc2_debug_batch_timing): events recorded on the stream between
    // the stages of every chunk (captured into the chunk's graph), device ms per
    // stage summed over the chunks, and the transforms' algorithmic bytes (the
    // kept spectra written: 3 H_c N_c complex values per curve)
    bool double_last = false;  // mixed path: double sums as the last fix-up tier (diagnostics)
    bool timing = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double stage_ms[5] = {0, 0, 0, 0, 0};
    double fft_alg_bytes = 0;

    void free_all() {
        release(t, s); release(x, s); release(sg, s); release(perm, s); release(tau, s);
        release(wq, s); release(wp, s); release(A, s); release(B, s); release(wq32, s);
        release(wp32, s); release(off, s); release(H, s); release(slot0, s); release(fmin, s);
        release(qown, s); release(pslot0, s);
        release(df, s); release(scal, s); release(out_off, s); release(sq, s); release(sp, s);
        release(s1n, s); release(chi0f, s); release(slot_cur, s); release(slot_k, s);
        release(slot_kind, s); release(slot_soff, s); release(slot_n, s); release(L, s);
        release(key, s); release(dlt, s); release(cs, s); release(grid0, s); release(grid1, s);
        release(spec, s); release(out, s); release(out2, s); release(list, s); release(list2, s); release(list3, s);
        release(list4, s); release(dftab, s); release(qbase, s); release(items, s); release(part, s);
        release(counts, s); release(curves, s); release(tops, s); release(bbest, s);
        release(theta, s); release(pent, s);
        release(recs, s); release(cnt_hist, s); release(red, s);
        release(cp.d_twlo, s); release(cp.d_twhi, s); release(cp.d_twst, s); release(cp.d_dec, s);
        for (int i = 0; i < 2; ++i) {
            if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
            gexec[i] = nullptr;
            if (ev_graph[i]) cudaEventDestroy(ev_graph[i]);
            if (ev_tab[i]) cudaEventDestroy(ev_tab[i]);
            ev_graph[i] = ev_tab[i] = nullptr;
        }
        release(scal_all, s); release(goff, s);
        pinned_release(pins);
        pins = PinnedPair();
        stage = nullptr;
        for (auto& e : ev)
            if (e) { cudaEventDestroy(e); e = nullptr; }
        for (int i = 0; i < 2; ++i) {
            if (ev_ready[i]) cudaEventDestroy(ev_ready[i]);
            if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
            ev_ready[i] = ev_copied[i] = nullptr;
        }
        if (cs2) cudaStreamDestroy(cs2);
        cs2 = nullptr;
        hmap = hmap_dev = nullptr;
    }
};

// Process-wide switch of the batched path's stage timing (diagnostics).
static bool g_batch_timing = false;
void set_batch_timing(bool on) { g_batch_timing = on; }


__global__ void k_set_count(int32_t* c, int32_t v) { *c = v; }

// Word copy by a kernel: small results go to mapped host memory (and counters to
// their history) without a copy-engine transfer, which would queue behind the
// large host copy of the previous chunk's periodogram.
__global__ void k_copy_words(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                             int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Shared sampling: every curve of the chunk must have the first curve's times
// and errors proportional to its errors (sigma_c = r_c sigma_0, so that their
// normalised weights and hence the Q transforms agree).  Violations set
// FC2_ERR_INVALID_ARG in *status.
__global__ void k_shared_check(const double* __restrict__ t, const double* __restrict__ sg,
                               const int64_t* __restrict__ off, int nc,
                               int* __restrict__ status) {
    const int c = blockIdx.y + 1;
    if (c >= nc) return;
    const int64_t n0 = off[1] - off[0];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n0) return;
    if (off[c + 1] - off[c] != n0) {
        if (i == 0) atomicExch(status, (int)FC2_ERR_INVALID_ARG);
        return;
    }
    const double r = sg[off[c]] / sg[off[0]];
    const double a = sg[off[0] + i], b = sg[off[c] + i];
    if (t[off[c] + i] != t[off[0] + i] || !(fabs(b - r * a) <= 1e-12 * b))
        atomicExch(status, (int)FC2_ERR_INVALID_ARG);
}

// Launches of one chunk after its tables are in place: everything from the
// gather to the coefficient records, no host synchronisation in between (so
// the sequence can be captured as a CUDA graph).
template <typename T>
static cudaError_t chunk_launches(Batch& b, int nc, int64_t ntot, int64_t nmax, int S,
                                  const std::vector<std::vector<int>>& hgroups,
                                  const std::vector<int>& hgroup_off, int K, float* out,
                                  int64_t nrec, double tau_drop) {
    cudaStream_t s = b.s;
    fc2_plan_s& p = b.cp;
    const int64_t N = p.N;
    int64_t nl = 0;
    CurveTab ct{b.off, b.H, b.fmin, b.df, b.scal, b.slot0, b.out_off, b.sq, b.sp, b.s1n, b.chi0f,
                b.qown, b.pslot0, b.bx_ch};
    // (inside a stream capture only an external event record becomes a node of
    // the graph; a plain record there would only order the capture)
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (b.timing && cudaStreamIsCapturing(s, &capturing) != cudaSuccess) {
        cudaGetLastError();
        capturing = cudaStreamCaptureStatusNone;
    }
    auto mark = [&](int i) {
        if (!b.timing) return;
        if (capturing == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(b.ev[i], s, cudaEventRecordExternal);
        else
            cudaEventRecord(b.ev[i], s);
    };
    mark(0);
    k_bgather<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(
        b.tc, b.xc, b.sgc, b.perm, ntot, b.off, nc, b.scal, b.fmin, b.df, b.tau, b.wq, b.wp, b.A, b.B,
        b.wq32, b.wp32);
    ++nl;
    cudaError_t e = launch_init_dftab(b.dftab, false, s);
    if (e != cudaSuccess) return e;
    ++nl;
    dim3 gph((unsigned)((nmax + 255) / 256), (unsigned)S);
    k_bphase<T><<<gph, 256, 0, s>>>(b.tau, b.wq, b.wp, b.A, b.B, (const dfc*)b.dftab, b.off,
                                    b.fmin, b.df, N, p.M, p.w,
                                    b.slot_cur, b.slot_k, b.slot_kind, b.slot_soff, b.key,
                                    (T*)b.dlt, (cpx<T>*)b.cs);
    ++nl;
    e = sort_wrapping_keys(&p, s);
    if (e != cudaSuccess) return e;
    e = launch_spread(&p, s);
    if (e != cudaSuccess) return e;
    mark(1);
    e = launch_fft(&p, s);
    if (e != cudaSuccess) return e;
    mark(2);
    nl += 1 + (int64_t)p.passes.size();
    cudaMemsetAsync(b.counts, 0, 8 * sizeof(int32_t), s);
    k_set_count<<<1, 1, 0, s>>>(b.counts + 4, (int32_t)nrec);  // record count for the peaks
    const bool f32 = sizeof(T) == 4;
    const double eps_spec = f32 ? 1e-7 : 1e-13;
    const double err_fix = 2e-5;
    int64_t* first_list = f32 ? b.list : b.list2;  // float: re-solve list; double: exact list
    int32_t* first_cnt = f32 ? b.counts + 0 : b.counts + 1;
    const int64_t first_cap = f32 ? (int64_t)b.cl1 : (int64_t)b.cl2;
    for (size_t gi = 0; gi < hgroups.size(); ++gi) {
        const int Hh = hgroups[gi].empty() ? 0 : (int)gi + 1;
        if (!Hh) continue;
        // block of 128 threads, or 256 for float when the autotuner chose it
        const int ant = (f32 && b.asm_nt == 256) ? 256 : 128;
        dim3 ga((unsigned)((N + ant - 1) / ant), (unsigned)hgroups[gi].size());
        const int* cl = b.curves + hgroup_off[gi];
        const double eps = f32 ? eps_spec + 3e-7 : eps_spec;
#define FC2_BASM(HH)                                                                          \
    case HH:                                                                                  \
        if (ant == 256)                                                                       \
            k_bassemble<T, HH, 256><<<ga, 256, 0, s>>>(                                       \
                (const cpx<T>*)p.d_spec, (const T*)p.d_dec, N, cl, ct, (T)tau_drop, (T)eps,   \
                (T)err_fix, out, first_list, first_cnt, first_cap);                           \
        else                                                                                  \
            k_bassemble<T, HH, 128><<<ga, 128, 0, s>>>(                                       \
                (const cpx<T>*)p.d_spec, (const T*)p.d_dec, N, cl, ct, (T)tau_drop, (T)eps,   \
                (T)err_fix, out, first_list, first_cnt, first_cap);                           \
        break;
        switch (Hh) {
            FC2_BASM(1) FC2_BASM(2) FC2_BASM(3) FC2_BASM(4) FC2_BASM(5) FC2_BASM(6) FC2_BASM(7)
            FC2_BASM(8)
            default: return cudaErrorInvalidValue;
        }
#undef FC2_BASM
        ++nl;
    }
    if (f32) {
        k_bresolve<BHM><<<4 * 152, 128, 0, s>>>((const cpx<float>*)p.d_spec, (const float*)p.d_dec,
                                                N, ct, tau_drop, eps_spec, err_fix, out, b.list,
                                                b.counts + 0, (int64_t)b.cl1, b.list2, b.counts + 1,
                                                (int64_t)b.cl2, b.list3, b.counts + 2,
                                                (int64_t)b.cl3, b.list4, b.counts + 3,
                                                (int64_t)b.cl4);
        ++nl;
    }
    mark(3);
    // exact fix-up: float sums over list2 (escalating to list3), double-float
    // sums over list3 (escalating to list4), double sums over list4
    const dfc* tab = (const dfc*)b.dftab;
    const unsigned gx = 2 * 152;
    int32_t* nitems = b.counts + 10;
    // one tier (or the records) over `list`: number the work items, sum them,
    // then add, solve and route each entry
    auto exact = [&](auto tier_tag, auto mode_tag, const int64_t* list, const int32_t* cnt,
                     int64_t cap, double tau, int64_t* next, int32_t* next_cnt, int64_t next_cap,
                     fc2_best* recs) {
        constexpr int TIER = decltype(tier_tag)::value, MODE = decltype(mode_tag)::value;
        k_bx_split<<<1, BX_SPLIT_NT, 0, s>>>(ct, list, cnt, cap, b.qbase, b.items, nitems);
        k_bx_part<BHM, TIER><<<gx, BX_NT, 0, s>>>(b.A, b.B, b.wq32, b.wp32, b.wq, b.wp, tab, ntot,
                                                  ct, list, b.items, nitems, b.part);
        k_bexact<BHM, TIER, MODE><<<gx, BX_NT, 0, s>>>(b.A, b.B, b.wq32, b.wp32, b.wq, b.wp, tab,
                                                       ntot, ct, N, list, cnt, cap, b.qbase, b.part,
                                                       tau, err_fix, out, next, next_cnt, next_cap,
                                                       recs);
        nl += 3;
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    exact(I1{}, I0{}, b.list2, b.counts + 1, (int64_t)b.cl2, 1e-13, b.list3, b.counts + 2,
          (int64_t)b.cl3, nullptr);
    exact(I2{}, I0{}, b.list3, b.counts + 2, (int64_t)b.cl3, 1e-13, b.list4, b.counts + 3,
          (int64_t)b.cl4, nullptr);
    // the last tier: sums exact in fixed point on the float and integer pipes for
    // the mixed path, double sums for the FP64 path
    if (f32 && !b.double_last)
        exact(I4{}, I0{}, b.list4, b.counts + 3, (int64_t)b.cl4, 1e-13, nullptr, nullptr, 0,
              nullptr);
    else
        exact(I3{}, I0{}, b.list4, b.counts + 3, (int64_t)b.cl4, 1e-13, nullptr, nullptr, 0,
              nullptr);
    mark(4);
    if (K > 0) {
        const int nblk = (int)((N + BP_B - 1) / BP_B);
        k_bpeaks0<<<dim3((unsigned)nblk, (unsigned)nc), BP_NT, 0, s>>>(out, N, ct, nblk, b.bbest);
        k_bpeaks_theta<<<(unsigned)nc, 256, 0, s>>>(b.bbest, nblk, K, b.theta);
        k_bpeaks1<<<dim3((unsigned)nblk, (unsigned)nc), BP_NT, 0, s>>>(out, N, ct, K, nblk, b.bbest,
                                                                        b.theta, b.tops);
        k_bpeaks2<<<(unsigned)nc, 256, 0, s>>>(b.tops, nblk, K, b.pent);
        nl += 4;
        exact(I2{}, I1{}, b.pent, b.counts + 4, nrec, tau_drop, nullptr, nullptr, 0, b.recs_now);
    }
    mark(5);
    b.launches += nl;
    return cudaGetLastError();
}

// One chunk's launches as a CUDA graph: captured from the stream, then the
// executable graph of the previous chunk is updated in place when the launch
// sequence has the same shape (same stages, H groups and passes), else a new
// one is instantiated.  A stream that cannot be captured gets the launches
// directly.
template <typename F>
static cudaError_t launch_as_graph(Batch& b, cudaGraphExec_t& gexec, F&& launches) {
    cudaStream_t s = b.s;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return launches();
    }
    const cudaError_t el = launches();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (el != cudaSuccess || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return el != cudaSuccess ? el : (ec != cudaSuccess ? ec : cudaErrorUnknown);
    }
    if (gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        }
    }
    cudaError_t e = cudaSuccess;
    if (!gexec) e = cudaGraphInstantiate(&gexec, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, s);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) ++b.graphs;
    return e;
}


// ------------------------------------------------------------ batch autotuner
// The batched path looks up the launch configuration by (device, N, M, oversampling, precision, kernel
// width, largest H of the chunk, shared sampling); on a miss it times the
// candidates on the chunk itself, one parameter after the other with the
// others held (each candidate run twice after a warm-up, the best of the two
// of the stage it affects), and keeps the fastest.  Choices are kept for the
// process and, unless disabled, appended to a text file read at the first
// lookup, so later processes skip the tuning.  Every candidate gives results
// within the same error bounds; the rounding of the float stages depends on
// the choice (radices, summation order within work items).

struct BatchTuneKey {
    std::string dev;
    int64_t N, M;
    int osmp, fp64, w, hmax, shared;
    bool operator<(const BatchTuneKey& o) const {
        return std::tie(dev, N, M, osmp, fp64, w, hmax, shared) <
               std::tie(o.dev, o.N, o.M, o.osmp, o.fp64, o.w, o.hmax, o.shared);
    }
};

static std::mutex g_btune_mu;
static std::map<BatchTuneKey, BatchConfig> g_btune;
static bool g_btune_loaded = false;

#ifndef FC2_SRC_VERSION
#define FC2_SRC_VERSION "unversioned"
#endif

// The cache file: $FC2_TUNE_CACHE ("" or "off": none), else
// $XDG_CACHE_HOME/fc2-gb300/batch_tune.txt or ~/.cache/fc2-gb300/batch_tune.txt.
static std::string tune_cache_path(bool make_dir) {
    const char* env = getenv("FC2_TUNE_CACHE");
    if (env) {
        const std::string v(env);
        if (v.empty() || v == "off") return std::string();
        return v;
    }
    std::string base;
    if (const char* x = getenv("XDG_CACHE_HOME")) base = x;
    else if (const char* h = getenv("HOME")) base = std::string(h) + "/.cache";
    else return std::string();
    const std::string dir = base + "/fc2-gb300";
    if (make_dir) {
        mkdir(base.c_str(), 0755);
        mkdir(dir.c_str(), 0755);
    }
    return dir + "/batch_tune.txt";
}

static std::string device_tag(int dev) {
    static std::mutex mu;
    static std::map<int, std::string> tags;
    std::lock_guard<std::mutex> lk(mu);
    auto it = tags.find(dev);
    if (it != tags.end()) return it->second;
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name(pr.name);
    for (char& c : name)
        if (c == ' ' || c == '\t' || c == ':') c = '_';
    return tags[dev] = name + "_" + std::to_string(pr.multiProcessorCount) + "sm";
}

static bool config_valid(const BatchTuneKey& k, const BatchConfig& c) {
    int logM = 0;
    while ((1ll << logM) < k.M) ++logM;
    if (!fft_choice_valid(logM, k.fp64 != 0, c.fft)) return false;
    if (spread_tile_of(k.M, c.spread_tile) != c.spread_tile) return false;
    if (c.asm_nt != 128 && c.asm_nt != 256) return false;
    if (c.bx_ch != 1024 && c.bx_ch != 2048 && c.bx_ch != 4096) return false;
    if (c.fft_group != 0 && c.fft_group != 8 && c.fft_group != 16 && c.fft_group != 32) return false;
    return true;
}

// (under g_btune_mu) read the cache file once; lines of other sources or
// malformed or invalid lines are skipped
static void load_tune_cache() {
    if (g_btune_loaded) return;
    g_btune_loaded = true;
    const std::string path = tune_cache_path(false);
    if (path.empty()) return;
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char tag[32], ver[64], dev[160];
        long long N, M;
        int osmp, fp64, w, hmax, shared, np, r[4] = {0, 0, 0, 0}, fam, tile, ant, ch, grp;
        const int got = sscanf(line, "%31s %63s %159s %lld %lld %d %d %d %d %d : %d %d %d %d %d %d %d %d %d %d",
                               tag, ver, dev, &N, &M, &osmp, &fp64, &w, &hmax, &shared, &np, &r[0],
                               &r[1], &r[2], &r[3], &fam, &tile, &ant, &ch, &grp);
        if (got != 20 || std::string(tag) != "fc2-batch-tune-2" ||
            std::string(ver) != FC2_SRC_VERSION || np < 1 || np > 4)
            continue;
        BatchTuneKey k{dev, N, M, osmp, fp64, w, hmax, shared};
        BatchConfig c{FftChoice{std::vector<int>(r, r + np), fam}, tile, ant, ch, grp};
        if (config_valid(k, c)) g_btune[k] = c;
    }
    fclose(f);
}

static void store_tune(const BatchTuneKey& k, const BatchConfig& c) {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune[k] = c;
    const std::string path = tune_cache_path(true);
    if (path.empty()) return;
    int r[4] = {0, 0, 0, 0};
    const int np = (int)std::min<size_t>(c.fft.rs.size(), 4);
    for (int i = 0; i < np; ++i) r[i] = c.fft.rs[i];
    char line[512];
    const int len = snprintf(line, sizeof line,
                             "fc2-batch-tune-2 %s %s %lld %lld %d %d %d %d %d : %d %d %d %d %d %d %d %d %d %d\n",
                             FC2_SRC_VERSION, k.dev.c_str(), (long long)k.N, (long long)k.M, k.osmp,
                             k.fp64, k.w, k.hmax, k.shared, np, r[0], r[1], r[2], r[3], c.fft.family,
                             c.spread_tile, c.asm_nt, c.bx_ch, c.fft_group);
    if (len <= 0 || len >= (int)sizeof line) return;
    FILE* f = fopen(path.c_str(), "a");
    if (!f) return;
    fwrite(line, 1, (size_t)len, f);
    fclose(f);
}

static bool lookup_tune(const BatchTuneKey& k, BatchConfig* c) {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    load_tune_cache();
    auto it = g_btune.find(k);
    if (it == g_btune.end()) return false;
    *c = it->second;
    return true;
}

void forget_batch_tuning() {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune.clear();
    g_btune_loaded = false;
}

// A fixed configuration chosen for the next calls (diagnostics and tests:
// every candidate must give the same results within the error bounds); zero
// fields keep the defaults.
static int g_force_tile = 0, g_force_asm = 0, g_force_ch = 0, g_force_grp = 0;
static std::vector<int> g_force_rs;  // forced transform plan (empty: none)
static int g_force_fam = -1;
void force_batch_plan(const int* rs, int n, int family) {
    g_force_rs.assign(rs, rs + (n > 0 ? n : 0));
    g_force_fam = family;
}
void force_batch_config(int spread_tile, int asm_nt, int bx_ch, int fft_group) {
    g_force_tile = spread_tile;
    g_force_asm = asm_nt;
    g_force_ch = bx_ch;
    g_force_grp = fft_group;
}

// Apply a configuration to the chunk plan and the batch.
static cudaError_t apply_config(Batch& b, const BatchConfig& c) {
    b.cp.spread_tile = c.spread_tile;
    b.asm_nt = c.asm_nt;
    b.bx_ch = c.bx_ch;
    std::vector<int> cur;
    for (const auto& ps : b.cp.passes) cur.push_back(ps.logR);
    cudaError_t e = cudaSuccess;
    if (!(cur == c.fft.rs && b.cp.fft_family == c.fft.family)) e = set_fft_choice(&b.cp, c.fft, b.s);
    b.cp.fft_group = c.fft_group;
    return e;
}

// Time the candidates on the chunk: run() launches the whole chunk (no graph);
// the stage events give each stage's milliseconds.  *best starts at the
// default configuration.
template <typename Run>
static cudaError_t tune_chunk(Batch& b, Run&& run, BatchConfig* best, int* timed) {
    const bool had_timing = b.timing;
    for (auto& ev : b.ev)
        if (!ev && cudaEventCreate(&ev) != cudaSuccess) return cudaGetLastError();
    b.timing = true;
    cudaError_t e = cudaSuccess;
    // stage milliseconds of configuration c: the better of two runs after a warm-up
    auto measure = [&](const BatchConfig& c, int stage, float* ms) {
        *ms = 1e30f;
        if ((e = apply_config(b, c)) != cudaSuccess) return;
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            if ((e = run()) != cudaSuccess) return;
            if ((e = cudaStreamSynchronize(b.s)) != cudaSuccess) return;
            float v = 0.f;
            if ((e = cudaEventElapsedTime(&v, b.ev[stage], b.ev[stage + 1])) != cudaSuccess) return;
            if (r > 0) *ms = std::min(*ms, v);
        }
        ++*timed;
    };
    const int logM = b.cp.logM;
    const bool fp64 = b.cp.fp64;
    // transforms: stage 1
    float bestms = 1e30f;
    BatchConfig cur = *best;
    for (const auto& fc : fft_tune_candidates(logM, fp64)) {
        BatchConfig c = cur;
        c.fft = fc;
        float ms;
        measure(c, 1, &ms);
        if (e != cudaSuccess) break;
        if (ms < bestms) { bestms = ms; cur = c; }
    }
    // spreading tile: stage 0
    if (e == cudaSuccess) {
        bestms = 1e30f;
        BatchConfig keep = cur;
        for (int tile : {1024, 2048, 512}) {
            if (spread_tile_of(b.cp.M, tile) != tile) continue;
            BatchConfig c = keep;
            c.spread_tile = tile;
            float ms;
            measure(c, 0, &ms);
            if (e != cudaSuccess) break;
            if (ms < bestms) { bestms = ms; cur = c; }
        }
    }
    // assembly block: stage 2 (float only: FP64 keeps 128)
    if (e == cudaSuccess && !fp64) {
        bestms = 1e30f;
        BatchConfig keep = cur;
        for (int nt : {128, 256}) {
            BatchConfig c = keep;
            c.asm_nt = nt;
            float ms;
            measure(c, 2, &ms);
            if (e != cudaSuccess) break;
            if (ms < bestms) { bestms = ms; cur = c; }
        }
    }
    // exact-sum work item: stage 3
    if (e == cudaSuccess) {
        bestms = 1e30f;
        BatchConfig keep = cur;
        for (int ch : {2048, 1024, 4096}) {
            BatchConfig c = keep;
            c.bx_ch = ch;
            float ms;
            measure(c, 3, &ms);
            if (e != cudaSuccess) break;
            if (ms < bestms) { bestms = ms; cur = c; }
        }
    }
    b.timing = had_timing;
    if (e != cudaSuccess) return e;
    *best = cur;
    return apply_config(b, cur);
}

fc2_status batched_execute(int64_t C, const int64_t* offsets, const double* t, const double* x,
                           const double* sigma, const int* Hc, const double* fminc,
                           const double* dfc, const int64_t* Nc, int oversample,
                           const fc2_options& opt, float* dchi2, fc2_best* peaks,
                           int64_t* launches_out, int64_t* stats_out) {
    // ---- validation (host)
    if (C < 1 || !offsets || !t || !x || !sigma || !Hc || !fminc || !dfc || !Nc)
        return FC2_ERR_INVALID_ARG;
    if (oversample < 2 || oversample > 64) return FC2_ERR_INVALID_ARG;
    if (opt.prec != FC2_PREC_FP64 && opt.prec != FC2_PREC_MIXED) return FC2_ERR_INVALID_ARG;
    if (opt.top_k < 0 || opt.top_k > 64) return FC2_ERR_INVALID_ARG;
    if (opt.fft_kernel < 0 || opt.fft_kernel > 5) return FC2_ERR_INVALID_ARG;
    if (opt.kernel_width != 0 && (opt.kernel_width < 2 || opt.kernel_width > 16))
        return FC2_ERR_INVALID_ARG;  // (the spreading kernels' key tables assume w <= 32)
    if (opt.autotune < -1 || opt.autotune > 1) return FC2_ERR_INVALID_ARG;
    if (opt.gridding < 0 || opt.gridding > 1) return FC2_ERR_INVALID_ARG;
    if (opt.gridding == 1) return FC2_ERR_UNSUPPORTED;
    if (opt.detrend < 0 || opt.detrend > 3) return FC2_ERR_INVALID_ARG;
    if (opt.detrend != 0) return FC2_ERR_UNSUPPORTED;
    if (opt.trend_fit < 0 || opt.trend_fit > 1) return FC2_ERR_INVALID_ARG;
    if (opt.trend_fit != 0) return FC2_ERR_UNSUPPORTED;
    if (opt.shared_sampling < 0 || opt.shared_sampling > 1) return FC2_ERR_INVALID_ARG;
    const bool shared = opt.shared_sampling == 1;
    for (int64_t c = 0; c < C && shared; ++c)  // one sampling: same n, H and trial grid
        if (offsets[c + 1] - offsets[c] != offsets[1] - offsets[0] || Hc[c] != Hc[0] ||
            fminc[c] != fminc[0] || dfc[c] != dfc[0] || Nc[c] != Nc[0])
            return FC2_ERR_INVALID_ARG;
    for (int64_t c = 0; c < C; ++c) {
        if (offsets[c + 1] - offsets[c] < 1 || offsets[c] < 0) return FC2_ERR_INVALID_ARG;
        if (offsets[c + 1] - offsets[c] > (1ll << 31) - 1) return FC2_ERR_INVALID_ARG;
        if (Hc[c] < 1 || Hc[c] > FC2_MAX_H || Nc[c] < 2 || Nc[c] > (1ll << 31) - 1)
            return FC2_ERR_INVALID_ARG;
        if (!(std::isfinite(fminc[c]) && fminc[c] >= 0.0) || !(std::isfinite(dfc[c]) && dfc[c] > 0.0))
            return FC2_ERR_INVALID_ARG;
        if (Hc[c] > BHM) return FC2_ERR_UNSUPPORTED;
        if (fc2_grid_size(Nc[c], oversample) == 0) return FC2_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return FC2_ERR_CUDA;
    if (opt.device < 0 || opt.device >= ndev) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(opt.device) != cudaSuccess) return FC2_ERR_CUDA;

    const bool fp64 = opt.prec == FC2_PREC_FP64;
    const size_t tsz = fp64 ? 8 : 4, csz = 2 * tsz;
    const int K = opt.top_k ? opt.top_k : 8;
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto ms_since = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point z) {
        return std::chrono::duration<double, std::milli>(z - a).count();
    };
    const auto t_entry = now();
    // host inputs are copied to the device whole: a batch whose samples would
    // take more than a quarter of the memory budget runs as two halves
    if (!opt.inputs_on_device && C > 1) {
        size_t fb = 0, tb = 0;
        cudaMemGetInfo(&fb, &tb);
        cudaGetLastError();
        const size_t bud = std::min<size_t>(fb / 2, (size_t)48 << 30);
        if ((size_t)(offsets[C] - offsets[0]) * 24 > bud / 4) {
            const int64_t h = C / 2;
            int64_t l1 = 0, l2 = 0, s1[32] = {0}, s2[32] = {0};
            fc2_status r = batched_execute(h, offsets, t, x, sigma, Hc, fminc, dfc, Nc, oversample, opt,
                                           dchi2, peaks, &l1, s1);
            if (r != FC2_OK) return r;
            int64_t o1 = 0;
            for (int64_t c = 0; c < h; ++c) o1 += (int64_t)Hc[c] * Nc[c];
            r = batched_execute(C - h, offsets + h, t, x, sigma, Hc + h, fminc + h, dfc + h, Nc + h,
                                oversample, opt, dchi2 ? dchi2 + o1 : nullptr,
                                peaks ? peaks + h * K : nullptr, &l2, s2);
            if (launches_out) *launches_out = l1 + l2;
            if (stats_out) {
                for (int i = 0; i < 5; ++i) stats_out[i] = s1[i] + s2[i];
                for (int i = 5; i < 18; ++i) {  // host phases, stage times, bytes: sums of doubles
                    double a1, a2;
                    std::memcpy(&a1, &s1[i], 8);
                    std::memcpy(&a2, &s2[i], 8);
                    a1 += a2;
                    std::memcpy(&stats_out[i], &a1, 8);
                }
                for (int i = 18; i < 32; ++i) stats_out[i] = s2[i];
            }
            return r;
        }
    }
    Batch b;
    if (opt.cuda_stream) b.s = (cudaStream_t)opt.cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking) != cudaSuccess) return FC2_ERR_CUDA;
        b.own_stream = true;
    }
    cudaStream_t s = b.s;
    b.double_last = last_fixup_tier() == 3;
    if (g_batch_timing) {
        b.timing = true;
        for (auto& ev : b.ev)
            if (cudaEventCreate(&ev) != cudaSuccess) b.timing = false;
        cudaGetLastError();
    }
    cudaPointerAttributes at;
    bool out_dev = false;
    if (dchi2 && cudaPointerGetAttributes(&at, dchi2) == cudaSuccess && at.type == cudaMemoryTypeDevice)
        out_dev = true;
    cudaGetLastError();
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    const size_t budget = std::min<size_t>(freeb / 2, (size_t)48 << 30);

    fc2_status st = FC2_OK;
    int64_t out_global = 0;
    int64_t curM = -1, curN = -1;
    int64_t c0 = 0;
    // ---- chunks: consecutive curves with the same N, within the memory budget,
    // planned up front so that every buffer is allocated once, at the largest
    // size any chunk needs
    struct Chunk { int64_t c0, c1, S, ntot, nmax, slot_samples, out, N, M; };
    std::vector<Chunk> chunks;
    Chunk mx{0, 0, 0, 0, 0, 0, 0, 0, 0};
    size_t mx_grid = 0, mx_spec = 0, mx_sort = 0, mx_tops = 0;
    for (int64_t a = 0; a < C;) {
        Chunk ch{a, a, 0, 0, 0, 0, 0, Nc[a], fc2_grid_size(Nc[a], oversample)};
        while (ch.c1 < C && Nc[ch.c1] == ch.N && ch.c1 - a < 2048) {
            const int64_t n = offsets[ch.c1 + 1] - offsets[ch.c1];
            const int64_t sl = (shared && ch.c1 > a) ? Hc[ch.c1] : 3 * Hc[ch.c1];
            const size_t bytes = (size_t)(ch.S + sl) * (size_t)ch.M * csz * 2 +
                                 (size_t)(ch.S + sl) * ch.N * csz +
                                 (size_t)(ch.slot_samples + sl * n) * (4 + tsz + csz) +
                                 (size_t)(ch.ntot + n) * 80;
            if (ch.c1 > a && bytes > budget) break;
            ch.S += sl;
            ch.ntot += n;
            ch.nmax = std::max(ch.nmax, n);
            ch.slot_samples += sl * n;
            ch.out += (int64_t)Hc[ch.c1] * ch.N;
            ++ch.c1;
        }
        chunks.push_back(ch);
        mx.S = std::max(mx.S, ch.S);
        mx.ntot = std::max(mx.ntot, ch.ntot);
        mx.slot_samples = std::max(mx.slot_samples, ch.slot_samples);
        mx.out = std::max(mx.out, ch.out);
        mx.c1 = std::max(mx.c1, ch.c1 - ch.c0);  // curves
        mx_grid = std::max(mx_grid, (size_t)ch.S * ch.M * csz);
        mx_spec = std::max(mx_spec, (size_t)ch.S * ch.N * csz);
        mx_sort = std::max(mx_sort, sort_scratch_bytes(ch.nmax));
        mx_tops = std::max(mx_tops, (size_t)(ch.c1 - ch.c0) * ((ch.N + BP_B - 1) / BP_B) * std::max(K, 1));
        a = ch.c1;
    }
    const int64_t mx_nc = mx.c1, mx_nrec = mx_nc * K;
    b.phase_ms[0] = ms_since(t_entry, now());
    // a host-bound periodogram is copied on a second stream (overlapping the next
    // chunk); with stage timing on, every chunk is waited for instead, so that
    // its stage events can be read before the next chunk records them again.
    // Every curve's peak records stay on the device until the end.
    const bool copy_out = !b.timing && dchi2 && !out_dev;
    const auto tsetup = now();
    {
        bool good = true;
        if (copy_out) {
            good = cudaStreamCreateWithFlags(&b.cs2, cudaStreamNonBlocking) == cudaSuccess;
            for (int i = 0; i < 2 && good; ++i)
                good = cudaEventCreateWithFlags(&b.ev_ready[i], cudaEventDisableTiming) == cudaSuccess &&
                       cudaEventCreateWithFlags(&b.ev_copied[i], cudaEventDisableTiming) == cudaSuccess;
        }
        for (int i = 0; i < 2 && good; ++i)
            good = cudaEventCreateWithFlags(&b.ev_graph[i], cudaEventDisableTiming) == cudaSuccess &&
                   cudaEventCreateWithFlags(&b.ev_tab[i], cudaEventDisableTiming) == cudaSuccess;
        if (!good) {
            cudaGetLastError();
            b.free_all();
            if (b.own_stream) cudaStreamDestroy(s);
            return FC2_ERR_CUDA;
        }
    }
    // pinned staging of the chunk tables (two halves) and mapped memory for the
    // moments of every curve and the status word
    {
        size_t half = 0;
        for (const Chunk& ch : chunks) {
            const size_t nc = (size_t)(ch.c1 - ch.c0), S = (size_t)ch.S;
            half = std::max(half, (nc + 1) * 8 + nc * SC_COUNT * 8 + nc * 72 + S * 44 + 16 * 64);
        }
        b.stage_half = (half + 255) & ~(size_t)255;
        const size_t mbytes = (size_t)C * SC_COUNT * 8 + 64;
        bool got = pinned_acquire(2 * b.stage_half, mbytes, &b.pins);
        if (got) {
            b.stage = b.pins.stage;
            b.hmap = b.pins.map;
            got = cudaHostGetDevicePointer((void**)&b.hmap_dev, b.hmap, 0) == cudaSuccess;
        }
        if (!got) {
            cudaGetLastError();
            b.free_all();
            if (b.own_stream) cudaStreamDestroy(s);
            return FC2_ERR_OOM;
        }
    }
    b.phase_ms[1] += ms_since(tsetup, now());  // streams, events, pinned buffers
    // configuration: 0 fixed (autotune -1, or a transform family requested),
    // 1 the tuning table with tuning on a miss (autotune 0), 2 tuning anew (1)
    const int tune_mode = (opt.autotune < 0 || opt.fft_kernel != 0) ? 0 : (opt.autotune == 1 ? 2 : 1);
    const size_t nchunks = chunks.size();
    std::vector<int32_t> hist(nchunks * 16, 0);
    size_t launched = 0;  // chunks whose graph was launched
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; return e == cudaSuccess; };

    // ---- inputs on the device (host inputs copied once), then the moments of
    // every curve in one launch and one wait
    const int64_t base0 = offsets[0], ntot_all = offsets[C] - base0;
    const double *tall = t + base0, *xall = x + base0, *sgall = sigma + base0;
    {
        const auto tpa = now();
        if (!opt.inputs_on_device) {
            ok(need(&b.t, &b.ct, (size_t)ntot_all, s)) && ok(need(&b.x, &b.cx, (size_t)ntot_all, s)) &&
                ok(need(&b.sg, &b.csg, (size_t)ntot_all, s)) &&
                ok(cudaMemcpyAsync(b.t, t + base0, ntot_all * 8, cudaMemcpyHostToDevice, s)) &&
                ok(cudaMemcpyAsync(b.x, x + base0, ntot_all * 8, cudaMemcpyHostToDevice, s)) &&
                ok(cudaMemcpyAsync(b.sg, sigma + base0, ntot_all * 8, cudaMemcpyHostToDevice, s));
            tall = b.t; xall = b.x; sgall = b.sg;
        }
        std::vector<int64_t> goffv(C + 1);
        for (int64_t c = 0; c <= C; ++c) goffv[c] = offsets[c] - base0;
        ok(need(&b.goff, &b.cgoff, (size_t)C + 1, s)) &&
            ok(need(&b.scal_all, &b.cscal_all, (size_t)C * SC_COUNT, s)) &&
            ok(need(&b.counts, &b.ccnt, 16, s)) &&
            ok(cudaMemcpyAsync(b.goff, goffv.data(), (C + 1) * 8, cudaMemcpyHostToDevice, s)) &&
            ok(cudaMemsetAsync(b.counts, 0, 16 * sizeof(int32_t), s));
        if (shared && e == cudaSuccess)
            for (const Chunk& ch : chunks) {
                const int nc = (int)(ch.c1 - ch.c0);
                if (nc < 2) continue;
                const int64_t n0 = offsets[ch.c0 + 1] - offsets[ch.c0];
                k_shared_check<<<dim3((unsigned)((n0 + 255) / 256), (unsigned)(nc - 1)), 256, 0, s>>>(
                    tall, sgall, b.goff + ch.c0, nc, b.counts + 8);
            }
        ok(cudaGetLastError());
        if (e == cudaSuccess) ok(launch_moments(tall, xall, sgall, b.goff, C, 0, b.scal_all, b.counts + 8, s));
        const int64_t nsw = C * SC_COUNT * 2;  // 32-bit words of the moments
        if (e == cudaSuccess) {
            k_copy_words<<<(unsigned)std::min<int64_t>((nsw + 255) / 256, 4096), 256, 0, s>>>(
                (const uint32_t*)b.scal_all, (uint32_t*)b.hmap_dev, nsw);
            k_copy_words<<<1, 32, 0, s>>>((const uint32_t*)(b.counts + 8),
                                          (uint32_t*)(b.hmap_dev + 4 * nsw), 1);
            ok(cudaGetLastError());
        }
        ok(cudaStreamSynchronize(s));
        int32_t status = 0;
        if (e == cudaSuccess) std::memcpy(&status, b.hmap + 4 * nsw, 4);
        if (e != cudaSuccess) st = map_cuda(e);
        else if (status) st = (fc2_status)status;
        b.phase_ms[2] += ms_since(tpa, now());
    }
    const double* scal_host = (const double*)b.hmap;

    for (size_t ci = 0; ci < nchunks; ++ci) {
        const Chunk& ch = chunks[ci];
        const int slot = (int)(ci & 1);
        if (st != FC2_OK) break;
        c0 = ch.c0;
        const int64_t c1 = ch.c1, S = ch.S, ntot = ch.ntot, nmax = ch.nmax, N = ch.N, M = ch.M;
        const int nc = (int)(c1 - c0);
        fc2_plan_s& p = b.cp;
        // ---- shared tables for this (N, M)
        if (M != curM || N != curN) {
            p.M = M;
            p.logM = 0;
            while ((1ll << p.logM) < M) ++p.logM;
            p.N = N;
            p.fp64 = fp64;
            p.oversample = oversample;
            p.w = opt.kernel_width ? opt.kernel_width : default_width(fp64, oversample);
            p.beta = 0.97 * M_PI * (1.0 - 0.5 / ((double)M / (double)N)) * (double)p.w;
            p.stream = s;
            plan_fft_passes(&p);
            p.fft_family = fft_family_of(opt.fft_kernel);
            release(p.d_twlo, s); release(p.d_twhi, s); release(p.d_twst, s); release(p.d_dec, s);
            const int sh = (p.logM + 1) / 2;
            cudaError_t ea = pool_alloc((void**)&p.d_twlo, (size_t)(1ll << sh) * csz, s);
            if (ea == cudaSuccess) ea = pool_alloc((void**)&p.d_twhi, (size_t)(M >> sh) * csz, s);
            if (ea == cudaSuccess) ea = pool_alloc((void**)&p.d_twst, (size_t)(8 * 4096 + 256) * csz, s);
            if (ea == cudaSuccess) ea = pool_alloc((void**)&p.d_dec, (size_t)N * tsz, s);
            if (ea == cudaSuccess) ea = need(&b.red, &b.cred, 8192, s);
            p.d_red = b.red;
            if (ea == cudaSuccess) ea = init_twiddles(&p, s);
            if (ea == cudaSuccess) ea = init_deconv(&p, s);
            if (ea != cudaSuccess) { st = map_cuda(ea); break; }
            curM = M;
            curN = N;
        }
        // ---- buffers (allocated by the first chunk at the largest size any needs)
        const auto tpb = now();
        const int64_t base = offsets[c0] - base0;
        b.tc = tall + base; b.xc = xall + base; b.sgc = sgall + base;
        const int64_t nrec = (int64_t)nc * K;
        const int64_t out_chunk = ch.out;
        const size_t mxs = (size_t)mx.S, mxn = (size_t)mx.ntot, mxc = (size_t)mx_nc;
        const size_t mxo = (size_t)mx.out, mxss = (size_t)mx.slot_samples;
        ok(need(&b.perm, &b.cperm, mxn, s)) && ok(need(&b.tau, &b.ctau, mxn, s)) &&
            ok(need(&b.wq, &b.cwq, mxn, s)) && ok(need(&b.wp, &b.cwp, mxn, s)) &&
            ok(need(&b.A, &b.cA, mxn, s)) && ok(need(&b.B, &b.cB, mxn, s)) &&
            ok(need(&b.wq32, &b.cwq32, 2 * mxn, s)) && ok(need(&b.wp32, &b.cwp32, 2 * mxn, s)) &&
            ok(need(&b.off, &b.coff, mxc + 1, s)) && ok(need(&b.H, &b.cH, mxc, s)) &&
            ok(need(&b.slot0, &b.cslot0, mxc, s)) && ok(need(&b.fmin, &b.cfmin, mxc, s)) &&
            ok(need(&b.qown, &b.cqown, mxc, s)) && ok(need(&b.pslot0, &b.cpslot0, mxc, s)) &&
            ok(need(&b.df, &b.cdf, mxc, s)) && ok(need(&b.scal, &b.cscal, mxc * SC_COUNT, s)) &&
            ok(need(&b.out_off, &b.coo, mxc, s)) && ok(need(&b.sq, &b.csq, mxc, s)) &&
            ok(need(&b.sp, &b.csp, mxc, s)) && ok(need(&b.s1n, &b.cs1n, mxc, s)) &&
            ok(need(&b.chi0f, &b.cchi0f, mxc, s)) && ok(need(&b.slot_cur, &b.cscur, mxs, s)) &&
            ok(need(&b.slot_k, &b.csk, mxs, s)) && ok(need(&b.slot_kind, &b.cskind, mxs, s)) &&
            ok(need(&b.slot_soff, &b.cssoff, mxs, s)) && ok(need(&b.slot_n, &b.csn, mxs, s)) &&
            ok(need(&b.L, &b.cL, mxs, s)) && ok(need(&b.key, &b.ckey, mxss, s)) &&
            ok(need(&b.dlt, &b.cdlt, mxss * tsz, s)) &&
            ok(need(&b.cs, &b.ccs, mxss * csz, s)) &&
            ok(need(&b.grid0, &b.cg0, mx_grid, s)) &&
            ok(need(&b.grid1, &b.cg1, std::max(mx_grid, mx_sort + 4096), s)) &&
            ok(need(&b.spec, &b.cspec, mx_spec, s)) &&
            ok(need(&b.list, &b.cl1, std::min<size_t>(mxo, 1 << 24), s)) &&
            ok(need(&b.list2, &b.cl2, std::min<size_t>(mxo, 1 << 22), s)) &&
            ok(need(&b.list3, &b.cl3, std::min<size_t>(mxo, 1 << 20), s)) &&
            ok(need(&b.list4, &b.cl4, std::min<size_t>(mxo, 1 << 20), s)) &&
            ok(need(&b.dftab, &b.cdftab, 2 * 512 * 16, s)) &&
            ok(need(&b.qbase, &b.cqbase,
                    std::max<size_t>({b.cl2, b.cl3, b.cl4, (size_t)std::max<int64_t>(mx_nrec, 1)}), s)) &&
            ok(need(&b.items, &b.citems, (size_t)BX_ITEMS, s)) &&
            ok(need(&b.part, &b.cpart, (size_t)BX_ITEMS * 6 * BHM, s)) &&
            ok(need(&b.curves, &b.ccurves, mxc, s)) &&
            ok(need(&b.tops, &b.ctops, mx_tops, s)) &&
            ok(need(&b.bbest, &b.cbbest, std::max<size_t>(mx_tops / std::max(K, 1), 1), s)) &&
            ok(need(&b.theta, &b.ctheta, mxc, s)) &&
            ok(need(&b.pent, &b.cpent, (size_t)std::max<int64_t>(mx_nrec, 1), s)) &&
            ok(need(&b.recs, &b.crecs, (size_t)std::max<int64_t>(C * K, 1), s)) &&
            ok(need(&b.cnt_hist, &b.chist, nchunks * 16, s));
        b.recs_now = b.recs + c0 * K;
        float* out = nullptr;
        if (dchi2 && out_dev) out = dchi2 + out_global;
        else if (copy_out && slot) { if (ok(need(&b.out2, &b.cout2, (size_t)mx.out, s))) out = b.out2; }
        else if (ok(need(&b.out, &b.cout, (size_t)mx.out, s))) out = b.out;
        if (e != cudaSuccess) { st = map_cuda(e); break; }
        const auto tp1 = now();
        b.phase_ms[1] += ms_since(tpb, tp1);
        // ---- host-side layout from the curves' moments
        std::vector<int64_t> offl(nc + 1);
        for (int c = 0; c <= nc; ++c) offl[c] = offsets[c0 + c] - offsets[c0];
        std::vector<double> scal(scal_host + (size_t)c0 * SC_COUNT, scal_host + (size_t)c1 * SC_COUNT);
        std::vector<int> Hv(nc), slot0(nc), scur, sk, skind, qownv(nc), pslotv(nc);
        std::vector<double> fminv(nc), dfv(nc);
        std::vector<int64_t> oo(nc), ssoff, sn, Lv;
        std::vector<float> sqv(nc), spv(nc), s1v(nc), c0v(nc);
        std::vector<std::vector<int>> hg(BHM);
        bool unsorted = false;
        // ---- launch configuration: fixed, from the tuning table, or tuned on
        // this chunk (then the occupied length of each grid is first rounded to
        // suit every candidate, and again to the choice afterwards)
        int hmax = 0;
        for (int c = 0; c < nc; ++c) hmax = std::max(hmax, Hc[c0 + c]);
        const BatchTuneKey tkey{device_tag(opt.device), N, M, oversample, fp64 ? 1 : 0, p.w, hmax,
                                shared ? 1 : 0};
        BatchConfig cfg{FftChoice{std::vector<int>(), p.fft_family}, spread_tile_of(M, 0), 128, BX_CH};
        {
            fc2_plan_s tmp;
            tmp.logM = p.logM;
            tmp.fp64 = p.fp64;
            plan_fft_passes(&tmp);
            for (const auto& ps : tmp.passes) cfg.fft.rs.push_back(ps.logR);
        }
        int source = 0;  // 0 fixed, 1 table, 2 tuned here
        if (tune_mode == 0) {
            cfg.spread_tile = spread_tile_of(M, g_force_tile);
            if (g_force_asm == 256 && !fp64) cfg.asm_nt = 256;
            if (g_force_ch == 1024 || g_force_ch == 4096) cfg.bx_ch = g_force_ch;
            if (g_force_grp == 8 || g_force_grp == 16 || g_force_grp == 32) cfg.fft_group = g_force_grp;
            if (!g_force_rs.empty()) {
                const FftChoice fc{g_force_rs, g_force_fam};
                if (fft_choice_valid(p.logM, fp64, fc)) cfg.fft = fc;
            }
        } else if (tune_mode == 1 && lookup_tune(tkey, &cfg)) {
            source = 1;
        } else {
            source = 2;
        }
        int64_t unit = std::max(M >> cfg.fft.rs[0], (int64_t)cfg.spread_tile);
        if (source == 2) {
            for (const auto& fc : fft_tune_candidates(p.logM, fp64)) unit = std::max(unit, M >> fc.rs[0]);
            for (int tile : {512, 1024, 2048}) unit = std::max(unit, (int64_t)spread_tile_of(M, tile));
        }
        if (e == cudaSuccess && source != 2) e = apply_config(b, cfg);
        int64_t acc_out = 0, acc_s = 0;
        std::vector<double> cellsv;  // per grid: occupied cells, or -1 for a full grid
        p.geom.assign(S, GridGeom{});
        int gi = 0;
        for (int c = 0; c < nc; ++c) {
            const int64_t cg = c0 + c;
            double* sc = &scal[(size_t)c * SC_COUNT];
            const double back = (0.5 * p.w + 1.0) / ((double)M * dfc[cg]);
            sc[SC_T0] -= back;
            sc[SC_TAUMAX] += back;
            if (sc[SC_SORTED] == 0.0) unsorted = true;
            Hv[c] = Hc[cg]; fminv[c] = fminc[cg]; dfv[c] = dfc[cg];
            oo[c] = acc_out;
            acc_out += (int64_t)Hc[cg] * N;
            const double W = sc[SC_W], chi0 = sc[SC_CHI0];
            sqv[c] = (float)(1.0 / W);
            spv[c] = (float)((chi0 > 0.0) ? 1.0 / sqrt(W * chi0) : 0.0);
            s1v[c] = (float)(sc[SC_S1] * ((chi0 > 0.0) ? 1.0 / sqrt(W * chi0) : 0.0));
            c0v[c] = (float)chi0;
            hg[Hc[cg] - 1].push_back(c);
            // shared sampling: the chunk's first curve owns the Q transforms
            const bool own_q = !shared || c == 0;
            qownv[c] = own_q ? c : 0;
            slot0[c] = own_q ? gi : slot0[0];
            pslotv[c] = own_q ? gi + 2 * Hc[cg] : gi;
            const int64_t n = offl[c + 1] - offl[c];
            for (int q = own_q ? 0 : 2 * Hc[cg]; q < 3 * Hc[cg]; ++q, ++gi) {
                const int k = (q < 2 * Hc[cg]) ? q + 1 : q - 2 * Hc[cg] + 1;
                const int kind = (q < 2 * Hc[cg]) ? 0 : 1;
                scur.push_back(c); sk.push_back(k); skind.push_back(kind);
                ssoff.push_back(acc_s); sn.push_back(n);
                acc_s += n;
                const double pmax = (double)k * dfc[cg] * sc[SC_TAUMAX];
                const double cells = pmax * (double)M;
                GridGeom& gg = p.geom[gi];
                gg.k = k; gg.kind = kind;
                if (!(pmax < 1.0) || cells + p.w + 2.0 >= (double)M) {
                    gg.wraps = (pmax >= 1.0) ? 1 : 0;
                    cellsv.push_back(-1.0);
                } else {
                    gg.wraps = 0;
                    cellsv.push_back(cells);
                }
            }
        }
        // occupied lengths: whole spreading tiles and whole first-pass rows
        auto fill_L = [&](int64_t u) {
            Lv.assign(S, M);
            for (int64_t g = 0; g < S; ++g) {
                if (cellsv[g] >= 0.0) {
                    int64_t Lc = (int64_t)floor(cellsv[g]) + p.w + 3;
                    Lc = ((Lc + u - 1) / u) * u;
                    Lv[g] = std::min(Lc, M);
                }
                p.geom[g].L = Lv[g];
            }
            p.h_L = Lv;
        };
        fill_L(unit);
        std::vector<int> curves_flat, hoff(BHM);
        for (int h = 0; h < BHM; ++h) {
            hoff[h] = (int)curves_flat.size();
            curves_flat.insert(curves_flat.end(), hg[h].begin(), hg[h].end());
        }
        // ---- the tables, through this chunk's half of the pinned staging (free
        // once the copies of the chunk two before are done), in stream order
        // after the previous chunk's launches
        if (b.tab_pending[slot]) {
            ok(cudaEventSynchronize(b.ev_tab[slot]));
            b.tab_pending[slot] = false;
        }
        char* stg = b.stage + (size_t)slot * b.stage_half;
        size_t sused = 0;
        auto put = [&](void* dst, const void* src, size_t bytes) {
            if (bytes == 0 || e != cudaSuccess) return;
            if (sused + bytes > b.stage_half) { e = cudaErrorInvalidValue; return; }
            std::memcpy(stg + sused, src, bytes);
            ok(cudaMemcpyAsync(dst, stg + sused, bytes, cudaMemcpyHostToDevice, s));
            sused += (bytes + 15) & ~(size_t)15;
        };
        put(b.off, offl.data(), (nc + 1) * 8);
        put(b.scal, scal.data(), scal.size() * 8);
        put(b.H, Hv.data(), nc * 4);
        put(b.slot0, slot0.data(), nc * 4);
        put(b.qown, qownv.data(), nc * 4);
        put(b.pslot0, pslotv.data(), nc * 4);
        put(b.fmin, fminv.data(), nc * 8);
        put(b.df, dfv.data(), nc * 8);
        put(b.out_off, oo.data(), nc * 8);
        put(b.sq, sqv.data(), nc * 4);
        put(b.sp, spv.data(), nc * 4);
        put(b.s1n, s1v.data(), nc * 4);
        put(b.chi0f, c0v.data(), nc * 4);
        put(b.slot_cur, scur.data(), S * 4);
        put(b.slot_k, sk.data(), S * 4);
        put(b.slot_kind, skind.data(), S * 4);
        put(b.slot_soff, ssoff.data(), S * 8);
        put(b.slot_n, sn.data(), S * 8);
        put(b.L, Lv.data(), S * 8);
        put(b.curves, curves_flat.data(), nc * 4);
        ok(cudaEventRecord(b.ev_tab[slot], s));
        b.tab_pending[slot] = true;
        ok(cudaMemsetAsync(b.counts, 0, 16 * sizeof(int32_t), s));
        // time order within each curve
        k_iota_plus<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(b.perm, ntot, 0);
        if (unsorted)
            for (int c = 0; c < nc; ++c)
                if (scal[(size_t)c * SC_COUNT + SC_SORTED] == 0.0) {
                    const int64_t n = offl[c + 1] - offl[c];
                    ok(sort_by_time(b.tc + offl[c], n, b.perm + offl[c], b.grid1, b.cg1, s));
                    k_add_base<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.perm + offl[c], n, offl[c]);
                }
        // chunk plan fields for the shared launchers
        p.G = (int)S;
        p.n = 0;
        p.d_key = b.key; p.d_dlt = b.dlt; p.d_cs = b.cs;
        p.d_grid[0] = b.grid0; p.d_grid[1] = b.grid1; p.d_spec = b.spec;
        p.d_L = b.L; p.d_slot_soff = b.slot_soff; p.d_slot_n = b.slot_n;
        p.d_status = b.counts + 8;  // status word of the chunk's kernels (bounded waits)
        p.h_slot_soff = ssoff; p.h_slot_n = sn;
        const double tau_drop = opt.alias_tau > 0.0 ? opt.alias_tau : (fp64 ? 1e-9 : 1e-6);
        if (e == cudaSuccess && source == 2) {
            const auto tt0 = now();
            e = tune_chunk(b, [&]() {
                return fp64 ? chunk_launches<double>(b, nc, ntot, nmax, (int)S, hg, hoff, K, out, nrec,
                                                     tau_drop)
                            : chunk_launches<float>(b, nc, ntot, nmax, (int)S, hg, hoff, K, out, nrec,
                                                    tau_drop);
            }, &cfg, &b.tune_timed);
            if (e == cudaSuccess) {
                store_tune(tkey, cfg);
                fill_L(std::max(M >> cfg.fft.rs[0], (int64_t)cfg.spread_tile));
                // (the tuning runs waited for every copy of this half)
                put(b.L, Lv.data(), S * 8);
                ok(cudaMemsetAsync(b.counts, 0, 16 * sizeof(int32_t), s));
                ok(cudaEventRecord(b.ev_tab[slot], s));
            }
            b.tune_ms += ms_since(tt0, now());
        }
        if (e != cudaSuccess) { st = map_cuda(e); break; }
        b.cfg = cfg;
        b.cfg_source = std::max(b.cfg_source, source);
        // this chunk's buffers are the ones of the chunk two before it: its copies
        // to the host must be done before the graph writes them again
        if (e == cudaSuccess && copy_out && b.copied_pending[slot]) {
            ok(cudaStreamWaitEvent(s, b.ev_copied[slot], 0));
            b.copied_pending[slot] = false;
        }
        // the executable graph of the chunk two before must have finished
        if (b.graph_pending[slot]) {
            ok(cudaEventSynchronize(b.ev_graph[slot]));
            b.graph_pending[slot] = false;
        }
        const auto tp2 = now();
        b.phase_ms[3] += ms_since(tp1, tp2);
        if (e == cudaSuccess)
            e = launch_as_graph(b, b.gexec[slot], [&]() {
                return fp64 ? chunk_launches<double>(b, nc, ntot, nmax, (int)S, hg, hoff, K, out, nrec,
                                                     tau_drop)
                            : chunk_launches<float>(b, nc, ntot, nmax, (int)S, hg, hoff, K, out, nrec,
                                                    tau_drop);
            });
        const auto tp3 = now();
        b.phase_ms[4] += ms_since(tp2, tp3);
        if (e != cudaSuccess) { st = map_cuda(e); break; }
        ++launched;
        ok(cudaEventRecord(b.ev_graph[slot], s));
        b.graph_pending[slot] = true;
        // ---- results: the chunk's counters kept on the device (read once at the
        // end), its outputs copied to the host
        k_copy_words<<<1, 32, 0, s>>>((const uint32_t*)b.counts, (uint32_t*)(b.cnt_hist + 16 * ci), 16);
        ok(cudaGetLastError());
        if (copy_out) {
            ok(cudaEventRecord(b.ev_ready[slot], s));
            ok(cudaStreamWaitEvent(b.cs2, b.ev_ready[slot], 0));
            // in pieces, so that another transfer waits for one piece at most
            const int64_t piece = (int64_t)64 << 20;  // floats
            for (int64_t a = 0; a < out_chunk; a += piece)
                ok(cudaMemcpyAsync(dchi2 + out_global + a, out + a,
                                   std::min(piece, out_chunk - a) * sizeof(float),
                                   cudaMemcpyDeviceToHost, b.cs2));
            ok(cudaEventRecord(b.ev_copied[slot], b.cs2));
            b.copied_pending[slot] = true;
        } else if (dchi2 && !out_dev) {
            ok(cudaMemcpyAsync(dchi2 + out_global, out, out_chunk * sizeof(float), cudaMemcpyDeviceToHost,
                               s));
        }
        if (b.timing) {
            // stage events are re-recorded by the next chunk: read them now
            ok(cudaStreamSynchronize(s));
            for (int i = 0; i < 5; ++i) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, b.ev[i], b.ev[i + 1]) == cudaSuccess) b.stage_ms[i] += ms;
                cudaGetLastError();
            }
            for (int c = 0; c < nc; ++c) b.fft_alg_bytes += 3.0 * Hv[c] * (double)N * (double)csz;
        }
        b.phase_ms[5] += ms_since(tp3, now());
        if (e != cudaSuccess) { st = map_cuda(e); break; }
        out_global += out_chunk;
    }
    const auto t_loop_end = now();
    cudaStreamSynchronize(s);
    if (b.cs2 && cudaStreamSynchronize(b.cs2) != cudaSuccess && st == FC2_OK) st = FC2_ERR_CUDA;
    if (peaks && K > 0 && launched > 0 && st == FC2_OK) {
        const int64_t ncur = (launched == nchunks) ? C : chunks[launched].c0;
        if (cudaMemcpy(peaks, b.recs, (size_t)ncur * K * sizeof(fc2_best), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            cudaGetLastError();
            st = FC2_ERR_CUDA;
        }
    }
    // ---- every launched chunk's counters: the status word [8], then the list
    // counts (re-solve, float, double-float, last tier; a list that overflowed
    // its capacity leaves bins unrepaired)
    if (launched > 0 && b.cnt_hist &&
        cudaMemcpy(hist.data(), b.cnt_hist, launched * 64, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        if (st == FC2_OK) st = FC2_ERR_CUDA;
        launched = 0;
    }
    for (size_t ci = 0; ci < launched; ++ci) {
        const int32_t* cnts = &hist[16 * ci];
        if (cnts[8] != 0) {
            if (st == FC2_OK) st = (fc2_status)cnts[8];
            break;
        }
        if ((size_t)cnts[0] > b.cl1 || (size_t)cnts[1] > b.cl2 || (size_t)cnts[2] > b.cl3 ||
            (size_t)cnts[3] > b.cl4) {
            if (st == FC2_OK) st = FC2_ERR_NUMERIC;
            break;
        }
        b.stats[0] += cnts[0];
        b.stats[1] += cnts[1];
        b.stats[2] += cnts[2];
        b.stats[3] += cnts[3];
    }
    b.cp.d_key = nullptr; b.cp.d_dlt = nullptr; b.cp.d_cs = nullptr;
    b.cp.d_grid[0] = b.cp.d_grid[1] = nullptr; b.cp.d_spec = nullptr; b.cp.d_L = nullptr;
    b.cp.d_slot_soff = b.cp.d_slot_n = nullptr; b.cp.d_red = nullptr; b.cp.d_status = nullptr;
    if (opt.inputs_on_device) { b.t = b.x = b.sg = nullptr; }
    b.free_all();
    cudaStreamSynchronize(s);
    if (b.own_stream) cudaStreamDestroy(s);
    b.phase_ms[6] = ms_since(t_loop_end, now());
    if (launches_out) *launches_out = b.launches;
    if (stats_out) {
        for (int i = 0; i < 4; ++i) stats_out[i] = b.stats[i];
        stats_out[4] = b.graphs;
        for (int i = 0; i < 7; ++i) std::memcpy(&stats_out[5 + i], &b.phase_ms[i], 8);
        for (int i = 0; i < 5; ++i) std::memcpy(&stats_out[12 + i], &b.stage_ms[i], 8);
        std::memcpy(&stats_out[17], &b.fft_alg_bytes, 8);
        stats_out[18] = b.cfg_source;
        stats_out[19] = b.cfg.fft.family;
        stats_out[20] = b.cfg.spread_tile;
        stats_out[21] = b.cfg.asm_nt;
        stats_out[22] = b.cfg.bx_ch;
        stats_out[23] = (int64_t)b.cfg.fft.rs.size();
        for (int i = 0; i < 4; ++i)
            stats_out[24 + i] = i < (int)b.cfg.fft.rs.size() ? b.cfg.fft.rs[i] : 0;
        stats_out[28] = b.tune_timed;
        stats_out[30] = b.cfg.fft_group;
        std::memcpy(&stats_out[29], &b.tune_ms, 8);
    }
    return st;
}


// Gradients and Newton refinement for K peaks of each of C curves
// (fc2_backward_batched): per-curve moments, time order and the sample
// arrays, then the adjoint kernel over all C K entries.
fc2_status batched_backward(int64_t C, const int64_t* offsets, const double* t, const double* x,
                            const double* sigma, const int* Hc, const double* fminc,
                            const double* dfc, const int64_t* Nc, int K, const int64_t* peak_j,
                            const double* grad_out, const fc2_options& opt, double* f_ref,
                            double* d_ref, double* d_df, double* d_dx, double* d_dsig) {
    if (C < 1 || K < 1 || !offsets || !t || !x || !sigma || !Hc || !fminc || !dfc || !Nc || !peak_j)
        return FC2_ERR_INVALID_ARG;
    for (int64_t c = 0; c < C; ++c) {
        if (offsets[c + 1] - offsets[c] < 1 || offsets[c] < 0) return FC2_ERR_INVALID_ARG;
        if (Hc[c] < 1 || Hc[c] > FC2_MAX_H || Nc[c] < 2) return FC2_ERR_INVALID_ARG;
        if (Hc[c] > 8) return FC2_ERR_UNSUPPORTED;
        if (!(std::isfinite(fminc[c]) && fminc[c] >= 0.0) || !(std::isfinite(dfc[c]) && dfc[c] > 0.0))
            return FC2_ERR_INVALID_ARG;
        for (int k = 0; k < K; ++k)
            if (peak_j[c * K + k] < 0 || peak_j[c * K + k] >= Nc[c]) return FC2_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return FC2_ERR_CUDA;
    if (opt.device < 0 || opt.device >= ndev) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(opt.device) != cudaSuccess) return FC2_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)opt.cuda_stream;
    bool own = false;
    if (!s) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FC2_ERR_CUDA;
        own = true;
    }
    const int64_t base = offsets[0], ntot = offsets[C] - base;
    const int64_t E = C * K;
    auto is_dev = [&](const void* q) {
        cudaPointerAttributes at;
        bool d = q && cudaPointerGetAttributes(&at, q) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        return d;
    };
    std::vector<void*> owned;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = pool_alloc((void**)p, std::max<size_t>(bytes, 64), s);
        if (e == cudaSuccess) owned.push_back(*p);
    };
    double *dt = nullptr, *dx = nullptr, *ds = nullptr;
    if (opt.inputs_on_device) { dt = (double*)(t + base); dx = (double*)(x + base); ds = (double*)(sigma + base); }
    else {
        alloc((void**)&dt, ntot * 8); alloc((void**)&dx, ntot * 8); alloc((void**)&ds, ntot * 8);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(dt, t + base, ntot * 8, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(dx, x + base, ntot * 8, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(ds, sigma + base, ntot * 8, cudaMemcpyHostToDevice, s);
        }
    }
    int64_t* off = nullptr; int* Hd = nullptr; double *fm = nullptr, *dfd = nullptr, *scal = nullptr;
    int32_t *perm = nullptr, *status = nullptr; double *tau = nullptr, *wq = nullptr, *wp = nullptr;
    uint64_t *A = nullptr, *B = nullptr; float *w32 = nullptr, *p32 = nullptr;
    int64_t* ent = nullptr; double* g = nullptr;
    double *of = nullptr, *od = nullptr, *og = nullptr, *oxx = nullptr, *oss = nullptr;
    alloc((void**)&off, (C + 1) * 8); alloc((void**)&Hd, C * 4); alloc((void**)&fm, C * 8);
    alloc((void**)&dfd, C * 8); alloc((void**)&scal, C * SC_COUNT * 8); alloc((void**)&status, 16);
    alloc((void**)&perm, ntot * 4); alloc((void**)&tau, ntot * 8); alloc((void**)&wq, ntot * 8);
    alloc((void**)&wp, ntot * 8); alloc((void**)&A, ntot * 8); alloc((void**)&B, ntot * 8);
    // float weights: high parts at [i], low parts at [ntot + i]
    alloc((void**)&w32, 2 * ntot * 4); alloc((void**)&p32, 2 * ntot * 4);
    alloc((void**)&ent, E * 8);
    alloc((void**)&of, E * 8); alloc((void**)&od, E * 8); alloc((void**)&og, E * 8);
    if (grad_out) alloc((void**)&g, E * 8);
    const bool dx_dev = is_dev(d_dx), ds_dev = is_dev(d_dsig);
    if (d_dx && !dx_dev) alloc((void**)&oxx, (size_t)K * ntot * 8);
    if (d_dsig && !ds_dev) alloc((void**)&oss, (size_t)K * ntot * 8);
    int64_t nmax = 0;
    std::vector<int64_t> offl(C + 1), entv(E);
    for (int64_t c = 0; c <= C; ++c) offl[c] = offsets[c] - base;
    for (int64_t c = 0; c < C; ++c) {
        nmax = std::max(nmax, offl[c + 1] - offl[c]);
        for (int k = 0; k < K; ++k) entv[c * K + k] = (c << 32) | peak_j[c * K + k];
    }
    fc2_status st = FC2_OK;
    if (e == cudaSuccess) {
        cudaMemcpyAsync(off, offl.data(), (C + 1) * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(Hd, Hc, C * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(fm, fminc, C * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dfd, dfc, C * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ent, entv.data(), E * 8, cudaMemcpyHostToDevice, s);
        if (grad_out) cudaMemcpyAsync(g, grad_out, E * 8, cudaMemcpyDefault, s);
        cudaMemsetAsync(status, 0, 16, s);
        launch_moments(dt, dx, ds, off, C, 0, scal, status, s);
        std::vector<double> hs((size_t)C * SC_COUNT);
        int32_t hst = 0;
        cudaMemcpyAsync(hs.data(), scal, hs.size() * 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && hst) st = (fc2_status)hst;
        if (e == cudaSuccess && st == FC2_OK) {
            k_iota_plus<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(perm, ntot, 0);
            char* scratch = nullptr;
            const size_t sb = sort_scratch_bytes(nmax) + 4096;
            for (int64_t c = 0; c < C && e == cudaSuccess; ++c)
                if (hs[c * SC_COUNT + SC_SORTED] == 0.0) {
                    if (!scratch) { alloc((void**)&scratch, sb); if (e != cudaSuccess) break; }
                    const int64_t n = offl[c + 1] - offl[c];
                    e = sort_by_time(dt + offl[c], n, perm + offl[c], scratch, sb, s);
                    k_add_base<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm + offl[c], n, offl[c]);
                }
            k_bgather<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(dt, dx, ds, perm, ntot, off, (int)C,
                                                                    scal, fm, dfd, tau, wq, wp, A, B,
                                                                    w32, p32);
            AdjTab tb{off, Hd, fm, dfd, scal, tau, wq, wp, perm, ent, g, K, 1e-10, 40};
            AdjOut out{of, od, og, d_dx ? (dx_dev ? d_dx : oxx) : nullptr,
                       d_dsig ? (ds_dev ? d_dsig : oss) : nullptr};
            if (e == cudaSuccess) e = launch_backward_tab(tb, E, out, s);
            if (e == cudaSuccess) {
                if (f_ref) cudaMemcpyAsync(f_ref, of, E * 8, cudaMemcpyDefault, s);
                if (d_ref) cudaMemcpyAsync(d_ref, od, E * 8, cudaMemcpyDefault, s);
                if (d_df) cudaMemcpyAsync(d_df, og, E * 8, cudaMemcpyDefault, s);
                if (d_dx && !dx_dev) cudaMemcpyAsync(d_dx, oxx, (size_t)K * ntot * 8, cudaMemcpyDeviceToHost, s);
                if (d_dsig && !ds_dev) cudaMemcpyAsync(d_dsig, oss, (size_t)K * ntot * 8, cudaMemcpyDeviceToHost, s);
                e = cudaStreamSynchronize(s);
            }
        }
    }
    for (void* q : owned) cudaFreeAsync(q, s);
    cudaStreamSynchronize(s);
    if (own) cudaStreamDestroy(s);
    if (st != FC2_OK) return st;
    return map_cuda(e);
}

}  // namespace fc2
