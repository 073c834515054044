// fc2_df.cuh -- double-float ("float-float") arithmetic for the exact sums.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// which carries about 48 significant bits.  The error-free transformations are
// Knuth's two-sum and the fused multiply-add product error (Dekker, Numer.
// Math. 18 (1971) 224; Joldes, Muller & Popescu, ACM TOMS 44 (2017) 48).  The
// float pipes of this part are some sixty times wider than its double pipe,
// so sums that need more than float but less than double precision are
// cheaper this way.  Not part of the public ABI.
#pragma once
#include "fc2_common.cuh"

namespace fc2 {

struct dfl {
    float h, l;
};
struct dfc {
    dfl re, im;
};

// s + e = a + b exactly (any magnitudes)
FC2_D dfl df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return dfl{s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly, for |a| >= |b| (or a == 0)
FC2_D dfl df_fast_sum(float a, float b) {
    const float s = a + b;
    return dfl{s, b - (s - a)};
}
// a * b, relative error ~2^-47
FC2_D dfl df_mul(dfl a, dfl b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_fast_sum(p, e);
}

// a * b for double-float complex numbers of modulus about one; each component
// is formed as one two-sum of the leading products plus the small terms, so
// its absolute error is ~2^-47 |a| |b|.
FC2_D dfc dfc_mul(const dfc& a, const dfc& b) {
    dfc r;
    {
        const float p1 = a.re.h * b.re.h, p2 = a.im.h * b.im.h;
        const float e1 = fmaf(a.re.h, b.re.h, -p1), e2 = fmaf(a.im.h, b.im.h, -p2);
        const dfl s = df_two_sum(p1, -p2);
        float lo = s.l + (e1 - e2);
        lo = fmaf(a.re.h, b.re.l, lo);
        lo = fmaf(a.re.l, b.re.h, lo);
        lo = fmaf(-a.im.h, b.im.l, lo);
        lo = fmaf(-a.im.l, b.im.h, lo);
        r.re = df_two_sum(s.h, lo);
    }
    {
        const float p1 = a.re.h * b.im.h, p2 = a.im.h * b.re.h;
        const float e1 = fmaf(a.re.h, b.im.h, -p1), e2 = fmaf(a.im.h, b.re.h, -p2);
        const dfl s = df_two_sum(p1, p2);
        float lo = s.l + (e1 + e2);
        lo = fmaf(a.re.h, b.im.l, lo);
        lo = fmaf(a.re.l, b.im.h, lo);
        lo = fmaf(a.im.h, b.re.l, lo);
        lo = fmaf(a.im.l, b.re.h, lo);
        r.im = df_two_sum(s.h, lo);
    }
    return r;
}

// Accumulator acc += w * z (w, z double-float reals); the running sum keeps
// its rounding errors in acc.l.
FC2_D void df_acc_mul(dfl& acc, dfl w, dfl z) {
    const float p = w.h * z.h;
    float e = fmaf(w.h, z.h, -p);
    e = fmaf(w.h, z.l, e);
    e = fmaf(w.l, z.h, e);
    const dfl s = df_two_sum(acc.h, p);
    acc.h = s.h;
    acc.l += s.l + e;
}

FC2_D dfl df_from_double(double v) {
    const float h = (float)v;
    return dfl{h, (float)(v - (double)h)};
}

// z (1 + eps + i s) for a double-float z of modulus about one and a small
// rotation: eps a float of modulus below 2^-27, s a double-float below 1e-4.
// Each component is z's plus one double-float product (leading product, its
// FMA error and the cross terms) and the float eps term, gathered by two-sums:
// absolute error ~2^-47, like dfc_mul, with fewer operations.
FC2_D dfc dfc_rot_small(const dfc& z, float eps, dfl s) {
    dfc r;
    {
        const float p = z.im.h * s.h;  // z.im s
        float e = fmaf(z.im.h, s.h, -p);
        e = fmaf(z.im.h, s.l, e);
        e = fmaf(z.im.l, s.h, e);
        const dfl t = df_two_sum(z.re.h, -p);
        const float lo = fmaf(z.re.h, eps, (t.l + z.re.l) - e);
        r.re = df_two_sum(t.h, lo);
    }
    {
        const float p = z.re.h * s.h;  // z.re s
        float e = fmaf(z.re.h, s.h, -p);
        e = fmaf(z.re.h, s.l, e);
        e = fmaf(z.re.l, s.h, e);
        const dfl t = df_two_sum(z.im.h, p);
        const float lo = fmaf(z.im.h, eps, (t.l + z.im.l) + e);
        r.im = df_two_sum(t.h, lo);
    }
    return r;
}

// e^{2 pi i u 2^-64} for a 64-bit phase u, to ~2^-46: the top 16 bits select
// two table factors e^{2 pi i a / 256} and e^{2 pi i b / 65536} (double-float,
// t1[a] and t2[b]); the remaining 48 bits give theta = 2 pi delta < 1e-4 and
// e^{i theta} = 1 - theta^2/2 + i (theta - theta^3/6) (the next terms are
// below 1e-17).  theta^2/2 < 4.6e-9 lies below half an ulp of 1, so the real
// part is 1 plus a float correction (float theta^2: 3e-16 absolute), and the
// product with the table factors is a small rotation (dfc_rot_small).
FC2_D dfc df_phasor(uint64_t u, const dfc* t1, const dfc* t2) {
    const int a = (int)(u >> 56), b = (int)((u >> 48) & 255u);
    const uint64_t r = u & ((1ull << 48) - 1);
    const float rh = (float)(uint32_t)(r >> 24), rl = (float)(uint32_t)(r & 0xffffffu);
    const dfl d = df_two_sum(rh * 9.094947017729282e-13f, rl * 5.421010862427522e-20f);  // 2^-40, 2^-64
    const dfl th = df_mul(d, dfl{6.28318548202514648f, -1.74845553146951525e-07f});  // 2 pi
    const float eps = -0.5f * th.h * th.h;
    const float t3 = th.h * th.h * th.h * (1.0f / 6.0f);
    const dfl s = df_fast_sum(th.h, th.l - t3);
    return dfc_rot_small(dfc_mul(t1[a], t2[b]), eps, s);
}

// e^{2 pi i u 2^-64} for a 64-bit phase u, to ~2^-46, from one table of
// 65536 double-float entries e^{2 pi i m / 65536} (t16[m], m = the top 16 bits;
// 1 MB, read through the caches) and the same small rotation by the remaining
// 48 bits as df_phasor: the product of two table factors (df_phasor's
// dfc_mul) is not needed.
FC2_D dfc df_phasor16(uint64_t u, const dfc* __restrict__ t16) {
    const int m = (int)(u >> 48);
    const uint64_t r = u & ((1ull << 48) - 1);
    const float rh = (float)(uint32_t)(r >> 24), rl = (float)(uint32_t)(r & 0xffffffu);
    const dfl d = df_two_sum(rh * 9.094947017729282e-13f, rl * 5.421010862427522e-20f);  // 2^-40, 2^-64
    const dfl th = df_mul(d, dfl{6.28318548202514648f, -1.74845553146951525e-07f});  // 2 pi
    const float eps = -0.5f * th.h * th.h;
    const float t3 = th.h * th.h * th.h * (1.0f / 6.0f);
    const dfl s = df_fast_sum(th.h, th.l - t3);
    return dfc_rot_small(t16[m], eps, s);
}

// e^{2 pi i u 2^-64} in double from the same split as df_phasor: two table
// factors times 1 - theta^2/2 + i (theta - theta^3/6), theta < 1e-4 (the
// dropped terms are below 4e-18).
FC2_D double2 d_phasor(uint64_t u, const double2* t1, const double2* t2) {
    const double2 A = t1[(int)(u >> 56)], B = t2[(int)((u >> 48) & 255u)];
    const double th = (double)(int64_t)(u & ((1ull << 48) - 1)) * 3.4061215800865545e-19;  // 2 pi 2^-64
    const double th2 = th * th;
    const double c = fma(-0.5, th2, 1.0);
    const double s = fma(th * th2, -1.0 / 6.0, th);
    const double pr = fma(A.x, B.x, -A.y * B.y), pi = fma(A.x, B.y, A.y * B.x);
    return make_double2(fma(pr, c, -pi * s), fma(pr, s, pi * c));
}

// ---------------------------------------------- sums exact in fixed point
// The last precision tier of the exact fix-up keeps the float pipes' speed but
// none of their accumulation error: each harmonic multiple's phasor is
// evaluated directly from its exact integer phase k u (df_phasor or
// df_phasor16, ~2^-46, no chains of products), the products with the double-float weights are summed
// in double-float over blocks of FX_BLOCK samples, and every block sum enters
// a 64-bit integer accumulator at a fixed scale 2^s -- integer additions are
// exact and associative, so the result does not depend on the order and the
// only errors are the per-term ones (phasor, product, block, and the
// conversion's rounding at 2^-s).
constexpr int FX_BLOCK = 8;

// Scale exponent s for sums of at most nterm terms of modulus <= vmax: the
// scaled terms add up to less than 2^61 in modulus, and so does every partial
// sum of the converted block pieces (each at most its terms' sum plus half a
// unit of rounding), far inside the 64-bit range.  Clamped to the float
// exponent range.
FC2_D int fx_exponent(float vmax, int64_t nterm) {
    const int ev = (vmax > 0.0f) ? ilogbf(vmax) + 1 : 0;  // vmax < 2^ev
    int en = 0;
    while ((1ll << en) < nterm) ++en;
    int s = 61 - ev - en;
    if (s > 126) s = 126;
    if (s < -126) s = -126;
    return s;
}

FC2_D void fx_flush(long long& acc, dfl& blk, float scale) {
    acc += __float2ll_rn(blk.h * scale) + __float2ll_rn(blk.l * scale);
    blk = dfl{0.f, 0.f};
}

// One lane's sums over samples i = i0 + start, + step, .. < i1 of multiple k
// (phasors by df_phasor16 from the table t1 when T16, else by df_phasor from
// the tables t1, t2; the two differ by float rounding, both ~2^-46):
// acc[0..1] = sum w e^{2 pi i k u_i} (re, im) and, when with_p, acc[2..3] the
// same with the weighted data; u_i = A_i + ju B_i (mod 2^64).  Weights as float
// high parts at [i] and low parts at [ntot + i]; sq, sp = 2^s of each kind.
template <bool T16>
FC2_D void fx_lane_sums(const uint64_t* __restrict__ Aph, const uint64_t* __restrict__ Bph,
                        const float* __restrict__ wq32, const float* __restrict__ wp32,
                        int64_t ntot, uint64_t ju, uint64_t k, int64_t i0, int64_t i1,
                        int64_t start, int64_t step, bool with_p, const dfc* __restrict__ t1,
                        const dfc* __restrict__ t2, float sq, float sp, long long acc[4]) {
    dfl b0{0.f, 0.f}, b1{0.f, 0.f}, b2{0.f, 0.f}, b3{0.f, 0.f};
    int cnt = 0;
    for (int64_t i = i0 + start; i < i1; i += step) {
        const uint64_t u = k * (Aph[i] + ju * Bph[i]);
        const dfc z = T16 ? df_phasor16(u, t1) : df_phasor(u, t1, t2);
        const dfl a{wq32[i], wq32[ntot + i]};
        df_acc_mul(b0, a, z.re);
        df_acc_mul(b1, a, z.im);
        if (with_p) {
            const dfl b{wp32[i], wp32[ntot + i]};
            df_acc_mul(b2, b, z.re);
            df_acc_mul(b3, b, z.im);
        }
        if (++cnt == FX_BLOCK) {
            fx_flush(acc[0], b0, sq);
            fx_flush(acc[1], b1, sq);
            if (with_p) {
                fx_flush(acc[2], b2, sp);
                fx_flush(acc[3], b3, sp);
            }
            cnt = 0;
        }
    }
    fx_flush(acc[0], b0, sq);
    fx_flush(acc[1], b1, sq);
    if (with_p) {
        fx_flush(acc[2], b2, sp);
        fx_flush(acc[3], b3, sp);
    }
}

FC2_D float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Every lane receives the warp's sum of (hi, lo) float pairs (butterfly of
// error-free two-sums; two-sum is symmetric in its operands, so all lanes end
// with the same bits).
FC2_D float2 warp_allsum_pair(float hi, float lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const dfl t = df_two_sum(hi, h2);
        hi = t.h;
        lo = (lo + l2) + t.l;
    }
    return make_float2(hi, lo);
}

}  // namespace fc2
