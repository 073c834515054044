// fc2_common.cuh -- shared device helpers of libfc2 (complex arithmetic, small
// DFTs, the spreading kernel, status reporting).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/fc2.h"

#define FC2_HD __host__ __device__ __forceinline__
#define FC2_D __device__ __forceinline__

namespace fc2 {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T x, y;
};

template <typename T> FC2_HD cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> FC2_HD cpx<T> add(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> FC2_HD cpx<T> sub(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> FC2_HD cpx<T> mul(cpx<T> a, cpx<T> b) {
    return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T> FC2_HD cpx<T> mul_i(cpx<T> a) { return mk(-a.y, a.x); }   // i * a
template <typename T> FC2_HD cpx<T> mul_mi(cpx<T> a) { return mk(a.y, -a.x); }  // -i * a
template <typename T> FC2_HD cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T> FC2_HD cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }

// Compile-time e^{+2 pi i k / Q} for Q | 16, from exact closed forms.
template <typename T>
FC2_HD cpx<T> root16(int k) {
    // k in [0, 16); cos/sin of k*pi/8
    const T c1 = (T)0.92387953251128675613;  // cos(pi/8)
    const T s1 = (T)0.38268343236508977173;  // sin(pi/8)
    const T r2 = (T)0.70710678118654752440;  // cos(pi/4)
    const T cs[5] = {(T)1, c1, r2, s1, (T)0};
    int q = k & 15;
    int quad = q >> 2, rem = q & 3;
    T c = cs[rem], s = cs[4 - rem];
    // rotate by quad * pi/2
    if (quad == 0) return mk(c, s);
    if (quad == 1) return mk(-s, c);
    if (quad == 2) return mk(-c, -s);
    return mk(s, -c);
}

// e^{+2 pi i k / 64} from cos(k pi / 32), k = 0..16 (double literals).
template <typename T>
FC2_HD cpx<T> root64(int k) {
    const double c[17] = {1.0, 0.99518472667219689, 0.98078528040323043, 0.95694033573220882,
                          0.92387953251128674, 0.88192126434835505, 0.83146961230254524,
                          0.77301045336273699, 0.70710678118654757, 0.63439328416364549,
                          0.55557023301960229, 0.47139673682599781, 0.38268343236508984,
                          0.29028467725446233, 0.19509032201612833, 0.098017140329560604, 0.0};
    const int q = k & 63;
    const int quad = q >> 4, rem = q & 15;
    const T cs = (T)c[rem], sn = (T)c[16 - rem];
    if (quad == 0) return mk(cs, sn);
    if (quad == 1) return mk(-sn, cs);
    if (quad == 2) return mk(-cs, -sn);
    return mk(sn, -cs);
}

// In-register DFT of length Q (power of two <= 64), sign +: X_k = sum_n x_n e^{+2 pi i n k / Q}.
template <typename T, int Q>
struct SmallDFT {
    static FC2_D void run(cpx<T>* v) {
        cpx<T> e[Q / 2], o[Q / 2];
#pragma unroll
        for (int i = 0; i < Q / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
        SmallDFT<T, Q / 2>::run(e);
        SmallDFT<T, Q / 2>::run(o);
#pragma unroll
        for (int k = 0; k < Q / 2; ++k) {
            cpx<T> t;
            if (k == 0) t = o[k];
            else if (4 * k == Q) t = mul_i(o[k]);
            else if constexpr (Q <= 16) t = mul(o[k], root16<T>(k * (16 / Q)));
            else t = mul(o[k], root64<T>(k * (64 / Q)));
            v[k] = add(e[k], t);
            v[k + Q / 2] = sub(e[k], t);
        }
    }
};
template <typename T>
struct SmallDFT<T, 1> { static FC2_D void run(cpx<T>*) {} };
template <typename T>
struct SmallDFT<T, 2> {
    static FC2_D void run(cpx<T>* v) {
        cpx<T> a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    }
};
template <typename T>
struct SmallDFT<T, 4> {
    static FC2_D void run(cpx<T>* v) {
        cpx<T> a = add(v[0], v[2]), b = sub(v[0], v[2]);
        cpx<T> c = add(v[1], v[3]), d = sub(v[1], v[3]);
        v[0] = add(a, c);
        v[2] = sub(a, c);
        v[1] = add(b, mul_i(d));
        v[3] = sub(b, mul_i(d));
    }
};

// Exponential-of-semicircle spreading kernel (Barnett, Magland & af Klinteberg,
// SIAM J. Sci. Comput. 41 (2019) C479):  phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1))
// for |z| < w/2, zero outside.  beta = 0.97 pi (1 - 1/(2 sigma)) w.
FC2_HD double es_beta(int w, int oversample) {
    return 0.97 * 3.14159265358979323846 * (1.0 - 0.5 / (double)oversample) * (double)w;
}

template <typename T>
FC2_D T es_kernel(T z, T inv_half_w, T beta) {
    T s = z * inv_half_w;
    T a = (T)1 - s * s;
    return a > (T)0 ? exp(beta * (sqrt(a) - (T)1)) : (T)0;
}
template <>
FC2_D float es_kernel<float>(float z, float inv_half_w, float beta) {
    float s = z * inv_half_w;
    float a = 1.0f - s * s;
    return a > 0.0f ? expf(beta * (sqrtf(a) - 1.0f)) : 0.0f;
}

// Device status word: first error code wins.
// Exact float -> double conversion on the integer pipes (the double pipe of
// this part is narrow).  Handles zeros, subnormals, infinities and NaN.
FC2_D double f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    uint32_t e = (b >> 23) & 0xffu, man = b & 0x7fffffu;
    uint64_t r;
    if (e == 0xffu) {
        r = sign | (0x7ffull << 52) | ((uint64_t)man << 29);
    } else if (e != 0) {
        r = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)man << 29);
    } else if (man == 0) {
        r = sign;
    } else {  // subnormal float: normalise
        const int sh = __clz(man) - 8;  // shift that moves the leading 1 to bit 23
        man = (man << sh) & 0x7fffffu;
        r = sign | ((uint64_t)(897u - (uint32_t)sh) << 52) | ((uint64_t)man << 29);
    }
    return __longlong_as_double((long long)r);
}

// double -> float on the integer pipes, truncating the mantissa (relative
// error below 2^-23); for finite v >= 0 -- values below the float range give
// 0, values above it +inf.
FC2_D float d2f_trunc(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __int_as_float(0x7f800000);
    return __uint_as_float(((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
}

FC2_D void set_status(int* st, int code) {
    if (st) atomicCAS(st, 0, code);
}

// Neumaier-compensated accumulator.
template <typename T>
struct CompSum {
    T s, c;
    FC2_D void init() { s = (T)0; c = (T)0; }
    FC2_D void add(T v) {
        T t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    FC2_D T val() const { return s + c; }
};

}  // namespace fc2
