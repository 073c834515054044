// k_adjoint.cu -- exact gradients and Newton refinement at peaks.
//
// Sec. 3e: near the best and the nearly-as-good frequencies the search should
// be refined "using the ungridded data".  For each requested peak (curve c,
// bin j) one CTA works straight from the samples, in double:
//   * chi^2(A, f) = sum_i w_i (x'_i - sum_l A_l M_l(f, tau_i))^2 (Sec. 2, Eq.
//     "eqchigen" with the Eq. "eqtrunc" basis, x' = x - xbar), minimised over A
//     by the normal equations (Eq. "eqchix");
//   * gradients of Delta = chi2_0 - chi2_min at the bin frequency by the
//     envelope theorem (the minimisers xbar and A need not be differentiated):
//       dDelta/dx_i     = 2 w_i (m_i - xbar)
//       dDelta/dsigma_i = -2 sigma_i^-3 [(x_i - xbar)^2 - (x_i - m_i)^2]
//       dDelta/df       = 2 sum_i w_i r_i m_f,i,  r = x' - m', m_f = d m'/df;
//   * Newton steps on f with the exact second derivative of chi2_min(f),
//       d2 chi2_min/df2 = 2 sum w (m_f^2 - r m_ff) - 2 V^T alpha^-1 V,
//       V_l = sum w (M_l m_f - r dM_l/df)  (Schur complement of the joint
//     Hessian in (A, f)), safeguarded to stay within one bin of the start and
//     to increase Delta.
#include <cuda_runtime.h>

#include <vector>

#include "fc2_common.cuh"
#include "fc2_internal.h"
#include "fc2_solve.cuh"

namespace fc2 {

constexpr int AD_NT = 256;
constexpr int AD_HM = 8;

// Block sum of NV values; result valid on all threads after the call.
template <int NV, int STRIDE>
FC2_D void block_sum(double* v, double (*red)[STRIDE], double* tot) {
    static_assert(NV <= STRIDE, "reduction buffer too small");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double y = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
        if (lane == 0) red[w][q] = y;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double y = 0.0;
        for (int q = 0; q < AD_NT / 32; ++q) y += red[q][threadIdx.x];
        tot[threadIdx.x] = y;
    }
    __syncthreads();
}

// e^{2 pi i f tau} with the phase frac(f tau) reduced exactly (fixed point).
FC2_D void unit_phasor(double f, double tau, double* c, double* s) {
    const int64_t ph = (int64_t)frac_fx(f, tau);
    sincospi(ldexp((double)ph, -63), s, c);
}

__global__ void __launch_bounds__(AD_NT) k_backward(AdjTab tb, int64_t E, AdjOut out) {
    constexpr int NQ = 6 * AD_HM;          // Q_1..Q_2H, P_1..P_H (re, im)
    constexpr int M1 = 2 * AD_HM + 1;
    constexpr int NB = 2 + M1;             // S1, S2, V_0..V_2H
    __shared__ double red[AD_NT / 32][NQ];
    __shared__ double tot[NQ];
    __shared__ double qsum[NQ];            // trigonometric sums at the current best f
    __shared__ double coef[M1];            // coefficients (tau frame, absolute units)
    __shared__ double sh_f, sh_fbest, sh_dbest, sh_step;
    __shared__ int sh_state;               // 0 continue, 1 backtracked, 2 done
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int c = (int)(tb.ent[e] >> 32);
        const int64_t j = tb.ent[e] & 0xffffffffll;
        const int H = tb.H[c];
        const int m = 2 * H + 1;
        const double* sc = tb.scal + (int64_t)c * SC_COUNT;
        const double W = sc[SC_W], chi0 = sc[SC_CHI0];
        const int64_t a0 = tb.off[c], a1 = tb.off[c + 1], n = a1 - a0;
        const double g_up = tb.gout ? tb.gout[e] : 1.0;
        const double df = tb.df[c];
        const double f0 = tb.fmin[c] + (double)j * df;
        const double lo = f0 - df, hi = f0 + df;
        const int r_in = (int)(e % (tb.K > 0 ? tb.K : 1));
        if (threadIdx.x == 0) { sh_f = f0; sh_fbest = f0; sh_dbest = -INFINITY; sh_step = 0.0; sh_state = 0; }
        __syncthreads();
        for (int it = 0; it <= tb.max_iter; ++it) {
            const double f = sh_f;
            // ---- pass A: trigonometric sums at f (Eq. "eqPQ") and the solve
            double acc[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
            for (int64_t i = a0 + threadIdx.x; i < a1; i += AD_NT) {
                double c1, s1;
                unit_phasor(f, tb.tau[i], &c1, &s1);
                double cr = c1, ci = s1;
                const double a = tb.wq[i], b = tb.wp[i];
#pragma unroll
                for (int k = 0; k < 2 * AD_HM; ++k) {
                    if (k < 2 * H) {
                        acc[2 * k] = fma(a, cr, acc[2 * k]);
                        acc[2 * k + 1] = fma(a, ci, acc[2 * k + 1]);
                        if (k < H) {
                            acc[4 * AD_HM + 2 * k] = fma(b, cr, acc[4 * AD_HM + 2 * k]);
                            acc[4 * AD_HM + 2 * k + 1] = fma(b, ci, acc[4 * AD_HM + 2 * k + 1]);
                        }
                        const double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                        cr = nr;
                        ci = ni;
                    }
                }
            }
            block_sum<NQ, NQ>(acc, red, tot);
            if (threadIdx.x == 0) {
                Sys<double, AD_HM> S;
                exact_sys_from_sums<AD_HM>(tot, H, sc, S);
                double o[AD_HM], an2;
                double L[M1][M1], z[M1];
                chol_solve<double, AD_HM, false>(S, 1e-13, o, &an2, L, z);
                const double dv = o[H - 1] * chi0;
                if (it > 0 && dv < sh_dbest) {
                    // the step lowered Delta: halve it from the best point
                    sh_step *= 0.5;
                    sh_f = sh_fbest + sh_step;
                    sh_state = (fabs(sh_step) < tb.tol) ? 2 : 1;
                } else {
                    sh_fbest = f;
                    sh_dbest = dv;
                    sh_state = 0;
                    double A[M1];
                    for (int l = m - 1; l >= 0; --l) {
                        double s = z[l];
                        for (int k = l + 1; k < m; ++k) s -= L[k][l] * A[k];
                        A[l] = (L[l][l] > 0.0) ? s / L[l][l] : 0.0;
                    }
                    const double unit = (W > 0.0) ? sqrt(chi0 / W) : 0.0;
                    for (int l = 0; l < M1; ++l) coef[l] = (l < m) ? A[l] * unit : 0.0;
                    for (int q = 0; q < NQ; ++q) qsum[q] = tot[q];
                }
            }
            __syncthreads();
            if (sh_state == 2 || it == tb.max_iter) break;
            if (sh_state == 1) continue;
            // ---- pass B: model, residual and f-derivatives at the best f
            double bs[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) bs[q] = 0.0;
            for (int64_t i = a0 + threadIdx.x; i < a1; i += AD_NT) {
                const double ta = tb.tau[i];
                double c1, s1;
                unit_phasor(f, ta, &c1, &s1);
                double cr = c1, ci = s1;
                const double w = tb.wq[i], xp = tb.wp[i] / w;  // x - xbar
                double mv = coef[0], mf = 0.0, mff = 0.0;
                double Ml[M1], dMl[M1];
                Ml[0] = 1.0;
                dMl[0] = 0.0;
#pragma unroll
                for (int h = 1; h <= AD_HM; ++h) {
                    Ml[2 * h - 1] = 0.0; Ml[2 * h] = 0.0; dMl[2 * h - 1] = 0.0; dMl[2 * h] = 0.0;
                    if (h <= H) {
                        const double om = 2.0 * M_PI * (double)h * ta;
                        const double as = coef[2 * h - 1], ac = coef[2 * h];
                        mv += as * ci + ac * cr;
                        mf += om * (as * cr - ac * ci);
                        mff -= om * om * (as * ci + ac * cr);
                        Ml[2 * h - 1] = ci;
                        Ml[2 * h] = cr;
                        dMl[2 * h - 1] = om * cr;
                        dMl[2 * h] = -om * ci;
                        const double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                        cr = nr;
                        ci = ni;
                    }
                }
                const double r = xp - mv;
                bs[0] += w * r * mf;
                bs[1] += w * (mf * mf - r * mff);
#pragma unroll
                for (int l = 0; l < M1; ++l) bs[2 + l] += w * (Ml[l] * mf - r * dMl[l]);
                if (it == 0) {
                    // gradients at the bin frequency, in the caller's sample order
                    const int64_t src = tb.perm ? (int64_t)tb.perm[i] : i;
                    const int64_t o = (int64_t)tb.K * a0 + (int64_t)r_in * n + (src - a0);
                    if (out.d_dx) out.d_dx[o] = g_up * 2.0 * w * mv;
                    if (out.d_dsig) out.d_dsig[o] = g_up * (-2.0 * w * sqrt(w)) * (xp * xp - r * r);
                }
            }
            block_sum<NB, NQ>(bs, red, tot);
            if (threadIdx.x == 0) {
                const double S1 = tot[0], S2 = tot[1];
                const double g = 2.0 * S1;  // dDelta/df
                if (it == 0 && out.d_df) out.d_df[e] = g_up * g;
                // V^T alpha^-1 V = W |L'^-1 (V / W)|^2 with alpha' = alpha / W = L' L'^T
                Sys<double, AD_HM> S;
                exact_sys_from_sums<AD_HM>(qsum, H, sc, S);
                double L[M1][M1], dinv[M1], y[M1];
                for (int l = 0; l < m; ++l) {
                    for (int k = 0; k < l; ++k) {
                        double s = S.alpha(l, k);
                        for (int p = 0; p < k; ++p) s -= L[l][p] * L[k][p];
                        L[l][k] = s * dinv[k];
                    }
                    const double all = S.alpha(l, l);
                    double d = all;
                    for (int p = 0; p < l; ++p) d -= L[l][p] * L[l][p];
                    if (all > 0.0 && d > 1e-13 * all) { L[l][l] = sqrt(d); dinv[l] = 1.0 / L[l][l]; }
                    else { L[l][l] = 0.0; dinv[l] = 0.0; }
                    double s = tot[2 + l] / W;
                    for (int p = 0; p < l; ++p) s -= L[l][p] * y[p];
                    y[l] = s * dinv[l];
                }
                double q = 0.0;
                for (int l = 0; l < m; ++l) q += y[l] * y[l];
                const double gpp = -(2.0 * S2 - 2.0 * W * q);  // d2 Delta / df2
                double step;
                if (gpp < 0.0) step = -g / gpp;
                else step = (g >= 0.0 ? 0.25 : -0.25) * df;  // not concave: move uphill
                if (step > 0.5 * df) step = 0.5 * df;
                if (step < -0.5 * df) step = -0.5 * df;
                double fn = f + step;
                if (fn < lo) fn = lo;
                if (fn > hi) fn = hi;
                sh_step = fn - f;
                if (fabs(sh_step) < tb.tol) {
                    sh_fbest = fn;  // converged: the last Newton update
                    sh_state = 2;
                } else {
                    sh_f = fn;
                    sh_state = 0;
                }
            }
            __syncthreads();
            if (sh_state == 2) break;
        }
        if (threadIdx.x == 0) {
            if (out.f_ref) out.f_ref[e] = sh_fbest;
            if (out.d_ref) out.d_ref[e] = sh_dbest;
        }
        __syncthreads();
    }
}

cudaError_t launch_backward_tab(const AdjTab& tb, int64_t E, const AdjOut& out, cudaStream_t s) {
    int blocks = (int)std::min<int64_t>(E, 4 * 152);
    if (blocks < 1) blocks = 1;
    k_backward<<<blocks, AD_NT, 0, s>>>(tb, E, out);
    return cudaGetLastError();
}

}  // namespace fc2

namespace fc2 {

// Host side of fc2_backward for one plan: entries (0 << 32 | j), outputs to
// the caller's buffers (device in place, host through staging).
fc2_status plan_backward(fc2_plan_s* p, int K, const int64_t* peak_j, const double* grad_out,
                         double* f_ref, double* d_ref, double* d_df, double* d_dx,
                         double* d_dsig) {
    if (!p || K < 1 || !peak_j) return FC2_ERR_INVALID_ARG;
    if (p->H > AD_HM) return FC2_ERR_UNSUPPORTED;
    for (int k = 0; k < K; ++k)
        if (peak_j[k] < 0 || peak_j[k] >= p->N) return FC2_ERR_INVALID_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return FC2_ERR_CUDA;
    cudaStream_t s = p->stream;
    const int64_t n = p->n;
    auto is_dev = [&](const void* q) {
        cudaPointerAttributes at;
        bool d = q && cudaPointerGetAttributes(&at, q) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        return d;
    };
    const bool dx_dev = is_dev(d_dx), ds_dev = is_dev(d_dsig);
    int64_t* d_off = nullptr; int* d_H = nullptr; double *d_fmin = nullptr, *d_df_c = nullptr;
    int64_t* d_ent = nullptr; double* d_g = nullptr;
    double *o_f = nullptr, *o_d = nullptr, *o_df = nullptr, *o_dx = nullptr, *o_ds = nullptr;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; return e == cudaSuccess; };
    ok(pool_alloc((void**)&d_off, 16, s)) && ok(pool_alloc((void**)&d_H, 4, s)) &&
        ok(pool_alloc((void**)&d_fmin, 8, s)) && ok(pool_alloc((void**)&d_df_c, 8, s)) &&
        ok(pool_alloc((void**)&d_ent, K * 8, s)) && ok(pool_alloc((void**)&o_f, K * 8, s)) &&
        ok(pool_alloc((void**)&o_d, K * 8, s)) && ok(pool_alloc((void**)&o_df, K * 8, s));
    if (grad_out) ok(pool_alloc((void**)&d_g, K * 8, s));
    if (d_dx && !dx_dev) ok(pool_alloc((void**)&o_dx, (size_t)K * n * 8, s));
    if (d_dsig && !ds_dev) ok(pool_alloc((void**)&o_ds, (size_t)K * n * 8, s));
    std::vector<int64_t> ent(K);
    for (int k = 0; k < K; ++k) ent[k] = peak_j[k];
    const int64_t offh[2] = {0, n};
    if (e == cudaSuccess) {
        ok(cudaMemcpyAsync(d_off, offh, 16, cudaMemcpyHostToDevice, s));
        ok(cudaMemcpyAsync(d_H, &p->H, 4, cudaMemcpyHostToDevice, s));
        ok(cudaMemcpyAsync(d_fmin, &p->f_min, 8, cudaMemcpyHostToDevice, s));
        ok(cudaMemcpyAsync(d_df_c, &p->df, 8, cudaMemcpyHostToDevice, s));
        ok(cudaMemcpyAsync(d_ent, ent.data(), K * 8, cudaMemcpyHostToDevice, s));
        if (grad_out) ok(cudaMemcpyAsync(d_g, grad_out, K * 8, cudaMemcpyDefault, s));
        AdjTab tb{d_off, d_H, d_fmin, d_df_c, p->d_scal, p->d_tau, p->d_wq, p->d_wp,
                  p->has_perm ? p->d_perm : nullptr, d_ent, d_g, K, 1e-10, 40};
        AdjOut out{o_f, o_d, o_df, dx_dev ? d_dx : o_dx, ds_dev ? d_dsig : o_ds};
        if (!d_dx) out.d_dx = nullptr;
        if (!d_dsig) out.d_dsig = nullptr;
        ok(launch_backward_tab(tb, K, out, s));
        std::vector<double> hf(K), hd(K), hg(K);
        ok(cudaMemcpyAsync(hf.data(), o_f, K * 8, cudaMemcpyDeviceToHost, s));
        ok(cudaMemcpyAsync(hd.data(), o_d, K * 8, cudaMemcpyDeviceToHost, s));
        ok(cudaMemcpyAsync(hg.data(), o_df, K * 8, cudaMemcpyDeviceToHost, s));
        if (d_dx && !dx_dev) ok(cudaMemcpyAsync(d_dx, o_dx, (size_t)K * n * 8, cudaMemcpyDeviceToHost, s));
        if (d_dsig && !ds_dev) ok(cudaMemcpyAsync(d_dsig, o_ds, (size_t)K * n * 8, cudaMemcpyDeviceToHost, s));
        ok(cudaStreamSynchronize(s));
        if (e == cudaSuccess) {
            for (int k = 0; k < K; ++k) {
                if (f_ref) f_ref[k] = hf[k];
                if (d_ref) d_ref[k] = hd[k];
                if (d_df) d_df[k] = hg[k];
            }
        }
    }
    for (void* q : {(void*)d_off, (void*)d_H, (void*)d_fmin, (void*)d_df_c, (void*)d_ent, (void*)d_g,
                    (void*)o_f, (void*)o_d, (void*)o_df, (void*)o_dx, (void*)o_ds})
        if (q) cudaFreeAsync(q, s);
    cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return FC2_ERR_OOM;
    return e == cudaSuccess ? FC2_OK : FC2_ERR_CUDA;
}

}  // namespace fc2
