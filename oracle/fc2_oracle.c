/*
 * fc2_oracle.c -- plain FP64 CPU oracle for the Fast chi-squared periodogram
 * (Palmer, "A Fast Chi-squared Technique For Period Search of Irregularly
 * Sampled Data", arXiv 0901.1913).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg call this code; the CUDA library never links,
 * includes or calls it, and it shares no code, header or table with it.
 *
 * What it computes is the exact quantity the FFT method approximates, written
 * out directly, with no gridding and no FFT:
 *   - model basis (Sec. 1, Eq. "eqtrunc"; Sec. 2 component functions):
 *       M_0 = 1, M_{2h-1} = sin(2 pi h f t), M_{2h} = cos(2 pi h f t);
 *   - weighted chi^2 (Sec. 2, Eq. "eqchigen") with w_i = 1 / sigma_i^2;
 *   - null model = weighted mean xbar (Sec. 3b), chi2_0 = sum w (x - xbar)^2
 *     (Sec. 3c, first equation after the H = 2 example);
 *   - Delta chi^2 = chi2_0 - min_A chi^2(A, f) for the nested models
 *     H' = 1..H (Sec. 1: all H' at once; Sec. 2 Eq. "eqchix").
 * The least-squares minimum is taken by Householder QR of the weighted design
 * matrix, one independent solve per H', so that it never forms the normal
 * equations or uses the trigonometric product identities the fast method
 * relies on (Sec. 2, Eqs. "eqalphafirst".."eqalpha").  Columns whose residual
 * norm after projection falls below tau_r times their own norm are dropped
 * (rank rule for exactly aliased frequencies, about which the paper is silent).
 *
 * Also provided, each written straight from its definition:
 *   - the trigonometric sums C, S, C', S' = Re/Im of P(f), Q(f) (Sec. 2,
 *     Eq. "eqPQ", sign e^{+i 2 pi f t});
 *   - the normal-equation matrix alpha and vector beta by direct sums over the
 *     samples (Sec. 2, the alpha_jk and beta_j definitions);
 *   - the Fourier coefficients A = alpha^{-1} beta (Sec. 2, Eq. "eqcoeffs"),
 *     with xbar added back to A_0 (Sec. 3b);
 *   - gradients of Delta chi^2 w.r.t. f, x_i, sigma_i at fixed f (envelope
 *     theorem applied to Eq. "eqchigen"; not printed in the paper);
 *   - Brent maximisation of the exact, ungridded Delta chi^2 near a bin
 *     (the local refinement with ungridded data advised in Sec. 3e).
 *
 * All arithmetic is IEEE double; sums over samples use Neumaier compensation.
 * Functions return 0 on success, a negative value on bad arguments or
 * allocation failure.  They are single-threaded and re-entrant: callers run
 * several of them at once on disjoint bins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ sums */
typedef struct { double s, c; } nsum_t;

static inline void nadd(nsum_t* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum_t* a) { return a->s + a->c; }

/* fractional part of h * f * t, reduced in double (Sec. 1 basis phase) */
static inline double phase_frac(int h, double f, double t) {
    double p = ((double)h * f) * t;
    return p - floor(p);
}

/* ------------------------------------------------------------- moments */
/* out[0] = W = sum w, out[1] = xbar = sum w x / W, out[2] = chi2_0 =
 * sum w (x - xbar)^2, out[3] = sum w (x - xbar) (zero up to rounding). */
int fc2o_moments(const double* t, const double* x, const double* sigma,
                 int64_t n, double* out) {
    (void)t;
    if (n < 1 || !x || !sigma || !out) return -1;
    nsum_t W = {0, 0}, WX = {0, 0}, C0 = {0, 0}, S1 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double w = 1.0 / (sigma[i] * sigma[i]);
        nadd(&W, w);
        nadd(&WX, w * x[i]);
    }
    double Wv = nval(&W), xbar = nval(&WX) / Wv;
    for (int64_t i = 0; i < n; ++i) {
        double w = 1.0 / (sigma[i] * sigma[i]);
        double d = x[i] - xbar;
        nadd(&C0, w * d * d);
        nadd(&S1, w * d);
    }
    out[0] = Wv;
    out[1] = xbar;
    out[2] = nval(&C0);
    out[3] = nval(&S1);
    return 0;
}

/* ------------------------------------------------------ design matrix */
/* Column-major weighted design for harmonics 1..Hp at frequency f:
 * D[l*n + i] = sqrt(w_i) * M_l(f, t_i), l = 0..2Hp. */
static void build_design(const double* t, const double* sw, int64_t n,
                         double f, int Hp, double* D) {
    for (int64_t i = 0; i < n; ++i) D[i] = sw[i];
    for (int h = 1; h <= Hp; ++h) {
        double* Ds = D + (int64_t)(2 * h - 1) * n;
        double* Dc = D + (int64_t)(2 * h) * n;
        for (int64_t i = 0; i < n; ++i) {
            double th = TWO_PI * phase_frac(h, f, t[i]);
            Ds[i] = sw[i] * sin(th);
            Dc[i] = sw[i] * cos(th);
        }
    }
}

/*
 * Householder QR least squares on D (n x m, column-major, overwritten) and
 * y (n, overwritten with Q^T y).  Columns are taken in their given order, and
 * column l is dropped when its residual norm after the previous reflections
 * is <= tau_r times its original norm.
 * On return: *rank, colmap[q] = column of the q-th reflection, diag[q] = R_qq,
 * qty[q] = (Q^T y)_q, and *minpiv = min over kept columns of
 * (residual norm / original norm)^2 -- the Cholesky relative pivot
 * d_l / alpha_ll of the same column order.
 */
static void householder_ls(double* D, int64_t n, int m, double* y,
                           double tau_r, int* rank, int* colmap,
                           double* diag, double* qty, double* minpiv) {
    double orig[2 * 64 + 9];  /* up to 2H + 1 harmonic and D + 1 <= 9 polynomial columns */
    for (int l = 0; l < m; ++l) {
        nsum_t s = {0, 0};
        const double* c = D + (int64_t)l * n;
        for (int64_t i = 0; i < n; ++i) nadd(&s, c[i] * c[i]);
        orig[l] = sqrt(nval(&s));
    }
    int p = 0;
    double mp = INFINITY;
    for (int l = 0; l < m && p < n; ++l) {
        double* c = D + (int64_t)l * n;
        nsum_t s2 = {0, 0};
        for (int64_t i = p; i < n; ++i) nadd(&s2, c[i] * c[i]);
        double s = sqrt(nval(&s2));
        if (!(orig[l] > 0.0) || s <= tau_r * orig[l]) continue;  /* dropped */
        double r = s / orig[l];
        if (r * r < mp) mp = r * r;
        double x0 = c[p];
        double alpha = (x0 >= 0.0) ? -s : s;
        double v0 = x0 - alpha;
        c[p] = v0;
        /* |v|^2 = s^2 - x0^2 + v0^2 = 2 s (s + |x0|) */
        double vn2 = 2.0 * s * (s + fabs(x0));
        for (int k = l + 1; k < m; ++k) {
            double* ck = D + (int64_t)k * n;
            nsum_t d = {0, 0};
            for (int64_t i = p; i < n; ++i) nadd(&d, c[i] * ck[i]);
            double g = 2.0 * nval(&d) / vn2;
            for (int64_t i = p; i < n; ++i) ck[i] -= g * c[i];
        }
        {
            nsum_t d = {0, 0};
            for (int64_t i = p; i < n; ++i) nadd(&d, c[i] * y[i]);
            double g = 2.0 * nval(&d) / vn2;
            for (int64_t i = p; i < n; ++i) y[i] -= g * c[i];
        }
        colmap[p] = l;
        diag[p] = alpha;
        qty[p] = y[p];
        ++p;
    }
    *rank = p;
    *minpiv = (p > 0) ? mp : 0.0;
}

/* Solve one H' model at frequency f.  Work buffers are allocated here.
 * dchi2: Delta chi^2; minpiv: see householder_ls; A (may be NULL): the
 * 2Hp+1 coefficients in the basis order, relative to x - xbar (basic
 * solution, dropped columns = 0).  mdl (may be NULL): fitted model of
 * x - xbar at every sample. */
static int solve_one(const double* t, const double* sw, const double* y0,
                     int64_t n, double f, int Hp, double tau_r,
                     double sum_wd, double W, double* dchi2, double* minpiv,
                     double* A, double* mdl) {
    int m = 2 * Hp + 1;
    double* D = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    if (!D || !y) { free(D); free(y); return -2; }
    build_design(t, sw, n, f, Hp, D);
    memcpy(y, y0, sizeof(double) * (size_t)n);
    int rank = 0, colmap[2 * 64 + 1];
    double diag[2 * 64 + 1], qty[2 * 64 + 1], mp = 0.0;
    householder_ls(D, n, m, y, tau_r, &rank, colmap, diag, qty, &mp);
    double ss = 0.0;
    for (int q = 0; q < rank; ++q) ss += qty[q] * qty[q];
    /* Delta chi^2 = |proj onto model span|^2 - |proj onto constant|^2 */
    *dchi2 = ss - sum_wd * sum_wd / W;
    if (minpiv) *minpiv = mp;
    if (A || mdl) {
        double coef[2 * 64 + 1];
        for (int l = 0; l < m; ++l) coef[l] = 0.0;
        for (int q = rank - 1; q >= 0; --q) {
            double acc = qty[q];
            for (int q2 = q + 1; q2 < rank; ++q2) {
                int c2 = colmap[q2];
                acc -= D[(int64_t)c2 * n + q] * coef[c2];
            }
            coef[colmap[q]] = acc / diag[q];
        }
        if (A) for (int l = 0; l < m; ++l) A[l] = coef[l];
        if (mdl) {
            for (int64_t i = 0; i < n; ++i) {
                double v = coef[0];
                for (int h = 1; h <= Hp; ++h) {
                    double th = TWO_PI * phase_frac(h, f, t[i]);
                    v += coef[2 * h - 1] * sin(th) + coef[2 * h] * cos(th);
                }
                mdl[i] = v;
            }
        }
    }
    free(D);
    free(y);
    return 0;
}

typedef struct { double W, xbar, chi2_0, sum_wd; double* sw; double* y; } prep_t;

static int prep(const double* x, const double* sigma, int64_t n, prep_t* P) {
    double mom[4];
    if (fc2o_moments(NULL, x, sigma, n, mom)) return -1;
    P->W = mom[0]; P->xbar = mom[1]; P->chi2_0 = mom[2]; P->sum_wd = mom[3];
    P->sw = (double*)malloc(sizeof(double) * (size_t)n);
    P->y = (double*)malloc(sizeof(double) * (size_t)n);
    if (!P->sw || !P->y) { free(P->sw); free(P->y); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        P->sw[i] = 1.0 / sigma[i];                  /* sqrt(w_i) */
        P->y[i] = P->sw[i] * (x[i] - P->xbar);      /* sqrt(w_i) (x_i - xbar) */
    }
    return 0;
}
static void unprep(prep_t* P) { free(P->sw); free(P->y); }

/* ------------------------------------------------------- public calls */

/* Delta chi^2 at arbitrary frequencies freqs[nf] for every H' = 1..H.
 * dchi2[k*H + (H'-1)], minpiv[k*H + (H'-1)] (minpiv may be NULL). */
int fc2o_dchi2_freqs(const double* t, const double* x, const double* sigma,
                     int64_t n, int H, const double* freqs, int64_t nf,
                     double tau_r, double* dchi2, double* minpiv) {
    if (n < 1 || H < 1 || H > 64 || nf < 0 || !t || !x || !sigma || !dchi2) return -1;
    prep_t P;
    int rc = prep(x, sigma, n, &P);
    if (rc) return rc;
    for (int64_t k = 0; k < nf; ++k) {
        for (int Hp = 1; Hp <= H; ++Hp) {
            double mp = 0.0;
            rc = solve_one(t, P.sw, P.y, n, freqs[k], Hp, tau_r, P.sum_wd, P.W,
                           &dchi2[k * H + (Hp - 1)], &mp, NULL, NULL);
            if (rc) { unprep(&P); return rc; }
            if (minpiv) minpiv[k * H + (Hp - 1)] = mp;
        }
    }
    unprep(&P);
    return 0;
}

/* ------------------------------------------- trend fitted with the harmonics
 * The polynomial detrending of Sec. 4 ("detrend the data with a polynomial
 * fit ... removing variation out to t^3") read as a joint fit: the null model is
 * the weighted least-squares polynomial of degree D in t, and the model at f is
 * that polynomial plus the H' harmonics (Sec. 1, Eq. "eqtrunc"), all fitted
 * together:  Delta chi^2_{H'}(f) = chi^2(poly) - chi^2(poly + H' harmonics).
 * The polynomial columns use u = (t - t_c) / s, t_c and s the centre and
 * half-width of the time span (a change of basis, the same span).  Householder
 * QR on the weighted design [u^0 .. u^D, sin 1, cos 1, ..] with the polynomial
 * columns first: Delta chi^2 = |projection onto the full span|^2 - |projection
 * onto the polynomial span|^2; minpiv as in householder_ls, over all columns.
 * chi2_0 (chi2_0[0], may be NULL): chi^2 of the polynomial alone. */
int fc2o_dchi2_trend_freqs(const double* t, const double* x, const double* sigma,
                           int64_t n, int H, int D, const double* freqs, int64_t nf,
                           double tau_r, double* dchi2, double* minpiv, double* chi2_0) {
    if (n < 1 || H < 1 || H > 64 || D < 0 || D > 8 || nf < 0 || !t || !x || !sigma || !dchi2)
        return -1;
    double lo = t[0], hi = t[0];
    for (int64_t i = 1; i < n; ++i) { if (t[i] < lo) lo = t[i]; if (t[i] > hi) hi = t[i]; }
    const double tc = 0.5 * (lo + hi), sc = (hi > lo) ? 0.5 * (hi - lo) : 1.0;
    const int mmax = D + 1 + 2 * H;
    double* Dm = (double*)malloc(sizeof(double) * (size_t)n * (size_t)mmax);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* sw = (double*)malloc(sizeof(double) * (size_t)n);
    if (!Dm || !y || !sw) { free(Dm); free(y); free(sw); return -2; }
    for (int64_t i = 0; i < n; ++i) sw[i] = 1.0 / sigma[i];
    int rc = 0;
    for (int64_t k = 0; k <= nf; ++k) {
        /* k == nf: the polynomial alone (chi2_0) */
        const int Hs = (k < nf) ? H : 0;
        for (int Hp = (k < nf) ? 1 : 0; Hp <= Hs; ++Hp) {
            const int m = D + 1 + 2 * Hp;
            for (int64_t i = 0; i < n; ++i) {
                const double u = (t[i] - tc) / sc;
                double up = 1.0;
                for (int q = 0; q <= D; ++q) { Dm[(int64_t)q * n + i] = sw[i] * up; up *= u; }
                y[i] = sw[i] * x[i];
            }
            for (int h = 1; h <= Hp; ++h) {
                double* Ds = Dm + (int64_t)(D + 2 * h - 1) * n;
                double* Dc = Dm + (int64_t)(D + 2 * h) * n;
                for (int64_t i = 0; i < n; ++i) {
                    const double th = TWO_PI * phase_frac(h, freqs[k], t[i]);
                    Ds[i] = sw[i] * sin(th);
                    Dc[i] = sw[i] * cos(th);
                }
            }
            int rank = 0, colmap[2 * 64 + 9];
            double diag[2 * 64 + 9], qty[2 * 64 + 9], mp = 0.0;
            householder_ls(Dm, n, m, y, tau_r, &rank, colmap, diag, qty, &mp);
            double ss_all = 0.0, ss_poly = 0.0;
            for (int q = 0; q < rank; ++q) {
                ss_all += qty[q] * qty[q];
                if (colmap[q] <= D) ss_poly += qty[q] * qty[q];
            }
            if (k < nf) {
                dchi2[k * H + (Hp - 1)] = ss_all - ss_poly;
                if (minpiv) minpiv[k * H + (Hp - 1)] = mp;
            } else if (chi2_0) {
                nsum_t yy = {0, 0};
                for (int64_t i = 0; i < n; ++i) nadd(&yy, (sw[i] * x[i]) * (sw[i] * x[i]));
                chi2_0[0] = nval(&yy) - ss_poly;
            }
        }
    }
    free(Dm); free(y); free(sw);
    return rc;
}

/* Same, at the trial bins f_j = f_min + j * df for j in bins[nb]. */
int fc2o_dchi2_bins(const double* t, const double* x, const double* sigma,
                    int64_t n, int H, double f_min, double df,
                    const int64_t* bins, int64_t nb, double tau_r,
                    double* dchi2, double* minpiv) {
    if (nb < 0 || (nb > 0 && !bins)) return -1;
    double* fr = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    if (!fr) return -2;
    for (int64_t k = 0; k < nb; ++k) fr[k] = f_min + (double)bins[k] * df;
    int rc = fc2o_dchi2_freqs(t, x, sigma, n, H, fr, nb, tau_r, dchi2, minpiv);
    free(fr);
    return rc;
}

/* Coefficients of the Hp-harmonic fit at f, in the basis order
 * [A0, sin1, cos1, ...], absolute time frame, with xbar added to A0. */
int fc2o_coeffs(const double* t, const double* x, const double* sigma,
                int64_t n, int Hp, double f, double tau_r, double* A,
                double* dchi2) {
    if (n < 1 || Hp < 1 || Hp > 64 || !A) return -1;
    prep_t P;
    int rc = prep(x, sigma, n, &P);
    if (rc) return rc;
    double d = 0.0;
    rc = solve_one(t, P.sw, P.y, n, f, Hp, tau_r, P.sum_wd, P.W, &d, NULL, A, NULL);
    A[0] += P.xbar;
    if (dchi2) *dchi2 = d;
    unprep(&P);
    return rc;
}

/* Direct trigonometric sums (Sec. 2, Eq. "eqPQ"):
 * re[k] + i im[k] = sum_i c_i exp(+i 2 pi freqs[k] t_i). */
int fc2o_trig_sums(const double* t, const double* c, int64_t n,
                   const double* freqs, int64_t nf, double* re, double* im) {
    if (n < 0 || nf < 0 || !re || !im) return -1;
    for (int64_t k = 0; k < nf; ++k) {
        nsum_t a = {0, 0}, b = {0, 0};
        double f = freqs[k];
        double af = fabs(f);
        double sg = (f < 0.0) ? -1.0 : 1.0;
        for (int64_t i = 0; i < n; ++i) {
            double p = af * t[i];
            double th = TWO_PI * (p - floor(p));
            nadd(&a, c[i] * cos(th));
            nadd(&b, sg * c[i] * sin(th));
        }
        re[k] = nval(&a);
        im[k] = nval(&b);
    }
    return 0;
}

/* Normal equations by direct sums (Sec. 2): alpha[j*m + k] = sum w M_j M_k,
 * beta[j] = sum w M_j (x - xbar), m = 2H + 1. */
int fc2o_normal_eq(const double* t, const double* x, const double* sigma,
                   int64_t n, int H, double f, double* alpha, double* beta) {
    if (n < 1 || H < 1 || H > 64 || !alpha || !beta) return -1;
    int m = 2 * H + 1;
    double mom[4];
    fc2o_moments(t, x, sigma, n, mom);
    nsum_t* A = (nsum_t*)calloc((size_t)m * (size_t)m, sizeof(nsum_t));
    nsum_t* B = (nsum_t*)calloc((size_t)m, sizeof(nsum_t));
    double* Mv = (double*)malloc(sizeof(double) * (size_t)m);
    if (!A || !B || !Mv) { free(A); free(B); free(Mv); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        double w = 1.0 / (sigma[i] * sigma[i]);
        double d = x[i] - mom[1];
        Mv[0] = 1.0;
        for (int h = 1; h <= H; ++h) {
            double th = TWO_PI * phase_frac(h, f, t[i]);
            Mv[2 * h - 1] = sin(th);
            Mv[2 * h] = cos(th);
        }
        for (int j = 0; j < m; ++j) {
            nadd(&B[j], w * Mv[j] * d);
            for (int k = 0; k < m; ++k) nadd(&A[j * m + k], w * Mv[j] * Mv[k]);
        }
    }
    for (int j = 0; j < m; ++j) {
        beta[j] = nval(&B[j]);
        for (int k = 0; k < m; ++k) alpha[j * m + k] = nval(&A[j * m + k]);
    }
    free(A); free(B); free(Mv);
    return 0;
}

/*
 * Gradients of Delta chi^2_H at fixed f.  With A the optimal coefficients and
 * m_i = xbar + sum_l A_l M_l(f, t_i) the fitted model, the envelope theorem on
 * chi2_0 (minimised over the constant) and on chi^2_min (minimised over A)
 * gives
 *   dD/dx_i     = 2 w_i (m_i - xbar)
 *   dD/dsigma_i = -2 sigma_i^-3 [ (x_i - xbar)^2 - (x_i - m_i)^2 ]
 *   dD/df       = 2 sum_i w_i (x_i - m_i) dm_i/df,
 *   dm_i/df     = sum_h 2 pi h t_i (A_{2h-1} cos th_ih - A_{2h} sin th_ih).
 * Any of the output pointers may be NULL.
 */
int fc2o_grad(const double* t, const double* x, const double* sigma,
              int64_t n, int H, double f, double tau_r, double* dchi2,
              double* d_df, double* d_dx, double* d_dsigma) {
    if (n < 1 || H < 1 || H > 64) return -1;
    prep_t P;
    int rc = prep(x, sigma, n, &P);
    if (rc) return rc;
    int m = 2 * H + 1;
    double A[2 * 64 + 1], d = 0.0;
    double* mdl = (double*)malloc(sizeof(double) * (size_t)n);
    if (!mdl) { unprep(&P); return -2; }
    rc = solve_one(t, P.sw, P.y, n, f, H, tau_r, P.sum_wd, P.W, &d, NULL, A, mdl);
    if (rc) { free(mdl); unprep(&P); return rc; }
    (void)m;
    if (dchi2) *dchi2 = d;
    nsum_t g = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double w = 1.0 / (sigma[i] * sigma[i]);
        double mi = P.xbar + mdl[i];
        double r = x[i] - mi;
        double dx0 = x[i] - P.xbar;
        if (d_dx) d_dx[i] = 2.0 * w * (mi - P.xbar);
        if (d_dsigma) d_dsigma[i] = -2.0 / (sigma[i] * sigma[i] * sigma[i]) * (dx0 * dx0 - r * r);
        if (d_df) {
            double dm = 0.0;
            for (int h = 1; h <= H; ++h) {
                double th = TWO_PI * phase_frac(h, f, t[i]);
                dm += TWO_PI * h * t[i] * (A[2 * h - 1] * cos(th) - A[2 * h] * sin(th));
            }
            nadd(&g, 2.0 * w * r * dm);
        }
    }
    if (d_df) *d_df = nval(&g);
    free(mdl);
    unprep(&P);
    return 0;
}

/* Delta chi^2_H at one frequency (helper for the maximiser). */
static double dchi2_at(const double* t, const prep_t* P, int64_t n, int H,
                       double f, double tau_r) {
    double d = 0.0;
    if (solve_one(t, P->sw, P->y, n, f, H, tau_r, P->sum_wd, P->W, &d, NULL,
                  NULL, NULL))
        return NAN;
    return d;
}

/*
 * Brent's method (R. P. Brent, "Algorithms for Minimization without
 * Derivatives", 1973, ch. 5: golden-section search combined with successive
 * parabolic interpolation) applied to -Delta chi^2_H(f) on [a, b], stopping
 * when the bracket half-width is below tol.  Returns the maximiser and value.
 */
int fc2o_refine(const double* t, const double* x, const double* sigma,
                int64_t n, int H, double a, double b, double tol,
                double tau_r, double* f_star, double* dchi2_star) {
    if (n < 1 || H < 1 || H > 64 || !(b > a) || !(tol > 0)) return -1;
    prep_t P;
    int rc = prep(x, sigma, n, &P);
    if (rc) return rc;
    const double cgold = 0.3819660112501051;  /* (3 - sqrt 5) / 2 */
    double v = a + cgold * (b - a), w = v, xx = v;
    double fx = -dchi2_at(t, &P, n, H, xx, tau_r), fv = fx, fw = fx;
    double d = 0.0, e = 0.0;
    for (int it = 0; it < 500; ++it) {
        double xm = 0.5 * (a + b);
        double tol1 = tol, tol2 = 2.0 * tol1;
        if (fabs(xx - xm) <= tol2 - 0.5 * (b - a)) break;
        int golden = 1;
        if (fabs(e) > tol1) {
            double r = (xx - w) * (fx - fv);
            double q = (xx - v) * (fx - fw);
            double p = (xx - v) * q - (xx - w) * r;
            q = 2.0 * (q - r);
            if (q > 0.0) p = -p; else q = -q;
            double etemp = e;
            e = d;
            if (!(fabs(p) >= fabs(0.5 * q * etemp) || p <= q * (a - xx) || p >= q * (b - xx))) {
                d = p / q;
                double u = xx + d;
                if (u - a < tol2 || b - u < tol2) d = (xm >= xx) ? tol1 : -tol1;
                golden = 0;
            }
        }
        if (golden) {
            e = (xx >= xm) ? a - xx : b - xx;
            d = cgold * e;
        }
        double u = (fabs(d) >= tol1) ? xx + d : xx + ((d >= 0) ? tol1 : -tol1);
        double fu = -dchi2_at(t, &P, n, H, u, tau_r);
        if (fu <= fx) {
            if (u >= xx) a = xx; else b = xx;
            v = w; fv = fw; w = xx; fw = fx; xx = u; fx = fu;
        } else {
            if (u < xx) a = u; else b = u;
            if (fu <= fw || w == xx) { v = w; fv = fw; w = u; fw = fu; }
            else if (fu <= fv || v == xx || v == w) { v = u; fv = fu; }
        }
    }
    *f_star = xx;
    if (dchi2_star) *dchi2_star = -fx;
    unprep(&P);
    return 0;
}
