// fc2_host.cpp -- host-side numerics of libfc2: Gauss-Legendre rule, the
// spreading kernel's Fourier transform, default widths, status strings.
#include <math.h>
#include <string.h>

#include "fc2_internal.h"

namespace fc2 {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on the Legendre
// three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
void gauss_legendre(int nq, double* x, double* w) {
    for (int i = 0; i < nq; ++i) {
        double z = cos(M_PI * (i + 0.75) / (nq + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < nq; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = nq * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static double es_host(double z, int w, double beta) {
    double s = 2.0 * z / (double)w;
    double a = 1.0 - s * s;
    return a > 0.0 ? exp(beta * (sqrt(a) - 1.0)) : 0.0;
}

// phihat(xi) = 2 int_0^{w/2} phi(z) cos(2 pi xi z) dz by an nq-point rule.
double kernel_ft_host(int w, double beta, double xi, int nq, const double* gx, const double* gw) {
    const double half = 0.5 * (double)w;
    double acc = 0.0;
    for (int i = 0; i < nq; ++i) {
        double z = 0.5 * half * (gx[i] + 1.0);
        acc += gw[i] * es_host(z, w, beta) * cos(2.0 * M_PI * xi * z);
    }
    return 2.0 * 0.5 * half * acc;
}

// Widths chosen so that the kernel's aliasing error, about
// exp(-pi w sqrt(1 - 1/sigma)) relative to sum |c_i| for this kernel family,
// sits below the spectrum precision of each path.
int default_width(bool fp64, int oversample) {
    if (fp64) return oversample >= 4 ? 12 : 14;
    return oversample >= 4 ? 7 : 9;
}

}  // namespace fc2

extern "C" {

void fc2_options_default(fc2_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->prec = FC2_PREC_FP64;
}

const char* fc2_status_string(fc2_status s) {
    switch (s) {
        case FC2_OK: return "ok";
        case FC2_ERR_INVALID_ARG: return "invalid argument";
        case FC2_ERR_CUDA: return "CUDA runtime error";
        case FC2_ERR_OOM: return "out of device memory";
        case FC2_ERR_TIMEOUT: return "bounded device wait timed out";
        case FC2_ERR_UNSUPPORTED: return "unsupported request";
        case FC2_ERR_NUMERIC: return "non-finite intermediate";
    }
    return "unknown status";
}

int64_t fc2_grid_size(int64_t N, int oversample) {
    if (N < 2 || oversample < 2 || N > (1ll << 30)) return 0;
    int64_t need = (int64_t)oversample * N;
    int64_t M = 512;
    while (M < need) M <<= 1;
    if (M > (1ll << 30)) return 0;
    return M;
}

int fc2_default_width(fc2_precision prec, int oversample) {
    return fc2::default_width(prec == FC2_PREC_FP64, oversample);
}

fc2_status fc2_kernel_ft(int w, int oversample, const double* xi, int64_t nxi, double* out) {
    if (w < 2 || w > 16 || oversample < 2 || nxi < 0 || (nxi > 0 && (!xi || !out)))
        return FC2_ERR_INVALID_ARG;
    int nq = 2 * w + 16;
    double gx[64], gw[64];
    fc2::gauss_legendre(nq, gx, gw);
    double beta = 0.97 * M_PI * (1.0 - 0.5 / (double)oversample) * (double)w;
    for (int64_t i = 0; i < nxi; ++i) out[i] = fc2::kernel_ft_host(w, beta, xi[i], nq, gx, gw);
    return FC2_OK;
}

fc2_status fc2_kernel_eval(int w, int oversample, const double* z, int64_t nz, double* out) {
    if (w < 2 || w > 16 || oversample < 2 || nz < 0 || (nz > 0 && (!z || !out)))
        return FC2_ERR_INVALID_ARG;
    double beta = 0.97 * M_PI * (1.0 - 0.5 / (double)oversample) * (double)w;
    for (int64_t i = 0; i < nz; ++i) out[i] = fc2::es_host(z[i], w, beta);
    return FC2_OK;
}

}  // extern "C"
