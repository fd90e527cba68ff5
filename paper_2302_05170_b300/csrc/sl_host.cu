// sl_host.cu -- host-side numerics and bookkeeping of the Seven-League library:
// Gauss-Hermite points by Golub-Welsch (FP64), quantile ranks, error text,
// device status word.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "sl_internal.cuh"

namespace sl {

static thread_local char g_err[512] = "";

int set_error(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_error(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return SL_OK;
    return set_error(SL_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Symmetric tridiagonal eigenproblem by the implicit QL algorithm with Wilkinson
// shifts (textbook form).  d: diagonal (in: matrix, out: eigenvalues),
// e: sub-diagonal in e[0..n-2], z: n x n row-major, in: identity, out: columns
// are the eigenvectors.
static int tridiag_ql(int n, double* d, double* e, double* z) {
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            int mm = l;
            for (; mm < n - 1; ++mm) {
                const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
                if (fabs(e[mm]) + dd == dd) break;   // negligible at working precision
            }
            if (mm == l) break;
            if (++iter > 64) return 1;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = mm - 1;
            for (; i >= l; --i) {
                double f = s * e[i];
                const double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int k = 0; k < n; ++k) {
                    f = z[k * n + i + 1];
                    z[k * n + i + 1] = s * z[k * n + i] + c * f;
                    z[k * n + i] = c * z[k * n + i] - s * f;
                }
            }
            if (r == 0.0 && i >= l) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    return 0;
}

int gauss_hermite_fp64(int m, double* x, double* w, double* bary) {
    if (m < SL_MIN_M || m > SL_MAX_M)
        return set_error(SL_ERR_UNSUPPORTED, "m=%d outside [%d,%d]", m, SL_MIN_M, SL_MAX_M);
    // Golub-Welsch: the Jacobi matrix of the probabilists' Hermite recurrence
    // He_{k+1} = x He_k - k He_{k-1} is tridiagonal with zero diagonal and
    // off-diagonal sqrt(k); its eigenvalues are the nodes and the squared first
    // components of its unit eigenvectors are the probability weights.
    double d[SL_MAX_M], e[SL_MAX_M], z[SL_MAX_M * SL_MAX_M];
    for (int i = 0; i < m; ++i) {
        d[i] = 0.0;
        e[i] = (i < m - 1) ? sqrt(static_cast<double>(i + 1)) : 0.0;
        for (int k = 0; k < m; ++k) z[i * m + k] = (i == k) ? 1.0 : 0.0;
    }
    if (tridiag_ql(m, d, e, z)) return set_error(SL_ERR_UNSUPPORTED, "QL did not converge");
    int order[SL_MAX_M];
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i)  // insertion sort by eigenvalue
        for (int k = i; k > 0 && d[order[k]] < d[order[k - 1]]; --k) {
            const int t = order[k];
            order[k] = order[k - 1];
            order[k - 1] = t;
        }
    double xs[SL_MAX_M], ws[SL_MAX_M];
    for (int i = 0; i < m; ++i) {
        xs[i] = d[order[i]];
        const double v0 = z[0 * m + order[i]];
        ws[i] = v0 * v0;
    }
    // Exact symmetry of the nodes and weights about 0.
    for (int j = 0; j < m / 2; ++j) {
        const double s = 0.5 * (xs[m - 1 - j] - xs[j]);
        xs[j] = -s;
        xs[m - 1 - j] = s;
        const double wv = 0.5 * (ws[j] + ws[m - 1 - j]);
        ws[j] = ws[m - 1 - j] = wv;
    }
    if (m % 2) xs[m / 2] = 0.0;
    double sum = 0.0;
    for (int i = 0; i < m; ++i) sum += ws[i];
    for (int i = 0; i < m; ++i) {
        if (x) x[i] = xs[i];
        if (w) w[i] = ws[i] / sum;
        if (bary) {
            double p = 1.0;
            for (int k = 0; k < m; ++k)
                if (k != i) p *= (xs[i] - xs[k]);
            bary[i] = 1.0 / p;
        }
    }
    return SL_OK;
}

int make_gh_const(int m, GHConst* out) {
    double x[SL_MAX_M], b[SL_MAX_M];
    const int rc = gauss_hermite_fp64(m, x, nullptr, b);
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    for (int j = 0; j < SL_MAX_M; ++j) {
        out->x[j] = (j < m) ? static_cast<float>(x[j]) : 0.0f;
        out->bary[j] = (j < m) ? static_cast<float>(b[j]) : 0.0f;
        out->dsc[j] = (j < m) ? 1.0f : 0.0f;
        out->doff[j] = (j < m) ? -out->x[j] : 1.0f;
    }
    return SL_OK;
}

}  // namespace sl

using namespace sl;

extern "C" {

int sl_version(void) { return 100; }

const char* sl_last_error_string(void) { return g_err; }

int64_t sl_n_params(int d_in, int m) {
    return static_cast<int64_t>(SL_WIDTH) * d_in + SL_WIDTH +
           static_cast<int64_t>(SL_N_HIDDEN - 1) * (SL_WIDTH * SL_WIDTH + SL_WIDTH) +
           static_cast<int64_t>(m) * SL_WIDTH + m;
}

int sl_gauss_hermite(int m, double* x, double* w, double* bary) {
    return gauss_hermite_fp64(m, x, w, bary);
}

int sl_quantile_ranks(int m, int64_t n, int64_t* ranks) {
    if (!ranks || n < 1) return set_error(SL_ERR_ARG, "ranks == NULL or n < 1");
    double x[SL_MAX_M];
    const int rc = gauss_hermite_fp64(m, x, nullptr, nullptr);
    if (rc) return rc;
    for (int j = 0; j < m; ++j) {
        const double level = 0.5 * erfc(-x[j] / sqrt(2.0));   // Phi(x_j)
        int64_t k = static_cast<int64_t>(ceil(static_cast<double>(n) * level)) - 1;
        ranks[j] = k < 0 ? 0 : (k > n - 1 ? n - 1 : k);
    }
    return SL_OK;
}

int sl_workspace_status(const void* ws, void* stream, uint32_t* bits) {
    if (!ws) return set_error(SL_ERR_ARG, "ws == NULL");
    uint32_t v = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = cuda_error(cudaMemcpyAsync(&v, ws, sizeof(v), cudaMemcpyDeviceToHost, s),
                        "status copy");
    if (rc) return rc;
    rc = cuda_error(cudaStreamSynchronize(s), "status sync");
    if (rc) return rc;
    if (bits) *bits = v;
    if (v & SL_DEV_TIMEOUT) return set_error(SL_ERR_TIMEOUT, "device wait timed out (bits 0x%x)", v);
    if (v) return set_error(SL_ERR_DEVICE, "device status bits 0x%x", v);
    return SL_OK;
}

}  // extern "C"
