/*
 * sl_oracle.c -- plain FP64 CPU oracle for the Seven-League (7L) scheme.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this file.  It shares
 * no code, header, table or constant generator with the CUDA library: every
 * routine here is written from the paper's definitions (or the published
 * definition of the random number generator) and kept deliberately simple:
 * one path at a time, one loop per sum, FP64 throughout.
 *
 * Paper: S. Liu, G. Colonna, L. Grzelak, C. Oosterlee, "GPU acceleration of
 * the Seven-League scheme for large time step simulations of SDEs"
 * (arXiv:2302.05170).  Citations below name its equations and Algorithm I.
 *
 * Pinned against (tests/test_oracle_*.py): Gauss-Hermite closed forms and
 * moment exactness, Philox published known-answer vectors, Lagrange
 * interpolation identities, closed-form moments of the exact-collocation GBM
 * chain, pathwise exactness of the exact-collocation OU chain, exact moment
 * recursions of Euler-Maruyama, brute-force order statistics, central finite
 * differences for every derivative, and closed-form Black-Scholes values;
 * the 7L-CDC variant against polynomial reproduction, scipy's exact marginal
 * and conditional quantiles, and the 7L chain wherever the conditional map is
 * affine in Y (tests/test_oracle_cdc.py); its quantile-coordinate reading
 * against the inverse-map identities, tensor-product polynomial reproduction
 * and the exact OU chain (tests/test_oracle_cdcq.py).
 * No function in this file is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Model / SDE / activation codes (the same integers the library uses, chosen
 * independently here and checked by the tests). */
enum { ORC_MODEL_MLP = 0, ORC_MODEL_GBM_EXACT = 1, ORC_MODEL_OU_EXACT = 2 };
enum { ORC_SDE_GBM = 0, ORC_SDE_OU = 1, ORC_SDE_CIR = 2 };
enum { ORC_ACT_RELU = 0, ORC_ACT_SOFTPLUS = 1 };
enum { ORC_TAG_7L = 0, ORC_TAG_EM = 1 };

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 *   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
 * with the key bumped by the Weyl constants between rounds.
 * The paper only requires X ~ N(0,1) (Eq. 6.2, Algorithm I step 6); the
 * generator is the library's choice and is reproduced here independently.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1) from the top 23 bits of a word: ((w >> 9) + 1/2) / 2^23.
 * 23 bits keep the value exactly representable in FP32 as well as FP64, so
 * a single-precision implementation starts from the identical number. */
static double word_to_uniform(uint32_t w) {
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Standard normal number `step` of the stream (seed, tag, set, path).
 * Counter = (step / 4, path, set, tag), key = (seed low word, seed high word).
 * Box-Muller on the word pairs (0,1) and (2,3): radius from the first word
 * of the pair, angle from the second; cosine for even `step`, sine for odd. */
double orc_normal(uint64_t seed, uint32_t tag, uint32_t set, uint32_t path, uint32_t step) {
    uint32_t ctr[4] = {step >> 2, path, set, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint32_t pair = (step & 3u) >> 1;      /* 0 -> words (0,1), 1 -> words (2,3) */
    double u_r = word_to_uniform(w[2 * pair]);
    double u_a = word_to_uniform(w[2 * pair + 1]);
    double radius = sqrt(-2.0 * log(u_r));
    double angle = 2.0 * M_PI * u_a;
    return (step & 1u) ? radius * sin(angle) : radius * cos(angle);
}

void orc_normals(uint64_t seed, uint32_t tag, uint32_t set, uint32_t path,
                 uint32_t first_step, int n, double* out) {
    for (int i = 0; i < n; ++i) out[i] = orc_normal(seed, tag, set, path, first_step + (uint32_t)i);
}

/* ------------------------------------------------------------------------
 * Gauss-Hermite points of the standard normal (the x_j of the 7L map g_m,
 * Section "Methodology": x_j are Gauss-Hermite points of X ~ N(0,1)).
 * Probabilists' Hermite polynomials He_0 = 1, He_1 = x,
 * He_{k+1} = x He_k - k He_{k-1}; the nodes are the m roots of He_m and the
 * probability weights are m! / (m^2 He_{m-1}(x_j)^2), which sum to one.
 * Roots are bracketed on a fine grid and refined by bisection (no eigen
 * solver: the library uses Golub-Welsch, the oracle deliberately does not).
 * ---------------------------------------------------------------------- */
static double hermite_e(int n, double x) {
    if (n == 0) return 1.0;
    double prev = 1.0, cur = x;
    for (int k = 1; k < n; ++k) {
        double next = x * cur - (double)k * prev;
        prev = cur;
        cur = next;
    }
    return cur;
}

int orc_gauss_hermite(int m, double* x, double* w) {
    if (m < 1 || m > 64) return 1;
    double R = sqrt(4.0 * m + 2.0) + 1.0;     /* all roots lie in (-R, R) */
    const int n_grid = 20001;                  /* odd count of intervals: 0 is never a grid point */
    int found = 0;
    double a = -R, fa = hermite_e(m, a);
    for (int g = 1; g <= n_grid && found < m; ++g) {
        double b = -R + 2.0 * R * (double)g / (double)n_grid;
        double fb = hermite_e(m, b);
        if ((fa < 0.0 && fb > 0.0) || (fa > 0.0 && fb < 0.0)) {
            double lo = a, hi = b, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double fm = hermite_e(m, mid);
                if (fm == 0.0) { lo = hi = mid; break; }
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            x[found++] = 0.5 * (lo + hi);
        }
        a = b;
        fa = fb;
    }
    if (found != m) return 2;
    /* The roots are symmetric about 0: average each pair, centre exactly 0. */
    for (int j = 0; j < m / 2; ++j) {
        double s = 0.5 * (x[m - 1 - j] - x[j]);
        x[j] = -s;
        x[m - 1 - j] = s;
    }
    if (m % 2 == 1) x[m / 2] = 0.0;
    double mfact = 1.0;
    for (int k = 2; k <= m; ++k) mfact *= (double)k;
    for (int j = 0; j < m; ++j) {
        double h = hermite_e(m - 1, x[j]);
        w[j] = mfact / ((double)m * (double)m * h * h);
    }
    return 0;
}

/* Standard normal CDF. */
static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* 0-based rank of the empirical quantile at level Phi(x_j) among n samples:
 * the inverse empirical CDF, ceil(n * Phi(x_j)) - 1, clamped to [0, n-1]. */
int orc_quantile_ranks(int m, int64_t n, int64_t* ranks) {
    double x[64], w[64];
    if (orc_gauss_hermite(m, x, w) != 0) return 1;
    for (int j = 0; j < m; ++j) {
        double level = std_normal_cdf(x[j]);
        int64_t k = (int64_t)ceil((double)n * level) - 1;
        if (k < 0) k = 0;
        if (k > n - 1) k = n - 1;
        ranks[j] = k;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Lagrange interpolation through (x_j, y_j), j = 0..m-1: the map g_m of the
 * 7L scheme (Section "Methodology", Algorithm I step 5).  Written as the
 * plain definition sum_j y_j prod_{k != j} (X - x_k) / (x_j - x_k); the
 * barycentric rearrangement the paper uses is the same polynomial.
 * ---------------------------------------------------------------------- */
double orc_lagrange(int m, const double* xn, const double* y, double X) {
    double g = 0.0;
    for (int j = 0; j < m; ++j) {
        double l = 1.0;
        for (int k = 0; k < m; ++k)
            if (k != j) l *= (X - xn[k]) / (xn[j] - xn[k]);
        g += y[j] * l;
    }
    return g;
}

/* d g_m / d y_j at X: the Lagrange basis polynomial l_j(X). */
static void lagrange_basis(int m, const double* xn, double X, double* l) {
    for (int j = 0; j < m; ++j) {
        double v = 1.0;
        for (int k = 0; k < m; ++k)
            if (k != j) v *= (X - xn[k]) / (xn[j] - xn[k]);
        l[j] = v;
    }
}

/* ------------------------------------------------------------------------
 * The network H of Eq. (6.3)/(6.4): d_in -> width (x n_hidden) -> m, fully
 * connected.  Parameters are one flat array, layer by layer: W_l (row-major
 * [out][in]) followed by b_l.  Hidden layers apply the activation (ReLU or
 * Softplus), the output layer is linear.
 * ---------------------------------------------------------------------- */
#define ORC_MAX_W 128
#define ORC_MAX_DEG 16   /* polynomial degrees of the 7L-CDC inverse (m - 1 <= 15) */

int64_t orc_n_params(int d_in, int width, int n_hidden, int m) {
    int64_t n = (int64_t)width * d_in + width;
    n += (int64_t)(n_hidden - 1) * ((int64_t)width * width + width);
    n += (int64_t)m * width + m;
    return n;
}

static double act_f(int act, double z) {
    if (act == ORC_ACT_SOFTPLUS) return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
    return z > 0.0 ? z : 0.0;
}

static double act_df(int act, double z) {
    if (act == ORC_ACT_SOFTPLUS) return 1.0 / (1.0 + exp(-z));
    return z > 0.0 ? 1.0 : 0.0;
}

/* Forward pass; if zs/hs are given, store pre-activations and activations of
 * every hidden layer (n_hidden x width each). */
static void mlp_forward(const double* P, int d_in, int width, int n_hidden, int m, int act,
                        const double* f, double* out, double* zs, double* hs) {
    double hin[ORC_MAX_W], h[ORC_MAX_W], z[ORC_MAX_W];
    const double* in = f;
    int n_in = d_in;
    for (int l = 0; l < n_hidden; ++l) {
        const double* W = P;
        const double* b = P + (int64_t)width * n_in;
        for (int o = 0; o < width; ++o) {
            double s = b[o];
            for (int i = 0; i < n_in; ++i) s += W[(int64_t)o * n_in + i] * in[i];
            z[o] = s;
        }
        for (int o = 0; o < width; ++o) h[o] = act_f(act, z[o]);
        if (zs) memcpy(zs + (int64_t)l * width, z, sizeof(double) * width);
        if (hs) memcpy(hs + (int64_t)l * width, h, sizeof(double) * width);
        P += (int64_t)width * n_in + width;
        memcpy(hin, h, sizeof(double) * width);   /* this layer's output is the next one's input */
        in = hin;
        n_in = width;
    }
    const double* W = P;
    const double* b = P + (int64_t)m * n_in;
    for (int o = 0; o < m; ++o) {
        double s = b[o];
        for (int i = 0; i < n_in; ++i) s += W[(int64_t)o * n_in + i] * in[i];
        out[o] = s;
    }
}

void orc_mlp_forward(const double* P, int d_in, int width, int n_hidden, int m, int act,
                     const double* feats, int64_t n_rows, double* out) {
    for (int64_t r = 0; r < n_rows; ++r)
        mlp_forward(P, d_in, width, n_hidden, m, act, feats + r * d_in, out + r * m, NULL, NULL);
}

/* Reverse mode (back-propagation) for one row: given dL/dout (m values),
 * ADD dL/dparams into gP (if non-NULL) and write dL/dfeatures into gf
 * (if non-NULL). */
static void mlp_backward_row(const double* P, int d_in, int width, int n_hidden, int m, int act,
                             const double* f, const double* gout, double* gP, double* gf) {
    double zs[8 * ORC_MAX_W], hs[8 * ORC_MAX_W], out[ORC_MAX_W];
    mlp_forward(P, d_in, width, n_hidden, m, act, f, out, zs, hs);
    /* offsets of each layer's parameters */
    int64_t off[16];
    int64_t o = 0;
    int n_in = d_in;
    for (int l = 0; l < n_hidden; ++l) {
        off[l] = o;
        o += (int64_t)width * n_in + width;
        n_in = width;
    }
    off[n_hidden] = o;
    /* output layer */
    double gh[ORC_MAX_W], gz[ORC_MAX_W];
    {
        const double* W = P + off[n_hidden];
        const double* hin = hs + (int64_t)(n_hidden - 1) * width;
        for (int i = 0; i < width; ++i) {
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += W[(int64_t)k * width + i] * gout[k];
            gh[i] = s;
        }
        if (gP) {
            double* gW = gP + off[n_hidden];
            double* gb = gW + (int64_t)m * width;
            for (int k = 0; k < m; ++k) {
                for (int i = 0; i < width; ++i) gW[(int64_t)k * width + i] += gout[k] * hin[i];
                gb[k] += gout[k];
            }
        }
    }
    for (int l = n_hidden - 1; l >= 0; --l) {
        int nin = (l == 0) ? d_in : width;
        const double* in = (l == 0) ? f : hs + (int64_t)(l - 1) * width;
        const double* z = zs + (int64_t)l * width;
        for (int k = 0; k < width; ++k) gz[k] = gh[k] * act_df(act, z[k]);
        const double* W = P + off[l];
        if (gP) {
            double* gW = gP + off[l];
            double* gb = gW + (int64_t)width * nin;
            for (int k = 0; k < width; ++k) {
                for (int i = 0; i < nin; ++i) gW[(int64_t)k * nin + i] += gz[k] * in[i];
                gb[k] += gz[k];
            }
        }
        double gin[ORC_MAX_W];
        for (int i = 0; i < nin; ++i) {
            double s = 0.0;
            for (int k = 0; k < width; ++k) s += W[(int64_t)k * nin + i] * gz[k];
            gin[i] = s;
        }
        if (l == 0) {
            if (gf) memcpy(gf, gin, sizeof(double) * d_in);
        } else {
            memcpy(gh, gin, sizeof(double) * width);
        }
    }
}

/* Mean-squared error over a batch of rows and all m outputs,
 * L = 1/(n_rows*m) sum_r sum_j (H_j(f_r) - y_rj)^2, and its gradient with
 * respect to the parameters (written to gP, overwritten). */
double orc_mse_grad(const double* P, int d_in, int width, int n_hidden, int m, int act,
                    const double* feats, const double* labels, const int32_t* rows, int64_t n_rows,
                    double* gP) {
    int64_t np = orc_n_params(d_in, width, n_hidden, m);
    if (gP) memset(gP, 0, sizeof(double) * np);
    double loss = 0.0;
    double scale = 1.0 / ((double)n_rows * (double)m);
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t row = rows ? rows[r] : r;
        const double* f = feats + row * d_in;
        const double* y = labels + row * m;
        double out[ORC_MAX_W], gout[ORC_MAX_W];
        mlp_forward(P, d_in, width, n_hidden, m, act, f, out, NULL, NULL);
        for (int j = 0; j < m; ++j) {
            double e = out[j] - y[j];
            loss += e * e * scale;
            gout[j] = 2.0 * e * scale;
        }
        if (gP) mlp_backward_row(P, d_in, width, n_hidden, m, act, f, gout, gP, NULL);
    }
    return loss;
}

/* Input gradient of sum_j c_j H_j(f) for each row (a vector-Jacobian product). */
void orc_mlp_vjp_input(const double* P, int d_in, int width, int n_hidden, int m, int act,
                       const double* feats, const double* c, int64_t n_rows, double* gfeats) {
    for (int64_t r = 0; r < n_rows; ++r)
        mlp_backward_row(P, d_in, width, n_hidden, m, act, feats + r * d_in, c + r * m, NULL,
                         gfeats + r * d_in);
}

/* ------------------------------------------------------------------------
 * Adam (Kingma & Ba 2015), the optimiser named in the experiments section:
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   P <- P - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * Runs n_batches steps, step counter t = t0+1 .. t0+n_batches; batch b uses
 * rows batch_rows[b*batch .. b*batch+batch-1].  Loss of each batch (before
 * its update) goes to losses[b].
 * ---------------------------------------------------------------------- */
void orc_train_adam(double* P, double* am, double* av, int64_t t0, int d_in, int width,
                    int n_hidden, int m, int act, const double* feats, const double* labels,
                    const int32_t* batch_rows, int n_batches, int batch, double lr, double b1,
                    double b2, double eps, double* losses) {
    int64_t np = orc_n_params(d_in, width, n_hidden, m);
    double* g = (double*)malloc(sizeof(double) * np);
    for (int b = 0; b < n_batches; ++b) {
        double loss = orc_mse_grad(P, d_in, width, n_hidden, m, act, feats, labels,
                                   batch_rows + (int64_t)b * batch, batch, g);
        if (losses) losses[b] = loss;
        double t = (double)(t0 + b + 1);
        double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
        for (int64_t i = 0; i < np; ++i) {
            am[i] = b1 * am[i] + (1.0 - b1) * g[i];
            av[i] = b2 * av[i] + (1.0 - b2) * g[i] * g[i];
            P[i] -= lr * (am[i] / c1) / (sqrt(av[i] / c2) + eps);
        }
    }
    free(g);
}

/* ------------------------------------------------------------------------
 * Conditional collocation points y_j | Y_i  (Eq. 6.3 / 6.4).
 *  - MLP: the network with features [Y_i, dt, theta_0..theta_{p-1}].
 *  - GBM_EXACT, theta = (mu, sigma): the exact lognormal quantile map,
 *      y_j = Y_i exp((mu - sigma^2/2) dt + sigma sqrt(dt) x_j).
 *  - OU_EXACT, theta = (Ybar, sigma, lambda), Eq. (6.5)/(6.6) restarted at Y_i:
 *      y_j = e^{-lambda dt} Y_i + Ybar (1 - e^{-lambda dt})
 *            + sigma sqrt((1 - e^{-2 lambda dt}) / (2 lambda)) x_j.
 * With tangents: dy[j*(1+p) + q] = d y_j / d(Y_i, theta)_q (q = 0 is Y_i).
 * ---------------------------------------------------------------------- */
typedef struct {
    int model, d_in, width, n_hidden, act, m, p;
    const double* P;
    const double* xn;
} orc_net;

static void collocation(const orc_net* N, double Y, double dt, const double* th, double* y,
                        double* dy) {
    int m = N->m, p = N->p, q1 = 1 + p;
    if (N->model == ORC_MODEL_GBM_EXACT) {
        double mu = th[0], sg = th[1], sdt = sqrt(dt);
        for (int j = 0; j < m; ++j) {
            double e = exp((mu - 0.5 * sg * sg) * dt + sg * sdt * N->xn[j]);
            y[j] = Y * e;
            if (dy) {
                dy[j * q1 + 0] = e;
                dy[j * q1 + 1] = y[j] * dt;
                dy[j * q1 + 2] = y[j] * (-sg * dt + sdt * N->xn[j]);
            }
        }
        return;
    }
    if (N->model == ORC_MODEL_OU_EXACT) {
        double yb = th[0], sg = th[1], lam = th[2];
        double e1 = exp(-lam * dt), e2 = exp(-2.0 * lam * dt);
        double s2 = (1.0 - e2) / (2.0 * lam), s = sqrt(s2);
        double ds2 = dt * e2 / lam - (1.0 - e2) / (2.0 * lam * lam);
        double ds = ds2 / (2.0 * s);
        for (int j = 0; j < m; ++j) {
            y[j] = e1 * Y + yb * (1.0 - e1) + sg * s * N->xn[j];
            if (dy) {
                dy[j * q1 + 0] = e1;
                dy[j * q1 + 1] = 1.0 - e1;
                dy[j * q1 + 2] = s * N->xn[j];
                dy[j * q1 + 3] = -dt * e1 * Y + yb * dt * e1 + sg * ds * N->xn[j];
            }
        }
        return;
    }
    double f[64];
    f[0] = Y;
    f[1] = dt;
    for (int k = 0; k < p; ++k) f[2 + k] = th[k];
    mlp_forward(N->P, N->d_in, N->width, N->n_hidden, m, N->act, f, y, NULL, NULL);
    if (dy) {
        /* Jacobian row by row: reverse mode with unit output cotangents. */
        for (int j = 0; j < m; ++j) {
            double c[ORC_MAX_W] = {0}, gf[64];
            c[j] = 1.0;
            mlp_backward_row(N->P, N->d_in, N->width, N->n_hidden, m, N->act, f, c, NULL, gf);
            dy[j * q1 + 0] = gf[0];
            for (int k = 0; k < p; ++k) dy[j * q1 + 1 + k] = gf[2 + k];
        }
    }
}

/* Largest s with offsets[s] <= g (the set owning flat path g; empty sets skipped). */
static int owning_set(const int64_t* offsets, int n_sets, int64_t g) {
    int lo = 0, hi = n_sets - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (offsets[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------
 * Algorithm I, online stage (steps 2-8) for one path of set s:
 *   Y_0 given; for i = 0..n_steps-1: y = H(Y_i, dt, theta_s) (step 3),
 *   draw X_{i+1} (step 6), Y_{i+1} = g_m(X_{i+1}) (steps 5-6).
 * The normal for step i is orc_normal(seed, tag 0, s, path-in-set, i).
 * If tangent is non-NULL it receives dY_T / d(Y0, theta) (1+p values),
 * propagated forward step by step (forward-mode chain rule).
 * ---------------------------------------------------------------------- */
static double path_7l(const orc_net* N, const double* th, double Y0, double T, int n_steps,
                      uint64_t seed, uint32_t set, uint32_t path, double* grid, double* tangent) {
    int m = N->m, p = N->p, q1 = 1 + p;
    double dt = T / (double)n_steps;
    double Y = Y0;
    double tg[16] = {0};
    tg[0] = 1.0;
    if (grid) grid[0] = Y;
    for (int i = 0; i < n_steps; ++i) {
        double y[ORC_MAX_W], dy[ORC_MAX_W * 16], l[ORC_MAX_W];
        collocation(N, Y, dt, th, y, tangent ? dy : NULL);
        double X = orc_normal(seed, ORC_TAG_7L, set, path, (uint32_t)i);
        double Ynew = orc_lagrange(m, N->xn, y, X);
        if (tangent) {
            lagrange_basis(m, N->xn, X, l);
            double ntg[16] = {0};
            for (int q = 0; q < q1; ++q) {
                double s = 0.0;
                for (int j = 0; j < m; ++j) {
                    /* chain rule through Y_i, plus the direct theta dependence */
                    double dyq = dy[j * q1 + 0] * tg[q];
                    if (q >= 1) dyq += dy[j * q1 + q];
                    s += l[j] * dyq;
                }
                ntg[q] = s;
            }
            memcpy(tg, ntg, sizeof(double) * q1);
        }
        Y = Ynew;
        if (grid) grid[i + 1] = Y;
    }
    if (tangent) memcpy(tangent, tg, sizeof(double) * q1);
    return Y;
}

/* Evaluate selected flat paths (idx == NULL: all of them) of a batched call.
 * theta is [n_sets][p]; Y0 is [n_sets]; offsets is the exclusive prefix of
 * per-set path counts ([n_sets+1]).  out_YT[k] is Y_T of path idx[k]; the
 * optional out_grid[k*(n_steps+1) + i] is Y_i. */
int orc_7l_paths(int model, const double* P, int d_in, int width, int n_hidden, int act,
                 const double* theta, int p, const double* Y0, const int64_t* offsets, int n_sets,
                 double T, int n_steps, int m, uint64_t seed, const int64_t* idx, int64_t n_idx,
                 double* out_YT, double* out_grid, int n_threads) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    orc_net N = {model, d_in, width, n_hidden, act, m, p, P, xn};
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t g = idx ? idx[k] : k;
        int s = owning_set(offsets, n_sets, g);
        uint32_t q = (uint32_t)(g - offsets[s]);
        out_YT[k] = path_7l(&N, theta + (int64_t)s * p, Y0[s], T, n_steps, seed, (uint32_t)s, q,
                            out_grid ? out_grid + k * (int64_t)(n_steps + 1) : NULL, NULL);
    }
    return 0;
}

/* Per-set mean and unbiased sample variance of Y_T over ALL paths of every
 * set (variance 0 when a set has fewer than two paths). */
int orc_7l_moments(int model, const double* P, int d_in, int width, int n_hidden, int act,
                   const double* theta, int p, const double* Y0, const int64_t* offsets,
                   int n_sets, double T, int n_steps, int m, uint64_t seed, double* out_mean,
                   double* out_var, int n_threads) {
    int64_t total = offsets[n_sets];
    double* yt = (double*)malloc(sizeof(double) * (total > 0 ? total : 1));
    int rc = orc_7l_paths(model, P, d_in, width, n_hidden, act, theta, p, Y0, offsets, n_sets, T,
                          n_steps, m, seed, NULL, total, yt, NULL, n_threads);
    if (rc) { free(yt); return rc; }
    for (int s = 0; s < n_sets; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1], n = b - a;
        double mean = 0.0;
        for (int64_t g = a; g < b; ++g) mean += yt[g];
        mean = n > 0 ? mean / (double)n : 0.0;
        double ss = 0.0;
        for (int64_t g = a; g < b; ++g) ss += (yt[g] - mean) * (yt[g] - mean);
        out_mean[s] = mean;
        if (out_var) out_var[s] = n > 1 ? ss / (double)(n - 1) : 0.0;
    }
    free(yt);
    return 0;
}

/* Pathwise sensitivities of the call payoff f = max(Y_T - K, 0):
 * per selected path, value[k] = f(Y_T) and grad[k*(1+p) + q] =
 * 1{Y_T > K} dY_T/d(Y0, theta)_q, by forward-mode propagation of dY/d(Y0, theta). */
int orc_7l_payoff_grad(int model, const double* P, int d_in, int width, int n_hidden, int act,
                       const double* theta, int p, const double* Y0, const int64_t* offsets,
                       int n_sets, double T, int n_steps, int m, uint64_t seed, double K,
                       const int64_t* idx, int64_t n_idx, double* out_YT, double* value,
                       double* grad, int n_threads) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    orc_net N = {model, d_in, width, n_hidden, act, m, p, P, xn};
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t g = idx ? idx[k] : k;
        int s = owning_set(offsets, n_sets, g);
        uint32_t q = (uint32_t)(g - offsets[s]);
        double tg[16];
        double YT = path_7l(&N, theta + (int64_t)s * p, Y0[s], T, n_steps, seed, (uint32_t)s, q,
                            NULL, tg);
        if (out_YT) out_YT[k] = YT;
        value[k] = YT > K ? YT - K : 0.0;
        for (int c = 0; c < 1 + p; ++c) grad[k * (1 + p) + c] = YT > K ? tg[c] : 0.0;
    }
    return 0;
}

/* Smallest |pre-activation| of any hidden unit over the network evaluations
 * at Y_0 .. Y_{n_steps-1} of each selected path (MLP model).  The ReLU
 * network is piecewise linear: its derivative jumps where a pre-activation
 * crosses 0, so two evaluations that differ by rounding can only disagree on
 * the derivative of paths whose margin is of the size of that rounding. */
int orc_7l_relu_margin(const double* P, int d_in, int width, int n_hidden, const double* theta,
                       int p, const double* Y0, const int64_t* offsets, int n_sets, double T,
                       int n_steps, int m, uint64_t seed, const int64_t* idx, int64_t n_idx,
                       double* margin, int n_threads) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    if (n_hidden > 8 || width > ORC_MAX_W) return 1;
    orc_net N = {ORC_MODEL_MLP, d_in, width, n_hidden, ORC_ACT_RELU, m, p, P, xn};
    double dt = T / (double)n_steps;
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t g = idx ? idx[k] : k;
        int s = owning_set(offsets, n_sets, g);
        uint32_t q = (uint32_t)(g - offsets[s]);
        const double* th = theta + (int64_t)s * p;
        double* grid = (double*)malloc(sizeof(double) * (size_t)(n_steps + 1));
        path_7l(&N, th, Y0[s], T, n_steps, seed, (uint32_t)s, q, grid, NULL);
        double mg = INFINITY;
        for (int i = 0; i < n_steps; ++i) {
            double f[64], y[ORC_MAX_W], zs[8 * ORC_MAX_W];
            f[0] = grid[i];
            f[1] = dt;
            for (int c = 0; c < p; ++c) f[2 + c] = th[c];
            mlp_forward(P, d_in, width, n_hidden, m, ORC_ACT_RELU, f, y, zs, NULL);
            for (int u = 0; u < n_hidden * width; ++u) mg = fabs(zs[u]) < mg ? fabs(zs[u]) : mg;
        }
        margin[k] = mg;
        free(grid);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Offline stage (Algorithm I step 1): Euler-Maruyama, Eq. (6.2), with
 * n_fine steps of d_tau = dt / n_fine from Y_i, normals from stream
 * (seed, tag 1, row, path), fine step k using normal number k.
 *   GBM (mu, sigma):          a = mu Y,             b = sigma Y
 *   OU  (Ybar, sigma, lambda): a = -lambda (Y - Ybar), b = sigma        (Eq. 6.5)
 *   CIR (kappa, ybar, gamma):  full truncation, a = kappa (ybar - Y+),
 *                              b = gamma sqrt(Y+), Y+ = max(Y, 0);
 *                              the returned sample is Y+ at the end.
 * ---------------------------------------------------------------------- */
static double em_path(int sde, const double* th, double Y, double dt, int n_fine, uint64_t seed,
                      uint32_t row, uint32_t path) {
    double dtau = dt / (double)n_fine, sq = sqrt(dtau);
    for (int k = 0; k < n_fine; ++k) {
        double X = orc_normal(seed, ORC_TAG_EM, row, path, (uint32_t)k);
        double a, b;
        if (sde == ORC_SDE_GBM) {
            a = th[0] * Y;
            b = th[1] * Y;
        } else if (sde == ORC_SDE_OU) {
            a = -th[2] * (Y - th[0]);
            b = th[1];
        } else {
            double yp = Y > 0.0 ? Y : 0.0;
            a = th[0] * (th[1] - yp);
            b = th[2] * sqrt(yp);
        }
        Y = Y + a * dtau + b * sq * X;
    }
    if (sde == ORC_SDE_CIR && Y < 0.0) Y = 0.0;
    return Y;
}

static int sde_p(int sde) { return sde == ORC_SDE_GBM ? 2 : 3; }

/* Terminal EM samples: out[r*n_paths + q] for rows r in [row0, row0+n_rows). */
int orc_em_terminal(int sde, const double* theta, const double* Yi, const double* dt, int row0,
                    int n_rows, int64_t n_paths, int n_fine, uint64_t seed, double* out,
                    int n_threads) {
    int p = sde_p(sde);
    set_threads(n_threads);
#pragma omp parallel for collapse(2) schedule(static)
    for (int r = 0; r < n_rows; ++r)
        for (int64_t q = 0; q < n_paths; ++q) {
            int row = row0 + r;
            out[(int64_t)r * n_paths + q] = em_path(sde, theta + (int64_t)row * p, Yi[row], dt[row],
                                                    n_fine, seed, (uint32_t)row, (uint32_t)q);
        }
    return 0;
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* k-th smallest (0-based) of each segment by sorting it: out[s*n_k + j] =
 * sorted(values[off[s]..off[s+1]))[ranks[j]]. */
int orc_order_statistics(const double* values, const int64_t* seg_off, int n_seg,
                         const int64_t* ranks, int n_k, double* out) {
    for (int s = 0; s < n_seg; ++s) {
        int64_t n = seg_off[s + 1] - seg_off[s];
        double* tmp = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
        memcpy(tmp, values + seg_off[s], sizeof(double) * n);
        qsort(tmp, (size_t)n, sizeof(double), cmp_double);
        for (int j = 0; j < n_k; ++j) out[(int64_t)s * n_k + j] = (ranks[j] < n) ? tmp[ranks[j]] : NAN;
        free(tmp);
    }
    return 0;
}

/* Collocation labels y_j | (theta, Y_i, dt) (Algorithm I step 1): the
 * empirical quantiles of n_paths EM terminal samples at levels Phi(x_j). */
int orc_em_labels(int sde, const double* theta, const double* Yi, const double* dt, int row0,
                  int n_rows, int64_t n_paths, int n_fine, int m, uint64_t seed, double* labels,
                  int n_threads) {
    int64_t ranks[64];
    if (orc_quantile_ranks(m, n_paths, ranks) != 0) return 1;
    double* buf = (double*)malloc(sizeof(double) * n_paths);
    for (int r = 0; r < n_rows; ++r) {
        orc_em_terminal(sde, theta, Yi, dt, row0 + r, 1, n_paths, n_fine, seed, buf, n_threads);
        int64_t off[2] = {0, n_paths};
        orc_order_statistics(buf, off, 1, ranks, m, labels + (int64_t)r * m);
    }
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------
 * The 7L-CDC variant (the remark after Algorithm I and the discussion of
 * Table 6.1): step 3 of Algorithm I -- the network evaluated for every path --
 * is replaced by a global interpolation built from a few network evaluations
 * per parameter set and time step.  The paper describes the variant in outline
 * only; the reading taken here:
 *
 *  - Marginal collocation points of Y at t_i = i dt (i >= 1): z_k = G_k(Y0,
 *    t_i, theta), k = 0..m-1, the collocation map at the same Gauss-Hermite
 *    abscissae x_k over the horizon t_i from the deterministic start Y0 (the
 *    law of Y_{t_i} given Y_0 is the marginal law).  G is the marginal network
 *    (features [Y0, t_i, theta]) or, for the exact models, the exact map with
 *    dt replaced by t_i.  At i = 0 the marginal is the point mass at Y0.
 *  - Conditional collocation points at the marginal nodes:
 *    C[k][j] = H_j(z_k, dt, theta) (m network evaluations).
 *  - Per path at Y_i: yhat_j = sum_k C[k][j] L_k(Y_i), the Lagrange
 *    interpolation in Y through the nodes z_k (the "global interpolation"),
 *    continued linearly beyond the outermost nodes (orc_cdc_conditional_points);
 *    then Y_{i+1} = g_m(X_{i+1}) through (x_j, yhat_j), with the same normals
 *    as the 7L scheme (tag 0).
 *  - If the marginal nodes all coincide (i = 0, or a degenerate law) every
 *    path sits at that point and yhat_j = C[0][j].
 * With a conditional map that is a polynomial of degree <= m-1 in Y (the
 * exact GBM and OU maps are linear in Y) the interpolation in Y is exact and
 * the 7L-CDC chain equals the 7L chain.
 * ---------------------------------------------------------------------- */

/* yhat_j at Y from the conditional points C[k*m + j] at the marginal nodes z_k:
 *  - all z_k equal: row 0;
 *  - Y inside [min z, max z]: sum_k C[k][j] L_k(Y), L_k the Lagrange basis
 *    through the z_k (plain definition);
 *  - Y beyond the outermost node on one side: the straight line through that
 *    node and the next one on the same side (a polynomial of degree m-1 grows
 *    without bound away from its nodes; the line agrees with the polynomial at
 *    the outermost node, and both are exact for maps affine in Y). */
void orc_cdc_conditional_points(int m, const double* z, const double* C, double Y, double* yhat) {
    int same = 1;
    for (int k = 1; k < m; ++k)
        if (z[k] != z[0]) same = 0;
    if (same) {
        for (int j = 0; j < m; ++j) yhat[j] = C[j];
        return;
    }
    /* the two smallest and the two largest nodes (ties keep the lower index) */
    int lo = 0, hi = 0;
    for (int k = 1; k < m; ++k) {
        if (z[k] < z[lo]) lo = k;
        if (z[k] > z[hi]) hi = k;
    }
    int lo2 = -1, hi2 = -1;
    for (int k = 0; k < m; ++k) {
        if (k != lo && (lo2 < 0 || z[k] < z[lo2])) lo2 = k;
        if (k != hi && (hi2 < 0 || z[k] > z[hi2])) hi2 = k;
    }
    if (Y < z[lo] || Y > z[hi]) {
        int a = Y < z[lo] ? lo : hi, b = Y < z[lo] ? lo2 : hi2;
        for (int j = 0; j < m; ++j)
            yhat[j] = C[a * m + j] + (Y - z[a]) * (C[b * m + j] - C[a * m + j]) / (z[b] - z[a]);
        return;
    }
    for (int j = 0; j < m; ++j) yhat[j] = 0.0;
    for (int k = 0; k < m; ++k) {
        double L = 1.0;
        for (int l = 0; l < m; ++l)
            if (l != k) L *= (Y - z[l]) / (z[k] - z[l]);
        for (int j = 0; j < m; ++j) yhat[j] += C[k * m + j] * L;
    }
}

/* Tables of the sets sets[r] (r < n_sel; sets == NULL: every set, r = s), every step i:
 * z[(r*n_steps + i)*m + k] and C[((r*n_steps + i)*m + k)*m + j].  Pm: the marginal
 * network's parameters (the same shape as P; NULL: P itself). */
int orc_cdc_tables(int model, const double* P, const double* Pm, int d_in, int width, int n_hidden,
                   int act, const double* theta, int p, const double* Y0, int n_sets, double T,
                   int n_steps, int m, const int64_t* sets, int64_t n_sel, double* z, double* C) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    orc_net N = {model, d_in, width, n_hidden, act, m, p, P, xn};
    orc_net NM = {model, d_in, width, n_hidden, act, m, p, Pm ? Pm : P, xn};
    double dt = T / (double)n_steps;
    int64_t n_rows = sets ? n_sel : n_sets;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t s = sets ? sets[r] : r;
        const double* th = theta + s * p;
        for (int i = 0; i < n_steps; ++i) {
            double* zi = z + (r * n_steps + i) * m;
            double* Ci = C + (r * n_steps + i) * m * m;
            if (i == 0) {
                for (int k = 0; k < m; ++k) zi[k] = Y0[s];
            } else {
                collocation(&NM, Y0[s], i * dt, th, zi, NULL);
            }
            for (int k = 0; k < m; ++k) collocation(&N, zi[k], dt, th, Ci + k * m, NULL);
        }
    }
    return 0;
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Y_T (and optionally the grid) of selected flat paths of a batched 7L-CDC
 * call; arguments as orc_7l_paths plus the marginal network Pm. */
int orc_cdc_paths(int model, const double* P, const double* Pm, int d_in, int width, int n_hidden,
                  int act, const double* theta, int p, const double* Y0, const int64_t* offsets,
                  int n_sets, double T, int n_steps, int m, uint64_t seed, const int64_t* idx,
                  int64_t n_idx, double* out_YT, double* out_grid, int n_threads) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    /* the tables of the sets the selected paths belong to (sorted, distinct) */
    int64_t* sets = (int64_t*)malloc(sizeof(int64_t) * (n_idx > 0 ? n_idx : 1));
    if (!sets) return 1;
    for (int64_t k = 0; k < n_idx; ++k) sets[k] = owning_set(offsets, n_sets, idx ? idx[k] : k);
    qsort(sets, (size_t)n_idx, sizeof(int64_t), cmp_i64);
    int64_t n_sel = 0;
    for (int64_t k = 0; k < n_idx; ++k)
        if (n_sel == 0 || sets[k] != sets[n_sel - 1]) sets[n_sel++] = sets[k];
    size_t nt = (size_t)(n_sel > 0 ? n_sel : 1) * n_steps;
    double* z = (double*)malloc(sizeof(double) * nt * m);
    double* C = (double*)malloc(sizeof(double) * nt * m * m);
    if (!z || !C) { free(sets); free(z); free(C); return 1; }
    set_threads(n_threads);
    int rc = orc_cdc_tables(model, P, Pm, d_in, width, n_hidden, act, theta, p, Y0, n_sets, T,
                            n_steps, m, sets, n_sel, z, C);
    if (rc) { free(sets); free(z); free(C); return rc; }
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t g = idx ? idx[k] : k;
        int s = owning_set(offsets, n_sets, g);
        uint32_t q = (uint32_t)(g - offsets[s]);
        int64_t key = s, *hit = (int64_t*)bsearch(&key, sets, (size_t)n_sel, sizeof(int64_t), cmp_i64);
        int64_t row = hit - sets;
        double* grid = out_grid ? out_grid + k * (int64_t)(n_steps + 1) : NULL;
        double Y = Y0[s];
        if (grid) grid[0] = Y;
        for (int i = 0; i < n_steps; ++i) {
            double yhat[ORC_MAX_W];
            size_t r = (size_t)row * n_steps + i;
            orc_cdc_conditional_points(m, z + r * m, C + r * m * m, Y, yhat);
            double X = orc_normal(seed, ORC_TAG_7L, (uint32_t)s, q, (uint32_t)i);
            Y = orc_lagrange(m, xn, yhat, X);
            if (grid) grid[i + 1] = Y;
        }
        out_YT[k] = Y;
    }
    free(sets);
    free(z);
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------
 * The 7L-CDC variant in the marginal's quantile coordinate (a second reading of
 * the same outline).  The marginal collocation points z^(i)_k of Y at t_i define
 * the marginal collocation map G_i(xi) = sum_k z^(i)_k L_k(xi) through the
 * Gauss-Hermite points x_k (the SCMC representation of Y_{t_i}: Y = G_i(xi) with
 * xi standard normal), continued beyond [x_0, x_{m-1}] by the line through the two
 * outermost nodes on that side.  A path carries xi_i instead of Y_i:
 *  - eta[k][j] = G_{i+1}^{-1}(C[k][j]): the conditional points at the marginal
 *    nodes of t_i, expressed in the quantile coordinate of t_{i+1};
 *  - xi_{i+1} = sum_k sum_j eta[k][j] L_k(xi_i) L_j(X_{i+1}) (Lagrange in both
 *    variables through the Gauss-Hermite points) for xi_i in [x_0, x_{m-1}];
 *    beyond, the line in xi through the two outermost node rows (degree m-1
 *    extrapolation in xi grows without bound along a path, as in Y);
 *  - Y_i = G_i(xi_i) wherever Y is output (the grid, Y_T = G_N(xi_N)).
 * At i = 0 the marginal is the point Y0: every row of C is H(Y0, dt), so xi_1
 * does not depend on xi_0 (taken as 0).  If the nodes at t_{i+1} all coincide,
 * G_{i+1} is constant: eta = 0 and Y_{i+1} = z^(i+1)_0.  G must increase from
 * its first to its last node (z_0 < z_{m-1}); the inverse inside the hull is
 * the smallest root of G(xi) = y in the first node interval [x_k, x_{k+1}]
 * with z_k <= y <= z_{k+1} (one exists whenever z_0 <= y <= z_{m-1}).  For a
 * G that increases it is the one root; a G that wiggles inside a node interval
 * can cross y several times, and the definition takes the first crossing, at
 * whatever distance the later ones lie.  It is found without any grid: the
 * roots of G' split the interval into pieces on which G is monotone (Rolle),
 * and the first piece on which G - y reaches zero holds the root, found there
 * by bisection.
 * With the exact OU map (G linear, C affine in z and x_j) the chain equals the
 * 7L chain exactly.
 * ---------------------------------------------------------------------- */

/* G(xi) through (x_k, z_k), k < m, with the linear continuation. */
double orc_cdcq_G(int m, const double* xn, const double* z, double xi) {
    if (xi < xn[0]) return z[0] + (xi - xn[0]) * (z[1] - z[0]) / (xn[1] - xn[0]);
    if (xi > xn[m - 1])
        return z[m - 1] + (xi - xn[m - 1]) * (z[m - 1] - z[m - 2]) / (xn[m - 1] - xn[m - 2]);
    return orc_lagrange(m, xn, z, xi);
}

/* Monomial coefficients c[0..m-1] of the interpolant through (xn[k], z[k]):
 * each Lagrange basis polynomial prod_{l != k} (xi - x_l) / (x_k - x_l)
 * multiplied out, weighted by z_k and summed. */
static void lagrange_monomials(int m, const double* xn, const double* z, double* c) {
    for (int a = 0; a < m; ++a) c[a] = 0.0;
    for (int k = 0; k < m; ++k) {
        double b[ORC_MAX_DEG + 1] = {1.0}, den = 1.0;
        int deg = 0;
        for (int l = 0; l < m; ++l) {
            if (l == k) continue;
            b[deg + 1] = 0.0;
            for (int a = deg + 1; a >= 1; --a) b[a] = b[a - 1] - xn[l] * b[a];
            b[0] = -xn[l] * b[0];
            ++deg;
            den *= xn[k] - xn[l];
        }
        for (int a = 0; a < m; ++a) c[a] += z[k] * b[a] / den;
    }
}

static double poly_at(int n, const double* c, double x) {
    double v = 0.0;
    for (int a = n; a >= 0; --a) v = v * x + c[a];
    return v;
}

/* Bisection for the root of f on [lo, hi], given f(lo) < 0 < f(hi) or
 * f(lo) > 0 > f(hi), until the midpoint no longer moves. */
static double bisect_poly(int n, const double* c, double lo, double hi) {
    const int neg_lo = poly_at(n, c, lo) < 0.0;
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if ((poly_at(n, c, mid) < 0.0) == neg_lo) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* The real roots in [a, b] of the degree-n polynomial c, ascending.  Between
 * consecutive roots of the derivative the polynomial is monotone (Rolle), so
 * each such piece holds at most one root: a piece end where it vanishes, or a
 * sign change inside, found by bisection. */
static int poly_roots_in(int n, const double* c, double a, double b, double* r) {
    if (n <= 0) return 0;
    if (n == 1) {
        if (c[1] == 0.0) return 0;
        double t = -c[0] / c[1];
        if (t >= a && t <= b) { r[0] = t; return 1; }
        return 0;
    }
    double d[ORC_MAX_DEG], cr[ORC_MAX_DEG], cut[ORC_MAX_DEG + 2];
    for (int i = 1; i <= n; ++i) d[i - 1] = i * c[i];
    int ncr = poly_roots_in(n - 1, d, a, b, cr), nc = 0, nr = 0;
    cut[nc++] = a;
    for (int i = 0; i < ncr; ++i)
        if (cr[i] > cut[nc - 1] && cr[i] < b) cut[nc++] = cr[i];
    cut[nc++] = b;
    for (int s = 0; s + 1 < nc; ++s) {
        double lo = cut[s], hi = cut[s + 1], flo = poly_at(n, c, lo), fhi = poly_at(n, c, hi);
        double t;
        if (flo == 0.0) t = lo;
        else if (fhi != 0.0 && (flo < 0.0) != (fhi < 0.0)) t = bisect_poly(n, c, lo, hi);
        else continue;
        if (nr == 0 || t > r[nr - 1]) r[nr++] = t;
    }
    if (poly_at(n, c, b) == 0.0 && (nr == 0 || b > r[nr - 1])) r[nr++] = b;
    return nr;
}

/* G^{-1}(y): the continuation lines beyond [z_0, z_{m-1}]; inside, the
 * smallest root of G(xi) = y in the first node interval [x_k, x_{k+1}] with
 * z_k <= y <= z_{k+1}.  G - y is negative at x_k (unless y = z_k, when x_k is
 * the root) and not negative at x_{k+1}; the roots of G' cut the interval into
 * monotone pieces, and the first piece whose far end has G - y >= 0 holds the
 * root (bisection on G's plain Lagrange form).  NaN if G does not increase
 * from its first to its last node; 0 if all nodes coincide. */
double orc_cdcq_Ginv(int m, const double* xn, const double* z, double y) {
    int same = 1;
    for (int k = 1; k < m; ++k)
        if (z[k] != z[0]) same = 0;
    if (same) return 0.0;
    if (!(z[m - 1] > z[0])) return NAN;
    if (y < z[0]) return xn[0] + (y - z[0]) * (xn[1] - xn[0]) / (z[1] - z[0]);
    if (y > z[m - 1]) return xn[m - 1] + (y - z[m - 1]) * (xn[m - 1] - xn[m - 2]) / (z[m - 1] - z[m - 2]);
    int k = 0;
    while (k < m - 2 && !(z[k] <= y && y <= z[k + 1])) ++k;
    if (y == z[k]) return xn[k];
    double c[ORC_MAX_DEG + 1], d[ORC_MAX_DEG], cr[ORC_MAX_DEG], cut[ORC_MAX_DEG + 2];
    lagrange_monomials(m, xn, z, c);
    for (int i = 1; i < m; ++i) d[i - 1] = i * c[i];
    int ncr = poly_roots_in(m - 2, d, xn[k], xn[k + 1], cr), nc = 0;
    cut[nc++] = xn[k];
    for (int i = 0; i < ncr; ++i)
        if (cr[i] > cut[nc - 1] && cr[i] < xn[k + 1]) cut[nc++] = cr[i];
    cut[nc++] = xn[k + 1];
    for (int s = 0; s + 1 < nc; ++s) {
        double lo = cut[s], hi = cut[s + 1];
        double fhi = (s + 2 == nc) ? z[k + 1] - y : orc_lagrange(m, xn, z, hi) - y;
        if (fhi < 0.0) continue;              /* G - y < 0 on the whole piece */
        if (fhi == 0.0) return hi;
        for (int it = 0; it < 2000; ++it) {   /* G - y < 0 at lo, > 0 at hi */
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (orc_lagrange(m, xn, z, mid) < y) lo = mid; else hi = mid;
        }
        return 0.5 * (lo + hi);
    }
    return xn[k + 1];                         /* not reached: G - y >= 0 at x_{k+1} */
}

/* sum_k sum_j eta[k*m + j] L_k(xi) L_j(X) (plain Lagrange definition) for xi in
 * [x_0, x_{m-1}]; beyond, the line in xi through the two outermost node rows
 * (R_k(X) = sum_j eta[k][j] L_j(X)), as the interpolation in Y is continued. */
static double cdcq_row(int m, const double* xn, const double* eta, int k, double X) {
    double r = 0.0;
    for (int j = 0; j < m; ++j) {
        double Lj = 1.0;
        for (int l = 0; l < m; ++l)
            if (l != j) Lj *= (X - xn[l]) / (xn[j] - xn[l]);
        r += eta[k * m + j] * Lj;
    }
    return r;
}

double orc_cdcq_F(int m, const double* xn, const double* eta, double xi, double X) {
    if (xi < xn[0] || xi > xn[m - 1]) {
        int a = xi < xn[0] ? 0 : m - 1, b = xi < xn[0] ? 1 : m - 2;
        double ra = cdcq_row(m, xn, eta, a, X), rb = cdcq_row(m, xn, eta, b, X);
        return ra + (xi - xn[a]) * (rb - ra) / (xn[b] - xn[a]);
    }
    double v = 0.0;
    for (int k = 0; k < m; ++k) {
        double Lk = 1.0;
        for (int l = 0; l < m; ++l)
            if (l != k) Lk *= (xi - xn[l]) / (xn[k] - xn[l]);
        double row = 0.0;
        for (int j = 0; j < m; ++j) {
            double Lj = 1.0;
            for (int l = 0; l < m; ++l)
                if (l != j) Lj *= (X - xn[l]) / (xn[j] - xn[l]);
            row += eta[k * m + j] * Lj;
        }
        v += Lk * row;
    }
    return v;
}

/* Tables of the sets sets[r] (NULL: every set), every step i: the nodes of t_{i+1},
 * zn[(r*n_steps + i)*m + k], and eta[((r*n_steps + i)*m + k)*m + j]. */
int orc_cdcq_tables(int model, const double* P, const double* Pm, int d_in, int width, int n_hidden,
                    int act, const double* theta, int p, const double* Y0, int n_sets, double T,
                    int n_steps, int m, const int64_t* sets, int64_t n_sel, double* zn, double* eta) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    orc_net N = {model, d_in, width, n_hidden, act, m, p, P, xn};
    orc_net NM = {model, d_in, width, n_hidden, act, m, p, Pm ? Pm : P, xn};
    double dt = T / (double)n_steps;
    int64_t n_rows = sets ? n_sel : n_sets;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t s = sets ? sets[r] : r;
        const double* th = theta + s * p;
        for (int i = 0; i < n_steps; ++i) {
            double z[ORC_MAX_W], znext[ORC_MAX_W], C[ORC_MAX_W * 8];
            if (i == 0) {
                for (int k = 0; k < m; ++k) z[k] = Y0[s];
            } else {
                collocation(&NM, Y0[s], i * dt, th, z, NULL);
            }
            collocation(&NM, Y0[s], (i + 1) * dt, th, znext, NULL);
            for (int k = 0; k < m; ++k) collocation(&N, z[k], dt, th, C + k * m, NULL);
            double* zo = zn + (r * n_steps + i) * m;
            double* eo = eta + (r * n_steps + i) * m * m;
            for (int k = 0; k < m; ++k) zo[k] = znext[k];
            for (int k = 0; k < m * m; ++k) eo[k] = orc_cdcq_Ginv(m, xn, znext, C[k]);
        }
    }
    return 0;
}

/* Y_T (and optionally the grid Y_i = G_i(xi_i)) of selected flat paths of the
 * quantile-coordinate 7L-CDC chain; arguments as orc_cdc_paths. */
int orc_cdcq_paths(int model, const double* P, const double* Pm, int d_in, int width, int n_hidden,
                   int act, const double* theta, int p, const double* Y0, const int64_t* offsets,
                   int n_sets, double T, int n_steps, int m, uint64_t seed, const int64_t* idx,
                   int64_t n_idx, double* out_YT, double* out_grid, int n_threads) {
    double xn[64], wn[64];
    if (orc_gauss_hermite(m, xn, wn) != 0) return 1;
    int64_t* sets = (int64_t*)malloc(sizeof(int64_t) * (n_idx > 0 ? n_idx : 1));
    if (!sets) return 1;
    for (int64_t k = 0; k < n_idx; ++k) sets[k] = owning_set(offsets, n_sets, idx ? idx[k] : k);
    qsort(sets, (size_t)n_idx, sizeof(int64_t), cmp_i64);
    int64_t n_sel = 0;
    for (int64_t k = 0; k < n_idx; ++k)
        if (n_sel == 0 || sets[k] != sets[n_sel - 1]) sets[n_sel++] = sets[k];
    size_t nt = (size_t)(n_sel > 0 ? n_sel : 1) * n_steps;
    double* zn = (double*)malloc(sizeof(double) * nt * m);
    double* eta = (double*)malloc(sizeof(double) * nt * m * m);
    if (!zn || !eta) { free(sets); free(zn); free(eta); return 1; }
    set_threads(n_threads);
    int rc = orc_cdcq_tables(model, P, Pm, d_in, width, n_hidden, act, theta, p, Y0, n_sets, T,
                             n_steps, m, sets, n_sel, zn, eta);
    if (rc) { free(sets); free(zn); free(eta); return rc; }
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t g = idx ? idx[k] : k;
        int s = owning_set(offsets, n_sets, g);
        uint32_t q = (uint32_t)(g - offsets[s]);
        int64_t key = s, *hit = (int64_t*)bsearch(&key, sets, (size_t)n_sel, sizeof(int64_t), cmp_i64);
        int64_t row = hit - sets;
        double* grid = out_grid ? out_grid + k * (int64_t)(n_steps + 1) : NULL;
        if (grid) grid[0] = Y0[s];
        double xi = 0.0, Y = Y0[s];
        for (int i = 0; i < n_steps; ++i) {
            size_t r = (size_t)row * n_steps + i;
            double X = orc_normal(seed, ORC_TAG_7L, (uint32_t)s, q, (uint32_t)i);
            xi = orc_cdcq_F(m, xn, eta + r * m * m, xi, X);
            Y = orc_cdcq_G(m, xn, zn + r * m, xi);
            if (grid) grid[i + 1] = Y;
        }
        out_YT[k] = Y;
    }
    free(sets);
    free(zn);
    free(eta);
    return 0;
}
