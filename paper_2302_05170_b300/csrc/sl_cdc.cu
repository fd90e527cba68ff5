// sl_cdc.cu -- the 7L-CDC online sampler: Algorithm I with the per-path network
// of step 3 replaced by a global interpolation (the variant timed beside the 7L
// scheme in Table 6.1).
//
// Reading: at t_i = i dt the marginal collocation points of Y are
// z_k = G_k(Y0, t_i, theta) (the collocation map over the horizon t_i from the
// deterministic start; G is the marginal network or the exact map), the
// conditional points at those nodes are C[k][j] = H_j(z_k, dt, theta), and a path
// at Y_i takes yhat_j = sum_k C[k][j] L_k(Y_i) (Lagrange in Y through the z_k)
// inside the nodes' hull and the line through the two outermost nodes beyond it,
// then Y_{i+1} = g_m(X) through (x_j, yhat_j).  At i = 0 (and whenever the nodes
// coincide) every path sits at z_0 and yhat = C[0].
//
// Two phases.  (1) Tables: for every (set, step) the m + 1 network evaluations,
// in FP32 on CUDA cores (weights staged in shared memory, 8 lanes per
// evaluation), plus the barycentric weights of the z_k in FP64; 768 bytes per
// (set, step), with the continuation lines beyond the hull.  (2) Paths: one thread per path for the whole time loop, the
// state and the normals in registers; the table of the path's (set, step) is
// read through the L1 cache (the lanes of a warp share a set, so a load is one
// broadcast).  Phase 2 has no network and no tensor-core work: per path-step it
// is a Philox normal, two Lagrange bases of m nodes and an m x m contraction,
// all FP32 ALU work.
#include <math.h>

#include <cstring>
#include <mutex>

#include "sl_check.cuh"
#include "sl_fastnormal.cuh"
#include "sl_internal.cuh"
#include "sl_simt_net.cuh"

namespace sl {
namespace {

using namespace simt;

// Table of one (set, step), floats: z[8] | w[8] | C[8][8] | S_lo[8] | S_hi[8] |
// C_lo[8] | C_hi[8] | z_lo, z_hi, pad | D[8] | A[8][8] | B_lo[8] | Sm_lo[8] | B_hi[8] |
// Sm_hi[8].  Below the smallest node z_lo the points are C_lo + (Y - z_lo) S_lo (the
// line through the two smallest nodes), above z_hi likewise with the two largest.
// g_m through points y is the polynomial sum_j y_j b_j Q_j(X), Q_j(X) = prod_{l!=j}
// (X - x_l), b_j the barycentric weights of the Gauss-Hermite points; its monomial
// coefficients sum_j y_j (b_j q_j[a]) are formed once per (set, step) in FP64 (q_j[a]
// the coefficients of Q_j, from the host):
//   A[k][a]: w_k times those of row k of C, so that inside the hull
//            Y_{i+1} = sum_k P_k(Y) sum_a A[k][a] X^a,  P_k(Y) = prod_{l!=k} (Y - z_l);
//   D: those of row 0 (coinciding nodes); B_lo, Sm_lo (B_hi, Sm_hi): those of C_lo and
//      S_lo (C_hi, S_hi), so that beyond the hull Y_{i+1} = B(X) + (Y - z_edge) Sm(X).
// The path kernel evaluates them by Horner's rule in X (X ~ N(0, 1): the coefficients
// of a collocation row decay, and Horner is as accurate as the barycentric form there).
constexpr int kTabFloats = 224;
constexpr int kSlo = 80, kShi = 88, kClo = 96, kChi = 104, kZlo = 112, kD = 120, kA = 128, kBlo = 192,
              kSmlo = 200, kBhi = 208, kSmhi = 216;
constexpr int kPathThreads = 256;

struct CdcArgs {
    const float* params;       // conditional network (FP32) or NULL (exact models)
    const float* mparams;      // marginal network
    int d_in, act, mact;
    const float* theta;
    int p;
    const float* Y0;
    int n_sets;
    int n_steps;
    float dt;
    int m;
    float* tab;                // [n_sets][n_steps][kTabFloats]
    GHConst gh;
    double bq[SL_MAX_M][SL_MAX_M];   // b_j q_j[a]: monomial coefficients of b_j Q_j (FP64, zero past m)
    double xg[SL_MAX_M];             // the Gauss-Hermite points in FP64
    // tb[k][i][l]: Bernstein coefficient i of the interpolant through (x_l, z_l) on node interval
    // k, per unit of z_l (FP64): G_{i+1}'s coefficients are linear in its nodes
    double tb[SL_MAX_M - 1][SL_MAX_M][SL_MAX_M];
};

// Collocation points of the exact models over the horizon h from Y:
// GBM y_j = Y exp((mu - sigma^2/2) h + sigma sqrt(h) x_j); OU (Eq. 6.6) restarted at Y.
template <int MODEL>
__device__ __forceinline__ void exact_map(const float* th, float Y, float h, const GHConst& gh, int m,
                                          float (&y)[SL_MAX_M]) {
    if (MODEL == SL_MODEL_GBM_EXACT) {
        const float mu = th[0], sg = th[1];
        const float am = (mu - 0.5f * sg * sg) * h, bm = sg * sqrtf(h);
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) y[j] = (j < m) ? Y * expf(fmaf(bm, gh.x[j], am)) : 0.0f;
    } else {
        const float yb = th[0], sg = th[1], lam = th[2];
        const float c1 = expf(-lam * h);
        const float sd = sg * sqrtf(-expm1f(-2.0f * lam * h) / (2.0f * lam));
        const float c0 = yb * (-expm1f(-lam * h));
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) y[j] = (j < m) ? fmaf(sd, gh.x[j], fmaf(c1, Y, c0)) : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Phase 1: the tables.  One kernel; a CTA takes kBatch (set, step) entries at a
// time in three rounds: (A) the marginal nodes of each entry, (B) the m conditional
// rows of each entry, (C) weights, continuation lines and the folded copy.  A
// network evaluation is shared by the 8 lanes of a group: lane `sub` computes the
// layer outputs sub, sub + 8, ... (the group's lanes read consecutive weight rows,
// 52 floats apart: conflict-free; the four groups of a warp read the same rows:
// broadcast), so that a small table (one set, a few steps) costs a few microseconds.
// ---------------------------------------------------------------------------
constexpr int kGroup = 8;                         // lanes per network evaluation
constexpr int kTabThreads = 256;
constexpr int kGroups = kTabThreads / kGroup;     // 32
constexpr int kBatch = 4;                         // entries per round (one pass of round B)
constexpr int kBufStride = 72;                    // floats per activation buffer (banks 8 apart)

__device__ __forceinline__ float dot50_smem(const float* __restrict__ row, const float* __restrict__ in, float acc) {
#pragma unroll
    for (int k = 0; k < 48; k += 4) {
        const float4 w4 = *reinterpret_cast<const float4*>(row + k);
        const float4 x4 = *reinterpret_cast<const float4*>(in + k);
        acc = fmaf(w4.x, x4.x, acc);
        acc = fmaf(w4.y, x4.y, acc);
        acc = fmaf(w4.z, x4.z, acc);
        acc = fmaf(w4.w, x4.w, acc);
    }
    acc = fmaf(row[48], in[48], acc);
    return fmaf(row[49], in[49], acc);
}

// One layer of 50 outputs for the 8 lanes of a group: lane `sub` computes outputs
// sub + 8 r, r < 7 (the last only for sub < 2), as seven interleaved dot products over
// the 50 inputs in src, so that the group's latency is one dot product, not seven.
template <int ACT>
__device__ __forceinline__ void group_layer50(const float* __restrict__ Wl, const float* __restrict__ bl,
                                              const float* __restrict__ src, float* __restrict__ dst, int sub) {
    constexpr int R = (W + kGroup - 1) / kGroup;   // 7
    float acc[R];
    // row r starts at Wl + (sub + 8 r) WS; rows past 49 recompute row 49 (not stored)
    const float* row0 = Wl + sub * WS;
    const int last = (W - 1 - sub) * WS;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = bl[min(sub + kGroup * r, W - 1)];
#pragma unroll 4
    for (int k = 0; k < 48; k += 4) {
        const float4 x4 = *reinterpret_cast<const float4*>(src + k);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 w4 = *reinterpret_cast<const float4*>(row0 + min(kGroup * WS * r, last) + k);
            acc[r] = fmaf(w4.x, x4.x, acc[r]);
            acc[r] = fmaf(w4.y, x4.y, acc[r]);
            acc[r] = fmaf(w4.z, x4.z, acc[r]);
            acc[r] = fmaf(w4.w, x4.w, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float* rr = row0 + min(kGroup * WS * r, last);
        acc[r] = fmaf(rr[48], src[48], acc[r]);
        acc[r] = fmaf(rr[49], src[49], acc[r]);
        const int o = sub + kGroup * r;
        if (o < W) dst[o] = activation<ACT>(acc[r]);
    }
}

// One network evaluation by the 8 lanes of the group (mask gm): features in in[0, DS),
// result y_j (j < m) in out[j]; `in` and `tmp` are the group's two buffers.
template <int ACT>
__device__ __forceinline__ void group_mlp(const SmemNet& s, float* in, float* tmp, int sub, unsigned gm, int m,
                                          float* out) {
    for (int o = sub; o < W; o += kGroup) {
        float acc = s.b1[o];
#pragma unroll
        for (int k = 0; k < DS; ++k) acc = fmaf(s.W1[o * DS + k], in[k], acc);
        tmp[o] = activation<ACT>(acc);
    }
    __syncwarp(gm);
    group_layer50<ACT>(s.Wh[0], s.bh[0], tmp, in, sub);
    __syncwarp(gm);
    group_layer50<ACT>(s.Wh[1], s.bh[1], in, tmp, sub);
    __syncwarp(gm);
    group_layer50<ACT>(s.Wh[2], s.bh[2], tmp, in, sub);
    __syncwarp(gm);
    if (sub < m) out[sub] = dot50_smem(s.W5 + sub * WS, in, s.b5[sub]);
    __syncwarp(gm);
}

// Collocation points at (Y, horizon h) for the group: the network (its features written
// to `in` first) or the exact map; y_j for j < m in out[j], zero for m <= j < 8.
template <int MODEL, int ACT>
__device__ __forceinline__ void group_map(const SmemNet& net, float* in, float* tmp, int sub, unsigned gm,
                                          const CdcArgs& a, const float* th, float Y, float h, float* out) {
    const int m = a.m;
    if (MODEL == SL_MODEL_MLP) {
        in[sub] = sub == 0 ? Y : sub == 1 ? h : (sub - 2 < a.p ? th[sub - 2] : 0.0f);
        __syncwarp(gm);
        group_mlp<ACT>(net, in, tmp, sub, gm, m, out);
        if (sub >= m) out[sub] = 0.0f;
    } else {
        float y[SL_MAX_M];
        exact_map<MODEL>(th, Y, h, a.gh, m, y);
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j)
            if (j == sub) v = y[j];
        out[sub] = sub < m ? v : 0.0f;
    }
    __syncwarp(gm);
}

size_t table_smem_bytes(int model) {
    return (model == SL_MODEL_MLP ? 2 * sizeof(SmemNet) : 0) +
           (static_cast<size_t>(kGroups) * 2 * kBufStride + kBatch * 8 + kBatch * 64 + kBatch * 8) * sizeof(float) +
           static_cast<size_t>(kBatch) * (8 + 2) * sizeof(double) + static_cast<size_t>(kBatch) * 4 * sizeof(int);
}

template <int MODEL, int ACT, int MACT>
__global__ void __launch_bounds__(kTabThreads, 2) cdc_table_kernel(const CdcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemNet& cnet = *reinterpret_cast<SmemNet*>(smem_raw);
    SmemNet& mnet = *reinterpret_cast<SmemNet*>(smem_raw + sizeof(SmemNet));
    float* bufs = reinterpret_cast<float*>(smem_raw + (MODEL == SL_MODEL_MLP ? 2 * sizeof(SmemNet) : 0));
    float* zs = bufs + kGroups * 2 * kBufStride;   // [kBatch][8] marginal nodes
    float* Cs = zs + kBatch * 8;                   // [kBatch][8][8] conditional rows
    float* ths = Cs + kBatch * 64;                 // [kBatch][8]: Y0 of the entry's set, then theta
    double* wsh = reinterpret_cast<double*>(ths + kBatch * 8);   // [kBatch][8] node weights (FP64)
    double* dsh = wsh + kBatch * 8;                // [kBatch][2] z_lo2 - z_lo, z_hi2 - z_hi
    int* ish = reinterpret_cast<int*>(dsh + kBatch * 2);         // [kBatch][4] lo, lo2, hi, hi2
    const bool one_net = a.mparams == a.params;     // the conditional network gives the marginals too
    if (MODEL == SL_MODEL_MLP) {
        stage_net(cnet, a.params, a.d_in, a.m);
        if (!one_net) stage_net(mnet, a.mparams, a.d_in, a.m);
        __syncthreads();
    }
    const SmemNet& gnet = one_net ? cnet : mnet;
    const int grp = threadIdx.x / kGroup, sub = threadIdx.x % kGroup;
    const unsigned gm = 0xFFu << (threadIdx.x & 24);
    float* in = bufs + grp * 2 * kBufStride;
    float* tmp = in + kBufStride;
    const int m = a.m;
    const int64_t n = static_cast<int64_t>(a.n_sets) * a.n_steps;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kBatch; base < n;
         base += static_cast<int64_t>(gridDim.x) * kBatch) {
        // the batch's Y0 and theta, one global round trip for all groups
        if (threadIdx.x < kBatch * 8) {
            const int e = threadIdx.x / 8, c = threadIdx.x % 8;
            const int64_t u = base + e;
            float v = 0.0f;
            if (u < n) {
                const int s = static_cast<int>(u / a.n_steps);
                v = c == 0 ? __ldg(a.Y0 + s) : (c - 1 < a.p ? __ldg(a.theta + static_cast<int64_t>(s) * a.p + c - 1) : 0.0f);
            }
            ths[threadIdx.x] = v;
        }
        __syncthreads();
        // (A) marginal nodes: group e < kBatch for entry base + e (warp 0)
        if (grp < kBatch) {
            const int64_t u = base + grp;
            float* z = zs + grp * 8;
            if (u < n) {
                const int i = static_cast<int>(u % a.n_steps);
                const float y0 = ths[grp * 8];
                if (i == 0) z[sub] = sub < m ? y0 : 0.0f;
                else group_map<MODEL, MACT>(gnet, in, tmp, sub, gm, a, ths + grp * 8 + 1, y0, static_cast<float>(i) * a.dt, z);
            } else {
                z[sub] = 0.0f;
            }
        }
        __syncthreads();
        // (B) conditional rows: job grp + 32 r = entry e, row k
#pragma unroll 1
        for (int r = 0; r < kBatch * 8 / kGroups; ++r) {
            const int job = grp + kGroups * r, e = job / 8, k = job % 8;
            const int64_t u = base + e;
            float* crow = Cs + e * 64 + k * 8;
            if (u < n && k < m) {
                group_map<MODEL, ACT>(cnet, in, tmp, sub, gm, a, ths + e * 8 + 1, zs[e * 8 + k], a.dt, crow);
            } else {
                crow[sub] = 0.0f;
            }
        }
        __syncthreads();
        // (C1) thread (e, k): node k of entry e -- its weight, row k of C, column k of the
        // continuation lines
        if (threadIdx.x < kBatch * 8) {
            const int e = threadIdx.x / 8, k = threadIdx.x % 8;
            const int64_t u = base + e;
            if (u < n) {
                const float* z = zs + e * 8;
                const float* C = Cs + e * 64;
                float* t = a.tab + u * kTabFloats;
                bool same = true;
                int lo = 0, hi = 0;
                for (int l = 1; l < m; ++l) {
                    same = same && z[l] == z[0];
                    if (z[l] < z[lo]) lo = l;
                    if (z[l] > z[hi]) hi = l;
                }
                int lo2 = -1, hi2 = -1;
                for (int l = 0; l < m; ++l) {
                    if (l != lo && (lo2 < 0 || z[l] < z[lo2])) lo2 = l;
                    if (l != hi && (hi2 < 0 || z[l] > z[hi2])) hi2 = l;
                }
                double wk = 0.0;
                if (!same && k < m) {
                    double prod = 1.0;
                    for (int l = 0; l < m; ++l)
                        if (l != k) prod *= static_cast<double>(z[k]) - static_cast<double>(z[l]);
                    wk = 1.0 / prod;
                }
                t[k] = z[k];
                t[8 + k] = static_cast<float>(wk);
                wsh[e * 8 + k] = wk;
                for (int j = 0; j < SL_MAX_M; ++j) t[16 + 8 * k + j] = C[k * 8 + j];
                // column k of the lines through the two outermost nodes on each side
                const double dlo = static_cast<double>(z[lo2]) - z[lo], dhi = static_cast<double>(z[hi2]) - z[hi];
                const float clo = C[lo * 8 + k], chi = C[hi * 8 + k];
                t[kClo + k] = clo;
                t[kChi + k] = chi;
                t[kSlo + k] = (k < m && dlo != 0.0) ? static_cast<float>((static_cast<double>(C[lo2 * 8 + k]) - clo) / dlo) : 0.0f;
                t[kShi + k] = (k < m && dhi != 0.0) ? static_cast<float>((static_cast<double>(C[hi2 * 8 + k]) - chi) / dhi) : 0.0f;
                t[kZlo + k] = k == 0 ? z[lo] : k == 1 ? z[hi] : 0.0f;   // z_lo, z_hi, then zero padding
                if (k == 0) {
                    ish[e * 4 + 0] = lo;
                    ish[e * 4 + 1] = lo2;
                    ish[e * 4 + 2] = hi;
                    ish[e * 4 + 3] = hi2;
                    dsh[e * 2 + 0] = dlo;
                    dsh[e * 2 + 1] = dhi;
                }
            }
        }
        __syncthreads();
        // (C2) thread (e, k, a), all 256: coefficient a of row k of A, and for k < 5 coefficient
        // a of the monomial row D (k = 0), B_lo, Sm_lo, B_hi, Sm_hi (k = 1..4); the lines'
        // slopes are linear in the rows: sum_j S_j bq[j][a] = (sum_j (C[b][j] - C[a][j]) bq[j][a]) / (z_b - z_a)
        {
            const int e = threadIdx.x / 64, k = (threadIdx.x / 8) % 8, ai = threadIdx.x % 8;
            const int64_t u = base + e;
            if (e < kBatch && u < n) {
                const float* C = Cs + e * 64;
                float* t = a.tab + u * kTabFloats;
                double acc = 0.0;
                for (int j = 0; j < m; ++j) acc += static_cast<double>(C[k * 8 + j]) * a.bq[j][ai];
                t[kA + 8 * k + ai] = static_cast<float>(wsh[e * 8 + k] * acc);
                if (k < 5) {
                    const int r0 = k == 0 ? 0 : ish[e * 4 + (k <= 2 ? 0 : 2)];   // D: row 0; B/Sm: lo or hi
                    const int r1 = ish[e * 4 + (k <= 2 ? 1 : 3)];                 // lo2 or hi2
                    const double d = dsh[e * 2 + (k <= 2 ? 0 : 1)];
                    double b0 = 0.0, b1 = 0.0;
                    for (int j = 0; j < m; ++j) {
                        b0 += static_cast<double>(C[r0 * 8 + j]) * a.bq[j][ai];
                        b1 += static_cast<double>(C[r1 * 8 + j]) * a.bq[j][ai];
                    }
                    const bool slope = (k == 2 || k == 4);
                    const float v = slope ? (d != 0.0 ? static_cast<float>((b1 - b0) / d) : 0.0f) : static_cast<float>(b0);
                    const int col = k == 0 ? kD : k == 1 ? kBlo : k == 2 ? kSmlo : k == 3 ? kBhi : kSmhi;
                    t[col + ai] = v;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The quantile-coordinate reading.  A path carries xi with Y = G_i(xi), G_i the
// marginal collocation map through the Gauss-Hermite points (continued beyond
// them by the lines through the two outermost nodes).  Per (set, step) the
// table holds, in the same 224-float slot:
//   [0,8) zn, the marginal nodes of t_{i+1}; [8,16) Gm, the monomial coefficients
//   of G_{i+1} inside [x_0, x_{m-1}]; [16] x_0, [17] x_{m-1}, [18] the slope below
//   x_0, [19] above x_{m-1}, [20] zn_0, [21] zn_{m-1}, [22] x_1, [23] x_{m-2};
//   [24,88) eta[k][j] =
//   G_{i+1}^{-1}(C[k][j]); [88,152) B[a][b], the monomial coefficients of the
//   tensor-product interpolant: xi_{i+1} = sum_a xi_i^a sum_b B[a][b] X^b for xi_i in
//   [x_0, x_{m-1}]; [152,184) the monomial rows in X of the node rows R_0, R_1,
//   R_{m-2}, R_{m-1} (R_k(X) = sum_j eta[k][j] L_j(X)): beyond the hull xi_{i+1}
//   follows the line in xi through the two outermost node rows.
// ---------------------------------------------------------------------------
constexpr int kQGm = 8, kQEdge = 16, kQEta = 24, kQB = 88, kQR = 152;

size_t tableq_smem_bytes(int model) {
    return (model == SL_MODEL_MLP ? 2 * sizeof(SmemNet) : 0) +
           (static_cast<size_t>(kGroups) * 2 * kBufStride + kBatch * 8 + kBatch * 8 + kBatch * 64 + kBatch * 8) *
               sizeof(float) +
           static_cast<size_t>(kBatch) * (8 + 64 + 64) * sizeof(double) + static_cast<size_t>(kBatch) * sizeof(int);
}

// Bernstein coefficient i of G_{i+1} on the node interval [x_k, x_{k+1}] (n = m - 1,
// G(x_k + h t) = sum_i bern[i] C(n, i) t^i (1 - t)^(n - i), h = x_{k+1} - x_k): linear in the
// nodes, sum_l zn[l] tb[k][i][l] with tb from the host (FP64).  The end coefficients are G's
// values at the nodes, set to the nodes themselves.
__device__ __forceinline__ double interval_bernstein(const float* zn, const double (&tbk)[SL_MAX_M][SL_MAX_M],
                                                    int m, int k, int i) {
    if (i == 0) return zn[k];
    if (i == m - 1) return zn[k + 1];
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < SL_MAX_M; ++l)
        if (l < m) acc = fma(static_cast<double>(zn[l]), tbk[i][l], acc);
    return acc;
}

// Sign variations of c[0..n], zeros skipped: by the Bernstein form of Descartes' rule an upper
// bound on the roots in the open interval, of the same parity, and exact when it is 0 or 1.
__device__ __forceinline__ int sign_variations(const double (&c)[SL_MAX_M], int n) {
    int v = 0, last = 0;
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i) {
        const int sg = i <= n ? (c[i] > 0.0) - (c[i] < 0.0) : 0;
        if (sg != 0) {
            if (last != 0 && sg != last) ++v;
            last = sg;
        }
    }
    return v;
}

// The Bernstein coefficients of the restriction of c (over [0, 1]) to [t0, t1]: de Casteljau at
// t1 keeps the left part, then at t0 / t1 the right part of that.
__device__ void bernstein_restrict(const double (&c)[SL_MAX_M], int n, double t0, double t1,
                                   double (&out)[SL_MAX_M]) {
    double w[SL_MAX_M], l[SL_MAX_M];
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i) w[i] = c[i];
    l[0] = w[0];
#pragma unroll
    for (int r = 1; r < SL_MAX_M; ++r) {
#pragma unroll
        for (int i = 0; i < SL_MAX_M - r; ++i)
            if (i <= n - r) w[i] = fma(t1, w[i + 1] - w[i], w[i]);
        l[r] = w[0];
    }
    const double s = t1 > 0.0 ? t0 / t1 : 0.0;
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i) w[i] = l[i];
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i)
        if (i == n) out[i] = w[i];
#pragma unroll
    for (int r = 1; r < SL_MAX_M; ++r) {
#pragma unroll
        for (int i = 0; i < SL_MAX_M - r; ++i)
            if (i <= n - r) w[i] = fma(s, w[i + 1] - w[i], w[i]);
#pragma unroll
        for (int i = 0; i < SL_MAX_M; ++i)
            if (i == n - r) out[i] = w[i];
    }
}

// The sub-interval [t0, t1] of [0, 1] that holds the smallest root of c = bern - y (Bernstein
// coefficients over [0, 1], c[0] < 0):
// depth-first over the dyadic intervals, left first, skipping those without a sign variation,
// until one has exactly one (a single root inside) or a root sits at an end of one without
// roots inside (t0 = t1).  Intervals still with two or more variations at depth kMaxDepth
// (roots closer than 2^-kMaxDepth of the node interval, or a touch within rounding) end the
// search there.  The visit count is bounded.  Only maps that wiggle inside a node interval
// come here.
constexpr int kMaxDepth = 40;
__device__ __noinline__ void isolate_first_root(const double* bern, double y, int n, double& t0, double& t1) {
    double c[SL_MAX_M];
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i) c[i] = i <= n ? bern[i] - y : 0.0;
    uint64_t idx = 0;                       // interval idx of depth d: [idx 2^-d, (idx + 1) 2^-d]
    int d = 0;
    double sub[SL_MAX_M];
#pragma unroll 1
    for (int visit = 0; visit < 16 * kMaxDepth; ++visit) {
        const double w = ldexp(1.0, -d);
        const double a = static_cast<double>(idx) * w, b = a + w;
        bernstein_restrict(c, n, a, b, sub);
        if (sub[0] == 0.0) { t0 = t1 = a; return; }
        const int v = sign_variations(sub, n);
        if (v == 1 || (v >= 2 && d == kMaxDepth)) { t0 = a; t1 = b; return; }
        double last = 0.0;
#pragma unroll
        for (int i = 0; i < SL_MAX_M; ++i)
            if (i == n) last = sub[i];
        if (v == 0 && last == 0.0) { t0 = t1 = b; return; }   // no root inside, one at the right end
        if (v >= 2) {                      // descend to the left child
            ++d;
            idx <<= 1;
            continue;
        }
        while (d > 0 && (idx & 1)) {       // no root here: the next interval to the right
            idx >>= 1;
            --d;
        }
        if (d == 0) break;
        ++idx;
    }
    t0 = 0.0;                               // not reached for c[0] < 0 <= c[n]
    t1 = 1.0;
}

// G_{i+1}^{-1}(y) (flag 1: the nodes coincide, 0; flag 2: G does not increase from its
// first to its last node, NaN).  Beyond [zn_0, zn_{m-1}] the lines through the two
// outermost nodes; inside, the smallest root of G = y in the first node interval
// [x_k, x_{k+1}] with zn_k <= y <= zn_{k+1}.  The sign variations of G - y's Bernstein
// coefficients on that interval (bern: FP64, per entry and interval) isolate it: one variation
// means one root in the whole interval; more (G wiggles) start a left-first search for the
// first sub-interval with one.  Inside that bracket, where G - y < 0 left of the root and > 0
// right of it: a scan at 32 equal steps for the first point where G >= y (FP32), Newton in FP32
// in that cell (bisecting whenever a step leaves it, 8 steps), then Newton steps on the FP64
// coefficients (residual and derivative in FP64, the derivative's reciprocal in FP32: each step
// then carries a relative error of ~1e-7 of itself), kept inside the bracket, until a step moves
// the root by less than 2^-22 of its size (at most four).
__device__ double quantile_inverse(const float* zn, const float* g32, const double* g64, const double* bern,
                                   const double* xg, int m, int flag, double y) {
    if (flag == 1) return 0.0;
    if (flag == 2) return __longlong_as_double(0x7ff8000000000000LL);
    const double z0 = zn[0], z1 = zn[1], zl = zn[m - 1], zl1 = zn[m - 2];
    if (y < z0) return xg[0] + (y - z0) * (xg[1] - xg[0]) / (z1 - z0);
    if (y > zl) return xg[m - 1] + (y - zl) * (xg[m - 1] - xg[m - 2]) / (zl - zl1);
    int k = 0;
    while (k < m - 2 && !(static_cast<double>(zn[k]) <= y && y <= static_cast<double>(zn[k + 1]))) ++k;
    if (y == static_cast<double>(zn[k])) return xg[k];
    const int n = m - 1;
    double c[SL_MAX_M];
#pragma unroll
    for (int i = 0; i < SL_MAX_M; ++i) c[i] = i <= n ? bern[k * 8 + i] - y : 0.0;
    double blo = xg[k], bhi = xg[k + 1];
    const int v = sign_variations(c, n);
    if (v == 0) return xg[k + 1];            // G - y < 0 up to x_{k+1}, where it is 0
    if (v >= 2) {
        double t0, t1;
        isolate_first_root(bern + k * 8, y, n, t0, t1);
        const double h = xg[k + 1] - xg[k];
        blo = xg[k] + t0 * h;
        bhi = xg[k] + t1 * h;
        if (t0 == t1) return blo;
    }
    const float yf = static_cast<float>(y);
    auto g32at = [&](float u) {
        float gv = g32[m - 1];
        for (int ai = m - 2; ai >= 0; --ai) gv = fmaf(gv, u, g32[ai]);
        return gv;
    };
    const double h = (bhi - blo) / 32.0;
    int cc = 1;
    while (cc < 32 && g32at(static_cast<float>(blo + cc * h)) < yf) ++cc;
    float lo = static_cast<float>(blo + (cc - 1) * h), hi = static_cast<float>(cc < 32 ? blo + cc * h : bhi);
    float xi = 0.5f * (lo + hi);
    for (int it = 0; it < 8; ++it) {
        float gv = g32[m - 1], gd = 0.0f;
        for (int ai = m - 2; ai >= 0; --ai) {
            gd = fmaf(gd, xi, gv);
            gv = fmaf(gv, xi, g32[ai]);
        }
        const float f = gv - yf;
        if (f < 0.0f) lo = xi; else hi = xi;
        float nx = (gd != 0.0f) ? xi - f / gd : 0.5f * (lo + hi);
        if (!(nx > lo && nx < hi)) nx = 0.5f * (lo + hi);
        xi = nx;
    }
    double x = fmin(fmax(static_cast<double>(xi), blo), bhi);
    for (int it = 0; it < 4; ++it) {
        double gv = g64[m - 1], gd = 0.0;
        for (int ai = m - 2; ai >= 0; --ai) {
            gd = fma(gd, x, gv);
            gv = fma(gv, x, g64[ai]);
        }
        const float gdf = static_cast<float>(gd);
        if (gdf == 0.0f) break;
        const double nx = fmin(fmax(x - (gv - y) * static_cast<double>(__frcp_rn(gdf)), blo), bhi);
        // Newton converges quadratically: after a step of 2^-22 of the root or less, the next
        // would move it by ~|G''/G'| 2^-44 (FP64 is slow here: a warp's FP64 FMA holds the unit
        // for tens of cycles, so the refinement stops as soon as it can)
        const bool done = fabs(nx - x) <= 0x1p-22 * (1.0 + fabs(x));
        x = nx;
        if (done) break;
    }
    return x;
}

template <int MODEL, int ACT, int MACT>
__global__ void __launch_bounds__(kTabThreads, 2) cdcq_table_kernel(const CdcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemNet& cnet = *reinterpret_cast<SmemNet*>(smem_raw);
    SmemNet& mnet = *reinterpret_cast<SmemNet*>(smem_raw + sizeof(SmemNet));
    float* bufs = reinterpret_cast<float*>(smem_raw + (MODEL == SL_MODEL_MLP ? 2 * sizeof(SmemNet) : 0));
    float* zs = bufs + kGroups * 2 * kBufStride;   // [kBatch][8] marginal nodes of t_i
    float* zns = zs + kBatch * 8;                  // [kBatch][8] marginal nodes of t_{i+1}
    float* Cs = zns + kBatch * 8;                  // [kBatch][8][8] conditional rows
    float* ths = Cs + kBatch * 64;                 // [kBatch][8]: Y0 of the entry's set, then theta
    double* g64 = reinterpret_cast<double*>(ths + kBatch * 8);   // [kBatch][8] coefficients of G_{i+1}
    double* e64 = g64 + kBatch * 8;                // [kBatch][8][8] eta
    double* r64 = e64 + kBatch * 64;               // [kBatch][8][8] node rows: sum_j eta[k][j] bq[j][b]
                                                   // (before C3: G's Bernstein coefficients per node interval)
    int* flag = reinterpret_cast<int*>(r64 + kBatch * 64);       // [kBatch]
    const bool one_net = a.mparams == a.params;
    if (MODEL == SL_MODEL_MLP) {
        stage_net(cnet, a.params, a.d_in, a.m);
        if (!one_net) stage_net(mnet, a.mparams, a.d_in, a.m);
        __syncthreads();
    }
    const SmemNet& gnet = one_net ? cnet : mnet;
    const int grp = threadIdx.x / kGroup, sub = threadIdx.x % kGroup;
    const unsigned gm = 0xFFu << (threadIdx.x & 24);
    float* in = bufs + grp * 2 * kBufStride;
    float* tmp = in + kBufStride;
    const int m = a.m;
    const int64_t n = static_cast<int64_t>(a.n_sets) * a.n_steps;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kBatch; base < n;
         base += static_cast<int64_t>(gridDim.x) * kBatch) {
        if (threadIdx.x < kBatch * 8) {
            const int e = threadIdx.x / 8, c = threadIdx.x % 8;
            const int64_t u = base + e;
            float v = 0.0f;
            if (u < n) {
                const int s = static_cast<int>(u / a.n_steps);
                v = c == 0 ? __ldg(a.Y0 + s) : (c - 1 < a.p ? __ldg(a.theta + static_cast<int64_t>(s) * a.p + c - 1) : 0.0f);
            }
            ths[threadIdx.x] = v;
        }
        __syncthreads();
        // (A) groups e < kBatch: the nodes of t_i; groups kBatch + e: the nodes of t_{i+1}
        if (grp < 2 * kBatch) {
            const int e = grp % kBatch;
            const bool next = grp >= kBatch;
            const int64_t u = base + e;
            float* z = (next ? zns : zs) + e * 8;
            if (u < n) {
                const int i = static_cast<int>(u % a.n_steps) + (next ? 1 : 0);
                const float y0 = ths[e * 8];
                if (i == 0) z[sub] = sub < m ? y0 : 0.0f;
                else group_map<MODEL, MACT>(gnet, in, tmp, sub, gm, a, ths + e * 8 + 1, y0, static_cast<float>(i) * a.dt, z);
            } else {
                z[sub] = 0.0f;
            }
        }
        __syncthreads();
        // (B) conditional rows at the nodes of t_i
#pragma unroll 1
        for (int r = 0; r < kBatch * 8 / kGroups; ++r) {
            const int job = grp + kGroups * r, e = job / 8, k = job % 8;
            const int64_t u = base + e;
            float* crow = Cs + e * 64 + k * 8;
            if (u < n && k < m) group_map<MODEL, ACT>(cnet, in, tmp, sub, gm, a, ths + e * 8 + 1, zs[e * 8 + k], a.dt, crow);
            else crow[sub] = 0.0f;
        }
        __syncthreads();
        // (C1) thread (e, a): coefficient a of G_{i+1}, node a of t_{i+1}, the edges
        if (threadIdx.x < kBatch * 8) {
            const int e = threadIdx.x / 8, ai = threadIdx.x % 8;
            const int64_t u = base + e;
            if (u < n) {
                const float* zn = zns + e * 8;
                float* t = a.tab + u * kTabFloats;
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += static_cast<double>(zn[k]) * a.bq[k][ai];
                g64[e * 8 + ai] = acc;
                t[kQGm + ai] = static_cast<float>(acc);
                t[ai] = zn[ai];
                if (ai == 0) {
                    bool same = true;
                    for (int k = 1; k < m; ++k) same = same && zn[k] == zn[0];
                    flag[e] = same ? 1 : (zn[m - 1] > zn[0] ? 0 : 2);
                    const double x0 = a.xg[0], x1 = a.xg[1], xl = a.xg[m - 1], xl1 = a.xg[m - 2];
                    t[kQEdge + 0] = static_cast<float>(x0);
                    t[kQEdge + 1] = static_cast<float>(xl);
                    t[kQEdge + 2] = static_cast<float>((static_cast<double>(zn[1]) - zn[0]) / (x1 - x0));
                    t[kQEdge + 3] = static_cast<float>((static_cast<double>(zn[m - 1]) - zn[m - 2]) / (xl - xl1));
                    t[kQEdge + 4] = zn[0];
                    t[kQEdge + 5] = zn[m - 1];
                    t[kQEdge + 6] = static_cast<float>(x1);
                    t[kQEdge + 7] = static_cast<float>(xl1);
                }
            }
        }
        __syncthreads();
        // (C1b) thread (e, k, i): Bernstein coefficient i of G_{i+1} on node interval k (kept in
        // the space of the node rows, which are formed only after C2)
        if (threadIdx.x < kBatch * 56) {
            const int e = threadIdx.x / 56, k = (threadIdx.x / 8) % 7, ci = threadIdx.x % 8;
            if (base + e < n && flag[e] == 0 && k < m - 1 && ci < m)
                r64[e * 64 + k * 8 + ci] = interval_bernstein(zns + e * 8, a.tb[k], m, k, ci);
        }
        __syncthreads();
        // (C2) thread (e, k, j): eta[k][j] = G_{i+1}^{-1}(C[k][j])
        {
            const int e = threadIdx.x / 64, k = (threadIdx.x / 8) % 8, j = threadIdx.x % 8;
            const int64_t u = base + e;
            if (u < n) {
                double v = 0.0;
                if (k < m && j < m) {
                    float* t = a.tab + u * kTabFloats;
                    v = quantile_inverse(zns + e * 8, t + kQGm, g64 + e * 8, r64 + e * 64, a.xg, m, flag[e],
                                         Cs[e * 64 + k * 8 + j]);
                }
                e64[e * 64 + k * 8 + j] = v;
                a.tab[u * kTabFloats + kQEta + k * 8 + j] = static_cast<float>(v);
            }
        }
        __syncthreads();
        // (C3) thread (e, k, b): the node row R_k[b] = sum_j eta[k][j] bq[j][b] (the monomial
        // coefficients in X of sum_j eta[k][j] L_j(X))
        {
            const int e = threadIdx.x / 64, k = (threadIdx.x / 8) % 8, b = threadIdx.x % 8;
            const int64_t u = base + e;
            if (u < n) {
                double row = 0.0;
                for (int j = 0; j < m; ++j) row = fma(e64[e * 64 + k * 8 + j], a.bq[j][b], row);
                r64[e * 64 + k * 8 + b] = row;
            }
        }
        __syncthreads();
        // (C4) thread (e, a, b): B[a][b] = sum_k bq[k][a] R_k[b]; and the outer node rows
        {
            const int e = threadIdx.x / 64, ai = (threadIdx.x / 8) % 8, b = threadIdx.x % 8;
            const int64_t u = base + e;
            if (u < n) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc = fma(a.bq[k][ai], r64[e * 64 + k * 8 + b], acc);
                float* t = a.tab + u * kTabFloats;
                t[kQB + ai * 8 + b] = static_cast<float>(acc);
                if (ai < 4) {                          // R_0, R_1, R_{m-2}, R_{m-1}
                    const int kr = ai < 2 ? ai : m - 4 + ai;
                    t[kQR + ai * 8 + b] = static_cast<float>(r64[e * 64 + kr * 8 + b]);
                } else if (ai == 4 && b == 0) {
                    for (int z = kQR + 32; z < kTabFloats; ++z) t[z] = 0.0f;
                }
            }
        }
        __syncthreads();
    }
}

// G^{-1} on caller-given marginal nodes: the table kernel's own steps C1, C1b and C2 for one
// node set per CTA (monomial coefficients of G in FP64 and FP32, Bernstein coefficients per
// node interval, then quantile_inverse for each requested y).
struct InvArgs {
    const float* zn;     // [n_maps][m]
    const double* y;     // [n_maps][n_y]
    double* out;         // [n_maps][n_y]
    int n_maps, n_y, m;
    double bq[SL_MAX_M][SL_MAX_M];
    double xg[SL_MAX_M];
    double tb[SL_MAX_M - 1][SL_MAX_M][SL_MAX_M];
};

__global__ void __launch_bounds__(128) cdcq_inverse_kernel(const InvArgs a) {
    __shared__ float zs[8], g32[8];
    __shared__ double g64[8], bern[64];
    __shared__ int flag;
    const int m = a.m;
    for (int map = blockIdx.x; map < a.n_maps; map += gridDim.x) {
        if (threadIdx.x < 8) zs[threadIdx.x] = threadIdx.x < m ? a.zn[static_cast<int64_t>(map) * m + threadIdx.x] : 0.0f;
        __syncthreads();
        if (threadIdx.x < 8) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += static_cast<double>(zs[k]) * a.bq[k][threadIdx.x];
            g64[threadIdx.x] = acc;
            g32[threadIdx.x] = static_cast<float>(acc);
        }
        if (threadIdx.x == 0) {
            bool same = true;
            for (int k = 1; k < m; ++k) same = same && zs[k] == zs[0];
            flag = same ? 1 : (zs[m - 1] > zs[0] ? 0 : 2);
        }
        __syncthreads();
        if (threadIdx.x < 56 && flag == 0) {
            const int k = threadIdx.x / 8, ci = threadIdx.x % 8;
            if (k < m - 1 && ci < m) bern[k * 8 + ci] = interval_bernstein(zs, a.tb[k], m, k, ci);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < a.n_y; j += blockDim.x) {
            const int64_t o = static_cast<int64_t>(map) * a.n_y + j;
            a.out[o] = quantile_inverse(zs, g32, g64, bern, a.xg, m, flag, a.y[o]);
        }
        __syncthreads();
    }
}

// P_k(X) = prod_{l != k} (X - n_l) for k < M (prefix and suffix products).
template <int M>
__device__ __forceinline__ void prod_except(float X, const float (&nd)[8], float (&P)[M]) {
    float d[M], pre[M];
#pragma unroll
    for (int k = 0; k < M; ++k) d[k] = X - nd[k];
    pre[0] = 1.0f;
#pragma unroll
    for (int k = 1; k < M; ++k) pre[k] = pre[k - 1] * d[k - 1];
    float suf = 1.0f;
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        P[k] = pre[k] * suf;
        suf *= d[k];
    }
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// sum_a c[a] X^a for a < M (Horner).
template <int M>
__device__ __forceinline__ float horner(const float (&c)[8], float X) {
    float h = c[M - 1];
#pragma unroll
    for (int a = M - 2; a >= 0; --a) h = fmaf(h, X, c[a]);
    return h;
}

// One step of NP paths of the same (set, step) table t: Y[p] <- g_m(X[p]) through the
// conditional points at Y[p].  The table is loaded once for all NP paths.
template <int M, int NP>
__device__ __forceinline__ void cdc_step(const float* __restrict__ t, float (&Y)[NP], const float (&X)[NP]) {
    const float4 w4 = __ldg(reinterpret_cast<const float4*>(t + 8));
    const float2 edge = __ldg(reinterpret_cast<const float2*>(t + kZlo));
    float row[8];
    if (w4.x == 0.0f) {                      // coinciding nodes: every path at z_0
        load8(t + kD, row);
#pragma unroll
        for (int p = 0; p < NP; ++p) Y[p] = horner<M>(row, X[p]);
        return;
    }
    bool out[NP];
    bool any_out = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        out[p] = Y[p] < edge.x || Y[p] > edge.y;
        any_out = any_out || out[p];
    }
    float zn[8];
    load8(t, zn);
    float P[NP][M], acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        prod_except<M>(Y[p], zn, P[p]);
        acc[p] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        load8(t + kA + 8 * k, row);
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] = fmaf(P[p][k], horner<M>(row, X[p]), acc[p]);
    }
    float ynew[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) ynew[p] = acc[p];
    if (any_out) {                           // beyond the hull: the outer line
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (!out[p]) continue;
            const bool below = Y[p] < edge.x;
            float sm[8];
            load8(t + (below ? kBlo : kBhi), row);
            load8(t + (below ? kSmlo : kSmhi), sm);
            const float dY = Y[p] - (below ? edge.x : edge.y);
            ynew[p] = fmaf(dY, horner<M>(sm, X[p]), horner<M>(row, X[p]));
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) Y[p] = ynew[p];
}

// Quantile coordinate: xi[p] <- sum_a xi^a sum_b B[a][b] X^b (Horner in X for every row,
// then in xi), the table loaded once for all NP paths.
template <int M, int NP>
__device__ __forceinline__ void cdcq_step(const float* __restrict__ t, float (&xi)[NP], const float (&X)[NP]) {
    float row[8], acc[NP];
    load8(t + kQB + 8 * (M - 1), row);
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = horner<M>(row, X[p]);
#pragma unroll
    for (int ai = M - 2; ai >= 0; --ai) {
        load8(t + kQB + 8 * ai, row);
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] = fmaf(acc[p], xi[p], horner<M>(row, X[p]));
    }
    const float2 hull = __ldg(reinterpret_cast<const float2*>(t + kQEdge));   // x_0, x_{m-1}
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (xi[p] < hull.x || xi[p] > hull.y) {    // beyond the hull: the line through the outer rows
            const bool below = xi[p] < hull.x;
            float ra[8], rb[8];
            load8(t + kQR + (below ? 0 : 24), ra);
            load8(t + kQR + (below ? 8 : 16), rb);
            const float va = horner<M>(ra, X[p]), vb = horner<M>(rb, X[p]);
            const float xa = below ? hull.x : hull.y;
            const float xb = below ? __ldg(t + kQEdge + 6) : __ldg(t + kQEdge + 7);   // x_1, x_{m-2}
            acc[p] = fmaf(xi[p] - xa, (vb - va) / (xb - xa), va);
        }
        xi[p] = acc[p];
    }
}

// Y = G_{i+1}(xi) from the table of step i: Horner inside [x_0, x_{m-1}], the lines beyond.
template <int M>
__device__ __forceinline__ float cdcq_value(const float* __restrict__ t, float xi) {
    const float4 e = __ldg(reinterpret_cast<const float4*>(t + kQEdge));       // x_0, x_{m-1}, slopes
    const float2 zz = __ldg(reinterpret_cast<const float2*>(t + kQEdge + 4));  // zn_0, zn_{m-1}
    if (xi < e.x) return fmaf(xi - e.x, e.z, zz.x);
    if (xi > e.y) return fmaf(xi - e.y, e.w, zz.y);
    float gmr[8];
    load8(t + kQGm, gmr);
    return horner<M>(gmr, xi);
}

// The whole time loop of NP paths of one set s (path indices q[p] within the set, flat
// indices g[p]; write[p] false for a padding lane).  SPACE: SL_CDC_SPACE_Y carries Y,
// SL_CDC_SPACE_QUANTILE carries xi (Y = G_i(xi) where it is output).
template <int M, int NP, int SPACE>
__device__ __forceinline__ void cdc_paths(const SimArgs& a, const float* __restrict__ ts, int s,
                                          const int64_t (&q)[NP], const int64_t (&g)[NP], const bool (&write)[NP]) {
    float Y[NP], X[NP];
    float4 z4[NP];
    const float y0 = __ldg(a.Y0 + s);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        Y[p] = SPACE == SL_CDC_SPACE_Y ? y0 : 0.0f;     // quantile coordinate: xi_0 = 0
        if (a.out_grid && write[p]) a.out_grid[g[p]] = y0;
    }
    for (int i = 0; i < a.n_steps; ++i) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if ((i & 3) == 0)
                z4[p] = normal4_fast(a.seed, 0u, static_cast<uint32_t>(s), static_cast<uint32_t>(q[p]),
                                     static_cast<uint32_t>(i >> 2));
            X[p] = pick4(z4[p], i & 3);
        }
        const float* t = ts + static_cast<int64_t>(i) * kTabFloats;
        if (SPACE == SL_CDC_SPACE_Y) cdc_step<M, NP>(t, Y, X);
        else cdcq_step<M, NP>(t, Y, X);
        if (a.out_grid) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
                if (write[p])
                    a.out_grid[static_cast<int64_t>(i + 1) * a.total + g[p]] =
                        SPACE == SL_CDC_SPACE_Y ? Y[p] : cdcq_value<M>(t, Y[p]);
        }
    }
    const float* tl = ts + static_cast<int64_t>(a.n_steps - 1) * kTabFloats;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (!write[p]) continue;
        const float yT = SPACE == SL_CDC_SPACE_Y ? Y[p] : cdcq_value<M>(tl, Y[p]);
        if (a.out_YT) a.out_YT[g[p]] = yT;
        if (!isfinite(yT)) raise_status(a.status, SL_DEV_NONFINITE);
    }
}

// Phase 2: the paths.  Each thread takes kPathsPerThread neighbouring flat paths; when they
// belong to one set (all but the groups that straddle a set boundary) they share the
// table loads of every step.
constexpr int kPathsPerThread = 4;

template <int M, int SPACE>
__global__ void __launch_bounds__(kPathThreads, 3) cdc_path_kernel(const SimArgs a, const float* __restrict__ tab) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * kPathsPerThread;
    for (int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * kPathsPerThread; g0 < a.total;
         g0 += stride) {
        int s[kPathsPerThread];
        int64_t q[kPathsPerThread], g[kPathsPerThread];
        bool write[kPathsPerThread];
        bool same = true;
#pragma unroll
        for (int p = 0; p < kPathsPerThread; ++p) {
            write[p] = g0 + p < a.total;
            g[p] = write[p] ? g0 + p : g0;
            s[p] = a.offsets ? owning_set(a.offsets, a.n_sets, g[p]) : 0;
            q[p] = a.offsets ? g[p] - __ldg(a.offsets + s[p]) : g[p];
            if (write[p]) write[p] = path_in_set(a.offsets, s[p], g[p], a.status);
            same = same && s[p] == s[0];
        }
        if (same) {
            cdc_paths<M, kPathsPerThread, SPACE>(a, tab + static_cast<int64_t>(s[0]) * a.n_steps * kTabFloats, s[0], q, g, write);
        } else {
#pragma unroll
            for (int p = 0; p < kPathsPerThread; ++p) {
                const int64_t q1[1] = {q[p]}, g1[1] = {g[p]};
                const bool w1[1] = {write[p]};
                cdc_paths<M, 1, SPACE>(a, tab + static_cast<int64_t>(s[p]) * a.n_steps * kTabFloats, s[p], q1, g1, w1);
            }
        }
    }
}

// Blocks per SM of kernel k launched with `threads` threads and `smem` dynamic bytes,
// after raising its dynamic shared-memory limit: asked of the runtime once per device
// (a query per call costs microseconds of host time, as much as a small launch's work).
constexpr int kMaxDevices = 64;

template <class K>
int blocks_per_sm(K k, int threads, size_t smem, int (&cache)[kMaxDevices], int* out) {
    int dev = 0;
    int rc = cuda_error(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev >= 0 && dev < kMaxDevices && cache[dev] > 0) {
        *out = cache[dev];
        return SL_OK;
    }
    rc = cuda_error(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
                    "kernel attribute");
    if (rc) return rc;
    int per_sm = 0;
    rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem), "occupancy");
    if (rc) return rc;
    if (per_sm < 1) per_sm = 1;
    if (dev >= 0 && dev < kMaxDevices) cache[dev] = per_sm;
    *out = per_sm;
    return SL_OK;
}

template <int MODEL, int ACT, int MACT, int SPACE>
int launch_table_kernel(const CdcArgs& c, cudaStream_t st) {
    static int cache[kMaxDevices] = {};
    auto k = SPACE == SL_CDC_SPACE_Y ? cdc_table_kernel<MODEL, ACT, MACT> : cdcq_table_kernel<MODEL, ACT, MACT>;
    const size_t smem = SPACE == SL_CDC_SPACE_Y ? table_smem_bytes(MODEL) : tableq_smem_bytes(MODEL);
    int per_sm = 1;
    int rc = blocks_per_sm(k, kTabThreads, smem, cache, &per_sm);
    if (rc) return rc;
    const int64_t need = (static_cast<int64_t>(c.n_sets) * c.n_steps + kBatch - 1) / kBatch;
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k<<<static_cast<unsigned>(blocks), kTabThreads, smem, st>>>(c);
    return cuda_error(cudaGetLastError(), "cdc_table launch");
}

template <int MODEL, int ACT>
int launch_tables(const CdcArgs& c, int mact, int space, cudaStream_t st) {
    // the marginal network may use another activation than the conditional one
    if (space == SL_CDC_SPACE_Y) {
        if (mact == SL_ACT_SOFTPLUS) return launch_table_kernel<MODEL, ACT, SL_ACT_SOFTPLUS, SL_CDC_SPACE_Y>(c, st);
        return launch_table_kernel<MODEL, ACT, SL_ACT_RELU, SL_CDC_SPACE_Y>(c, st);
    }
    if (mact == SL_ACT_SOFTPLUS) return launch_table_kernel<MODEL, ACT, SL_ACT_SOFTPLUS, SL_CDC_SPACE_QUANTILE>(c, st);
    return launch_table_kernel<MODEL, ACT, SL_ACT_RELU, SL_CDC_SPACE_QUANTILE>(c, st);
}

template <int M, int SPACE>
int launch_paths_m(const SimArgs& a, const float* tab, cudaStream_t st) {
    static int cache[kMaxDevices] = {};
    auto kern = cdc_path_kernel<M, SPACE>;
    int per_sm = 1;
    int rc = blocks_per_sm(kern, kPathThreads, 0, cache, &per_sm);
    if (rc) return rc;
    const int64_t per_block = static_cast<int64_t>(kPathThreads) * kPathsPerThread;
    const int64_t need = (a.total + per_block - 1) / per_block;
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), kPathThreads, 0, st>>>(a, tab);
    return cuda_error(cudaGetLastError(), "cdc_path launch");
}

template <int SPACE>
int launch_paths_s(const SimArgs& a, const float* tab, cudaStream_t st) {
    switch (a.m) {
        case 2: return launch_paths_m<2, SPACE>(a, tab, st);
        case 3: return launch_paths_m<3, SPACE>(a, tab, st);
        case 4: return launch_paths_m<4, SPACE>(a, tab, st);
        case 5: return launch_paths_m<5, SPACE>(a, tab, st);
        case 6: return launch_paths_m<6, SPACE>(a, tab, st);
        case 7: return launch_paths_m<7, SPACE>(a, tab, st);
        default: return launch_paths_m<8, SPACE>(a, tab, st);
    }
}

int launch_paths(const SimArgs& a, const float* tab, int space, cudaStream_t st) {
    return space == SL_CDC_SPACE_Y ? launch_paths_s<SL_CDC_SPACE_Y>(a, tab, st)
                                   : launch_paths_s<SL_CDC_SPACE_QUANTILE>(a, tab, st);
}

// bq[j][a]: the monomial coefficients of b_j Q_j(X) = b_j prod_{l!=j} (X - x_l) (FP64,
// from the FP64 Gauss-Hermite points; zero for j or a >= m); xg: those points.
int gh_monomials(int m, double (&bq)[SL_MAX_M][SL_MAX_M], double (&xg)[SL_MAX_M]) {
    double x[SL_MAX_M], w[SL_MAX_M], b[SL_MAX_M];
    const int rc = gauss_hermite_fp64(m, x, w, b);
    if (rc) return rc;
    for (int j = 0; j < SL_MAX_M; ++j) xg[j] = j < m ? x[j] : 0.0;
    for (int j = 0; j < SL_MAX_M; ++j)
        for (int ai = 0; ai < SL_MAX_M; ++ai) bq[j][ai] = 0.0;
    for (int j = 0; j < m; ++j) {
        double c[SL_MAX_M] = {1.0};          // coefficients, lowest degree first
        int deg = 0;
        for (int l = 0; l < m; ++l) {
            if (l == j) continue;
            for (int ai = deg + 1; ai >= 1; --ai) c[ai] = c[ai - 1] - x[l] * c[ai];   // times (X - x_l)
            c[0] = -x[l] * c[0];
            ++deg;
        }
        for (int ai = 0; ai < m; ++ai) bq[j][ai] = b[j] * c[ai];
    }
    return SL_OK;
}

// tb[k][i][l]: Bernstein coefficient i, on node interval k ([x_k, x_{k+1}] mapped to [0, 1]), of
// the Lagrange basis polynomial L_l through the FP64 Gauss-Hermite points (zero past m): the
// monomial coefficients of L_l (bq[l][a] / b_l times b_l, i.e. bq[l]), a Taylor shift to x_k,
// the powers of h = x_{k+1} - x_k, then bern_i = sum_{j <= i} C(i, j) / C(n, j) q_j.
void interval_tables(int m, const double (&bq)[SL_MAX_M][SL_MAX_M], const double (&xg)[SL_MAX_M],
                     double (&tb)[SL_MAX_M - 1][SL_MAX_M][SL_MAX_M]) {
    const int n = m - 1;
    double binom[SL_MAX_M][SL_MAX_M] = {};
    for (int i = 0; i < SL_MAX_M; ++i) {
        binom[i][0] = 1.0;
        for (int j = 1; j <= i; ++j) binom[i][j] = binom[i - 1][j - 1] + (j < i ? binom[i - 1][j] : 0.0);
    }
    for (int k = 0; k < SL_MAX_M - 1; ++k)
        for (int i = 0; i < SL_MAX_M; ++i)
            for (int l = 0; l < SL_MAX_M; ++l) tb[k][i][l] = 0.0;
    for (int k = 0; k < n; ++k) {
        const double x0 = xg[k], h = xg[k + 1] - xg[k];
        for (int l = 0; l < m; ++l) {
            double q[SL_MAX_M];
            for (int a = 0; a < m; ++a) q[a] = bq[l][a];      // sum_l z_l bq[l][a]: G's coefficients
            for (int i = 0; i < n; ++i)
                for (int j = n - 1; j >= i; --j) q[j] += x0 * q[j + 1];
            double hp = 1.0;
            for (int j = 0; j <= n; ++j) {
                q[j] *= hp;
                hp *= h;
            }
            for (int i = 0; i <= n; ++i) {
                double acc = 0.0;
                for (int j = 0; j <= i; ++j) acc += binom[i][j] / binom[n][j] * q[j];
                tb[k][i][l] = acc;
            }
        }
    }
}

// The per-m host constants of the tables (bq, xg, tb), computed once per m and copied out.
int cdc_host_tables(int m, double (&bq)[SL_MAX_M][SL_MAX_M], double (&xg)[SL_MAX_M],
                    double (&tb)[SL_MAX_M - 1][SL_MAX_M][SL_MAX_M]) {
    struct Entry {
        std::once_flag once;
        int rc = SL_ERR_UNSUPPORTED;
        double bq[SL_MAX_M][SL_MAX_M], xg[SL_MAX_M], tb[SL_MAX_M - 1][SL_MAX_M][SL_MAX_M];
    };
    static Entry cache[SL_MAX_M + 1];
    if (m < SL_MIN_M || m > SL_MAX_M) return set_error(SL_ERR_UNSUPPORTED, "m=%d", m);
    Entry& e = cache[m];
    std::call_once(e.once, [&] {
        e.rc = gh_monomials(m, e.bq, e.xg);
        if (e.rc == SL_OK) interval_tables(m, e.bq, e.xg, e.tb);
    });
    if (e.rc != SL_OK) return set_error(e.rc, "Gauss-Hermite points for m=%d", m);
    memcpy(bq, e.bq, sizeof(bq));
    memcpy(xg, e.xg, sizeof(xg));
    memcpy(tb, e.tb, sizeof(tb));
    return SL_OK;
}

size_t table_bytes(int n_sets, int n_steps) {
    return align256(static_cast<size_t>(n_sets) * static_cast<size_t>(n_steps) * kTabFloats * sizeof(float));
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" {

size_t sl_cdc_workspace_size(int64_t total_paths, int n_sets, int n_steps) {
    if (total_paths < 0) total_paths = 0;
    if (n_sets < 1) n_sets = 1;
    if (n_steps < 1) n_steps = 1;
    return kStatusBytes + table_bytes(n_sets, n_steps) +
           align256(static_cast<size_t>(total_paths) * sizeof(float)) + set_moments_scratch_bytes(n_sets);
}

int seven_league_cdc_simulate_batched(int model, const sl_net* net, const sl_net* marg_net, int space,
                                      const float* theta, int p, const float* Y0,
                                      const int64_t* path_offsets, int n_sets, int64_t total_paths,
                                      float T, int n_steps, int m, uint64_t seed, float* out_YT,
                                      float* out_grid, double* out_mean, double* out_var, void* ws,
                                      size_t ws_bytes, void* stream) {
    int rc = check_common(model, net, theta, p, T, n_steps, m);
    if (rc) return rc;
    if (space != SL_CDC_SPACE_Y && space != SL_CDC_SPACE_QUANTILE) return set_error(SL_ERR_ARG, "space=%d", space);
    if (model == SL_MODEL_MLP && marg_net) {
        rc = check_net(marg_net, m, p);
        if (rc) return rc;
    }
    if (n_sets < 1 || n_sets > SL_MAX_SETS) return set_error(SL_ERR_ARG, "n_sets=%d", n_sets);
    if (total_paths < 0) return set_error(SL_ERR_ARG, "total_paths < 0");
    if (total_paths > (int64_t(1) << 40)) return set_error(SL_ERR_UNSUPPORTED, "total_paths too large");
    if (!Y0 || !path_offsets) return set_error(SL_ERR_ARG, "Y0 / path_offsets == NULL");
    if (!out_YT && !out_grid && !out_mean && !out_var) return set_error(SL_ERR_ARG, "no output requested");
    if (!ws) return set_error(SL_ERR_WORKSPACE, "ws == NULL");
    const bool moments = out_mean || out_var;
    const size_t tbytes = table_bytes(n_sets, n_steps);
    const size_t need = kStatusBytes + tbytes +
                        ((moments && !out_YT) ? align256(static_cast<size_t>(total_paths) * 4) : 0) +
                        (moments ? set_moments_scratch_bytes(n_sets) : 0);
    if (ws_bytes < need) return set_error(SL_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* w = static_cast<unsigned char*>(ws);
    unsigned* status = reinterpret_cast<unsigned*>(w);
    size_t off = kStatusBytes;
    float* tab = reinterpret_cast<float*>(w + off);
    off += tbytes;
    float* yt = out_YT;
    if (moments && !out_YT) {
        yt = reinterpret_cast<float*>(w + off);
        off += align256(static_cast<size_t>(total_paths) * 4);
    }
    void* part = w + off;

    CdcArgs c{};
    const sl_net* mn = (model == SL_MODEL_MLP) ? (marg_net ? marg_net : net) : nullptr;
    if (model == SL_MODEL_MLP) {
        c.params = net->params;
        c.mparams = mn->params;
        c.d_in = net->d_in;
        c.act = net->act;
        c.mact = mn->act;
    }
    c.theta = theta;
    c.p = p;
    c.Y0 = Y0;
    c.n_sets = n_sets;
    c.n_steps = n_steps;
    c.dt = T / static_cast<float>(n_steps);
    c.m = m;
    c.tab = tab;
    rc = make_gh_const(m, &c.gh);
    if (rc) return rc;
    rc = cdc_host_tables(m, c.bq, c.xg, c.tb);
    if (rc) return rc;

    SimArgs a{};
    a.theta = theta;
    a.p = p;
    a.Y0 = Y0;
    a.offsets = path_offsets;
    a.n_sets = n_sets;
    a.total = total_paths;
    a.dt = c.dt;
    a.n_steps = n_steps;
    a.seed = seed;
    a.out_YT = yt;
    a.out_grid = out_grid;
    a.status = status;
    a.m = m;
    a.gh = c.gh;

    rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (model == SL_MODEL_GBM_EXACT) rc = launch_tables<SL_MODEL_GBM_EXACT, 0>(c, 0, space, st);
    else if (model == SL_MODEL_OU_EXACT) rc = launch_tables<SL_MODEL_OU_EXACT, 0>(c, 0, space, st);
    else if (c.act == SL_ACT_SOFTPLUS) rc = launch_tables<SL_MODEL_MLP, SL_ACT_SOFTPLUS>(c, c.mact, space, st);
    else rc = launch_tables<SL_MODEL_MLP, SL_ACT_RELU>(c, c.mact, space, st);
    if (rc) return rc;
    if (total_paths > 0) {
        rc = launch_paths(a, tab, space, st);
        if (rc) return rc;
    }
    if (moments) return launch_set_moments(yt, path_offsets, n_sets, total_paths, out_mean, out_var, part, st);
    return SL_OK;
}

int sl_cdcq_inverse(int m, const float* zn, int n_maps, const double* y, int n_y, double* out, void* stream) {
    if (m < SL_MIN_M || m > SL_MAX_M) return set_error(SL_ERR_UNSUPPORTED, "m=%d outside [%d,%d]", m, SL_MIN_M, SL_MAX_M);
    if (n_maps < 0 || n_y < 0) return set_error(SL_ERR_ARG, "n_maps=%d n_y=%d", n_maps, n_y);
    if (n_maps == 0 || n_y == 0) return SL_OK;
    if (!zn || !y || !out) return set_error(SL_ERR_ARG, "zn / y / out == NULL");
    InvArgs a{};
    a.zn = zn;
    a.y = y;
    a.out = out;
    a.n_maps = n_maps;
    a.n_y = n_y;
    a.m = m;
    int rc = cdc_host_tables(m, a.bq, a.xg, a.tb);
    if (rc) return rc;
    const int grid = n_maps < 65535 ? n_maps : 65535;
    cdcq_inverse_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cuda_error(cudaGetLastError(), "cdcq_inverse launch");
}

}  // extern "C"
