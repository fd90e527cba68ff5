// sl_adjoint.cu -- pathwise sensitivities of E[f(Y_T)] for the 7L sampler,
// f(Y) = max(Y - K, 0), with respect to Y0 and theta: reverse-mode (adjoint)
// differentiation through g_m and the collocation map, with the path state
// checkpointed every k steps and recomputed between checkpoints.
//
// Per path (one thread):
//  1. forward sweep of Algorithm I steps 3-8, writing Y_{ck} to the
//     checkpoint buffer [n_ckpt][total] of the workspace;
//  2. lambda = f'(Y_T) = 1{Y_T > K}; out-of-the-money paths stop here (all
//     their sensitivities are 0);
//  3. for segments c = n_ckpt-1 .. 0: recompute Y_{ck} .. Y_{ck+k-1} from the
//     checkpoint, then for i from the segment's last step down to its first:
//     with c_j = lambda * ell_j(X_{i+1}) (d Y_{i+1} / d y_j is the Lagrange
//     basis value), back-propagate c through the collocation map at Y_i:
//     lambda <- sum_j c_j dy_j/dY_i,  g_theta += sum_j c_j dy_j/dtheta;
//  4. write f(Y_T), lambda (= f'(Y_T) dY_T/dY0) and g_theta per path.
// Per-set FP64 means of these per-path values come from the deterministic
// set-moment reduction.  The network's input gradient is the transposed
// product of the stored hidden activations' derivative masks.
#include <math.h>

#include "sl_internal.cuh"
#include "sl_simt_net.cuh"

namespace sl {
namespace {

using namespace simt;

constexpr int kAdjThreads = 128;
constexpr int kMaxCkptK = 32;

struct AdjArgs {
    SimArgs s;
    float K;
    int k;            // checkpoint interval
    int n_ckpt;       // ceil(n_steps / k)
    float* ckpt;      // [n_ckpt][total]
    float* pv;        // [(2+p)][total]: payoff, dY0, dtheta_0 ..
};

template <int ACT>
__device__ __forceinline__ float act_deriv_from_h(float h) {
    // ReLU: 1{z>0} = 1{h>0};  Softplus: sigmoid(z) = 1 - exp(-h) since h = log(1+e^z).
    if (ACT == SL_ACT_SOFTPLUS) return -expm1f(-h);
    return h > 0.0f ? 1.0f : 0.0f;
}

// Forward pass storing the four hidden outputs in the thread's column of hb
// (h_l[o] at hb[(l*W + o) * nt]); returns the collocation points in y.
template <int ACT>
__device__ __forceinline__ void forward_store(const SmemNet& s, float* hb, int nt, const float (&f)[DS],
                                              float (&y)[SL_MAX_M]) {
#pragma unroll 2
    for (int o = 0; o < W; ++o) {
        const float4 a = *reinterpret_cast<const float4*>(s.W1 + o * DS);
        const float4 b = *reinterpret_cast<const float4*>(s.W1 + o * DS + 4);
        float acc = s.b1[o];
        acc = fmaf(a.x, f[0], acc);
        acc = fmaf(a.y, f[1], acc);
        acc = fmaf(a.z, f[2], acc);
        acc = fmaf(a.w, f[3], acc);
        acc = fmaf(b.x, f[4], acc);
        acc = fmaf(b.y, f[5], acc);
        acc = fmaf(b.z, f[6], acc);
        acc = fmaf(b.w, f[7], acc);
        hb[o * nt] = activation<ACT>(acc);
    }
    float h[W];
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int k = 0; k < W; ++k) h[k] = hb[(l * W + k) * nt];
#pragma unroll 2
        for (int o = 0; o < W; ++o)
            hb[((l + 1) * W + o) * nt] = activation<ACT>(dot50(s.Wh[l] + o * WS, h, s.bh[l][o]));
    }
#pragma unroll
    for (int k = 0; k < W; ++k) h[k] = hb[(3 * W + k) * nt];
#pragma unroll
    for (int o = 0; o < SL_MAX_M; ++o) y[o] = dot50(s.W5 + o * WS, h, s.b5[o]);
}

// Input gradient of sum_j c_j H_j at the point whose activations forward_store
// left in hb (overwritten).  gf[k] = d/df_k.
template <int ACT>
__device__ __forceinline__ void vjp_input(const SmemNet& s, float* hb, int nt, const float (&c)[SL_MAX_M],
                                          float (&gf)[DS]) {
    float dh[W];
#pragma unroll
    for (int k = 0; k < W; ++k) dh[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < SL_MAX_M; ++j) {
        const float* row = s.W5 + j * WS;
#pragma unroll
        for (int k = 0; k < 48; k += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(row + k);
            dh[k] = fmaf(w4.x, c[j], dh[k]);
            dh[k + 1] = fmaf(w4.y, c[j], dh[k + 1]);
            dh[k + 2] = fmaf(w4.z, c[j], dh[k + 2]);
            dh[k + 3] = fmaf(w4.w, c[j], dh[k + 3]);
        }
        dh[48] = fmaf(row[48], c[j], dh[48]);
        dh[49] = fmaf(row[49], c[j], dh[49]);
    }
    // hidden layers L = 4 .. 2: dz_L = dh_L * act'(h_L) (stored over h_L), dh_{L-1} = W_L^T dz_L
    for (int L = 4; L >= 2; --L) {
        float* hl = hb + (L - 1) * W * nt;
#pragma unroll
        for (int o = 0; o < W; ++o) hl[o * nt] = dh[o] * act_deriv_from_h<ACT>(hl[o * nt]);
#pragma unroll
        for (int k = 0; k < W; ++k) dh[k] = 0.0f;
        const float* Wl = s.Wh[L - 2];
#pragma unroll 2
        for (int o = 0; o < W; ++o) {
            const float dz = hl[o * nt];
            const float* row = Wl + o * WS;
#pragma unroll
            for (int k = 0; k < 48; k += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(row + k);
                dh[k] = fmaf(w4.x, dz, dh[k]);
                dh[k + 1] = fmaf(w4.y, dz, dh[k + 1]);
                dh[k + 2] = fmaf(w4.z, dz, dh[k + 2]);
                dh[k + 3] = fmaf(w4.w, dz, dh[k + 3]);
            }
            dh[48] = fmaf(row[48], dz, dh[48]);
            dh[49] = fmaf(row[49], dz, dh[49]);
        }
    }
    // layer 1
#pragma unroll
    for (int k = 0; k < DS; ++k) gf[k] = 0.0f;
#pragma unroll 2
    for (int o = 0; o < W; ++o) {
        const float dz = dh[o] * act_deriv_from_h<ACT>(hb[o * nt]);
        const float4 a = *reinterpret_cast<const float4*>(s.W1 + o * DS);
        const float4 b = *reinterpret_cast<const float4*>(s.W1 + o * DS + 4);
        gf[0] = fmaf(a.x, dz, gf[0]);
        gf[1] = fmaf(a.y, dz, gf[1]);
        gf[2] = fmaf(a.z, dz, gf[2]);
        gf[3] = fmaf(a.w, dz, gf[3]);
        gf[4] = fmaf(b.x, dz, gf[4]);
        gf[5] = fmaf(b.y, dz, gf[5]);
        gf[6] = fmaf(b.z, dz, gf[6]);
        gf[7] = fmaf(b.w, dz, gf[7]);
    }
}

// Per-path constants of the exact maps and their theta-derivatives.
struct ExactMap {
    float e[SL_MAX_M];    // GBM: y_j = Y e_j;  OU: y_j = c1 Y + e_j
    float c1, dt, sdt, mu, sg, yb, lam, s_ou, ds_ou;
};

template <int MODEL>
__device__ __forceinline__ void exact_setup(const SimArgs& a, const float* th, ExactMap& E) {
    E.dt = a.dt;
    E.sdt = sqrtf(a.dt);
    if (MODEL == SL_MODEL_GBM_EXACT) {
        E.mu = __ldg(th);
        E.sg = __ldg(th + 1);
        const float am = (E.mu - 0.5f * E.sg * E.sg) * a.dt, bm = E.sg * E.sdt;
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) E.e[j] = (j < a.m) ? expf(fmaf(bm, a.gh.x[j], am)) : 0.0f;
    } else if (MODEL == SL_MODEL_OU_EXACT) {
        E.yb = __ldg(th);
        E.sg = __ldg(th + 1);
        E.lam = __ldg(th + 2);
        E.c1 = expf(-E.lam * a.dt);
        const float one_m_e2 = -expm1f(-2.0f * E.lam * a.dt);
        const float s2 = one_m_e2 / (2.0f * E.lam);
        E.s_ou = sqrtf(s2);
        const float ds2 = a.dt * expf(-2.0f * E.lam * a.dt) / E.lam - one_m_e2 / (2.0f * E.lam * E.lam);
        E.ds_ou = ds2 / (2.0f * E.s_ou);
        const float c0 = E.yb * (-expm1f(-E.lam * a.dt));
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) E.e[j] = fmaf(E.sg * E.s_ou, a.gh.x[j], c0);
    }
}

// One forward step Y_i -> Y_{i+1} with normal X.
template <int MODEL, int ACT>
__device__ __forceinline__ float step_fwd(const SimArgs& a, const SmemNet& net, float* hb, int nt,
                                          float (&f)[DS], const ExactMap& E, float Y, float X) {
    float y[SL_MAX_M];
    if (MODEL == SL_MODEL_MLP) {
        f[0] = Y;
        forward_store<ACT>(net, hb, nt, f, y);
    } else if (MODEL == SL_MODEL_GBM_EXACT) {
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) y[j] = Y * E.e[j];
    } else {
#pragma unroll
        for (int j = 0; j < SL_MAX_M; ++j) y[j] = fmaf(E.c1, Y, E.e[j]);
    }
    return lagrange_eval_m(y, X, a.gh, a.m);
}

struct NormalCache {
    int blk = -1;
    float4 z;
    __device__ __forceinline__ float get(const SimArgs& a, int s, uint32_t q, int i) {
        if ((i >> 2) != blk) {
            blk = i >> 2;
            z = normal4(a.seed, 0u, static_cast<uint32_t>(s), q, static_cast<uint32_t>(blk));
        }
        return pick4(z, i & 3);
    }
};

template <int MODEL, int ACT>
__global__ void __launch_bounds__(kAdjThreads) adjoint_simt_kernel(const AdjArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemNet& net = *reinterpret_cast<SmemNet*>(smem_raw);
    const int nt = blockDim.x;
    float* hb = reinterpret_cast<float*>(smem_raw + sizeof(SmemNet)) + threadIdx.x;
    const SimArgs& a = A.s;
    if (MODEL == SL_MODEL_MLP) {
        stage_net(net, a.params, a.d_in, a.m);
        __syncthreads();
    }
    const int p = a.p;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * nt;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * nt + threadIdx.x; g < a.total; g += stride) {
        int s = 0;
        int64_t q64 = g;
        if (a.offsets) {
            s = owning_set(a.offsets, a.n_sets, g);
            q64 = g - __ldg(a.offsets + s);
            if (!path_in_set(a.offsets, s, g, a.status)) continue;
        }
        const uint32_t q = static_cast<uint32_t>(q64);
        const float* th = a.theta + static_cast<int64_t>(s) * p;
        float f[DS];
#pragma unroll
        for (int k = 0; k < DS; ++k) f[k] = 0.0f;
        f[1] = a.dt;
        if (MODEL == SL_MODEL_MLP)
            for (int k = 0; k < p && k < DS - 2; ++k) f[2 + k] = __ldg(th + k);
        ExactMap E;
        exact_setup<MODEL>(a, th, E);
        NormalCache nc;
        // 1. forward sweep with checkpoints
        float Y = a.Y0 ? __ldg(a.Y0 + s) : a.y0_scalar;
        for (int i = 0; i < a.n_steps; ++i) {
            if (i % A.k == 0) A.ckpt[static_cast<int64_t>(i / A.k) * a.total + g] = Y;
            Y = step_fwd<MODEL, ACT>(a, net, hb, nt, f, E, Y, nc.get(a, s, q, i));
        }
        if (!isfinite(Y)) raise_status(a.status, SL_DEV_NONFINITE);
        const float payoff = fmaxf(Y - A.K, 0.0f);
        float lam = Y > A.K ? 1.0f : 0.0f;
        float gth[DS - 2];
#pragma unroll
        for (int k = 0; k < DS - 2; ++k) gth[k] = 0.0f;
        // 2-3. reverse sweep over checkpointed segments (in-the-money paths only)
        if (lam != 0.0f) {
            for (int c = A.n_ckpt - 1; c >= 0; --c) {
                const int i0 = c * A.k;
                const int i1 = min(i0 + A.k, a.n_steps);
                float Ys[kMaxCkptK];
                Ys[0] = A.ckpt[static_cast<int64_t>(c) * a.total + g];
                for (int i = i0; i < i1 - 1; ++i)
                    Ys[i - i0 + 1] = step_fwd<MODEL, ACT>(a, net, hb, nt, f, E, Ys[i - i0], nc.get(a, s, q, i));
                for (int i = i1 - 1; i >= i0; --i) {
                    const float Yi = Ys[i - i0];
                    float l[SL_MAX_M];
                    const float X = nc.get(a, s, q, i);
                    {   // Lagrange basis at X (unused nodes: weight 0)
                        float d[SL_MAX_M], pre[SL_MAX_M];
#pragma unroll
                        for (int j = 0; j < SL_MAX_M; ++j) d[j] = (j < a.m) ? X - a.gh.x[j] : 1.0f;
                        pre[0] = 1.0f;
#pragma unroll
                        for (int j = 1; j < SL_MAX_M; ++j) pre[j] = pre[j - 1] * d[j - 1];
                        float suf = 1.0f;
#pragma unroll
                        for (int j = SL_MAX_M - 1; j >= 0; --j) {
                            l[j] = a.gh.bary[j] * (pre[j] * suf) * lam;
                            suf *= d[j];
                        }
                    }
                    if (MODEL == SL_MODEL_MLP) {
                        float y[SL_MAX_M], gf[DS];
                        f[0] = Yi;
                        forward_store<ACT>(net, hb, nt, f, y);
                        vjp_input<ACT>(net, hb, nt, l, gf);
                        lam = gf[0];
#pragma unroll
                        for (int k = 0; k < DS - 2; ++k) gth[k] += gf[2 + k];
                    } else if (MODEL == SL_MODEL_GBM_EXACT) {
                        float se = 0.0f, sex = 0.0f;
#pragma unroll
                        for (int j = 0; j < SL_MAX_M; ++j) {
                            se = fmaf(l[j], E.e[j], se);
                            sex = fmaf(l[j] * E.e[j], a.gh.x[j], sex);
                        }
                        lam = se;
                        gth[0] = fmaf(Yi * E.dt, se, gth[0]);
                        gth[1] = fmaf(Yi, fmaf(-E.sg * E.dt, se, E.sdt * sex), gth[1]);
                    } else {
                        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                        for (int j = 0; j < SL_MAX_M; ++j) {
                            s0 += l[j];
                            s1 = fmaf(l[j], a.gh.x[j], s1);
                        }
                        lam = E.c1 * s0;
                        gth[0] = fmaf(1.0f - E.c1, s0, gth[0]);
                        gth[1] = fmaf(E.s_ou, s1, gth[1]);
                        gth[2] += (E.yb - Yi) * E.dt * E.c1 * s0 + E.sg * E.ds_ou * s1;
                    }
                }
            }
        }
        // 4. per-path outputs
        A.pv[g] = payoff;
        A.pv[a.total + g] = lam;
        for (int k = 0; k < p; ++k) A.pv[static_cast<int64_t>(2 + k) * a.total + g] = gth[k];
        if (!isfinite(lam) || !isfinite(payoff)) raise_status(a.status, SL_DEV_NONFINITE);
    }
}

template <int MODEL, int ACT>
int launch_adj(const AdjArgs& A, cudaStream_t st) {
    auto kern = adjoint_simt_kernel<MODEL, ACT>;
    const size_t smem = (MODEL == SL_MODEL_MLP)
                            ? sizeof(SmemNet) + static_cast<size_t>(4 * W) * kAdjThreads * sizeof(float)
                            : 16;
    int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)), "adjoint attribute");
    if (rc) return rc;
    int per_sm = 0;
    rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, smem),
                    "adjoint occupancy");
    if (rc) return rc;
    const int64_t need = (A.s.total + kAdjThreads - 1) / kAdjThreads;
    int64_t blocks = static_cast<int64_t>(sm_count()) * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), kAdjThreads, smem, st>>>(A);
    return cuda_error(cudaGetLastError(), "adjoint launch");
}

int model_p(int model) { return model == SL_MODEL_GBM_EXACT ? 2 : 3; }

}  // namespace

int launch_tc_adjoint(const SimArgs& s, float K, int k, int n_ckpt, float* ckpt, float* pv, float* yt,
                      uint32_t* list, unsigned* count, cudaStream_t st);

}  // namespace sl

using namespace sl;

extern "C" {

size_t sl_adjoint_workspace_size(int64_t total_paths, int n_sets, int n_steps, int ckpt_k, int p) {
    if (total_paths < 0) total_paths = 0;
    if (ckpt_k < 1) ckpt_k = 1;
    if (n_steps < 1) n_steps = 1;
    if (p < 0) p = 0;
    const int64_t n_ckpt = (n_steps + ckpt_k - 1) / ckpt_k;
    // checkpoints (one spare row: the BF16 form's forward sweep also writes Y_T when k divides
    // n_steps), per-path values, and for the BF16 form Y_T, the in-the-money list and its length
    return kStatusBytes + align256(static_cast<size_t>((n_ckpt + 1) * total_paths) * 4) +
           align256(static_cast<size_t>((2 + p) * total_paths) * 4) +
           2 * align256(static_cast<size_t>(total_paths) * 4) + 256 +
           set_moments_scratch_bytes(n_sets < 1 ? 1 : n_sets);
}

int seven_league_adjoint(int model, const sl_net* net, const float* theta, int p, const float* Y0,
                         const int64_t* path_offsets, int n_sets, int64_t total_paths, float T,
                         int n_steps, int m, uint64_t seed, int payoff, float K, int ckpt_k,
                         double* out_value, double* out_dY0, double* out_dtheta,
                         const double* seed_grad, float* out_paths, void* ws, size_t ws_bytes,
                         void* stream) {
    if (model != SL_MODEL_MLP && model != SL_MODEL_GBM_EXACT && model != SL_MODEL_OU_EXACT)
        return set_error(SL_ERR_ARG, "model=%d", model);
    if (payoff != SL_PAYOFF_CALL) return set_error(SL_ERR_UNSUPPORTED, "payoff=%d", payoff);
    if (m < SL_MIN_M || m > SL_MAX_M) return set_error(SL_ERR_UNSUPPORTED, "m=%d", m);
    if (n_steps < 1) return set_error(SL_ERR_UNSUPPORTED, "n_steps=%d", n_steps);
    if (ckpt_k < 1 || ckpt_k > kMaxCkptK) return set_error(SL_ERR_UNSUPPORTED, "ckpt_k=%d outside [1,%d]", ckpt_k, kMaxCkptK);
    if (!(T > 0.0f) || !isfinite(T) || !isfinite(K)) return set_error(SL_ERR_ARG, "T / K");
    if (n_sets < 1 || n_sets > SL_MAX_SETS || total_paths < 0) return set_error(SL_ERR_ARG, "n_sets / total_paths");
    if (!theta || !Y0 || !path_offsets) return set_error(SL_ERR_ARG, "theta / Y0 / path_offsets == NULL");
    if (model == SL_MODEL_MLP) {
        if (!net || !net->params) return set_error(SL_ERR_ARG, "network required");
        if (net->m != m || net->d_in != p + 2) return set_error(SL_ERR_ARG, "network shape");
        if (net->d_in > SL_MAX_DIN) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d", net->d_in);
        if (net->act != SL_ACT_RELU && net->act != SL_ACT_SOFTPLUS) return set_error(SL_ERR_ARG, "act");
        if (net->prec != SL_PREC_FP32 && net->prec != SL_PREC_BF16) return set_error(SL_ERR_ARG, "prec");
        if (net->prec == SL_PREC_BF16) {
            if (net->d_in > SL_MAX_DIN_TC)
                return set_error(SL_ERR_UNSUPPORTED, "BF16 form: d_in=%d > %d", net->d_in, SL_MAX_DIN_TC);
        }
    } else if (p != model_p(model)) {
        return set_error(SL_ERR_ARG, "model %d needs p=%d", model, model_p(model));
    }
    const size_t need = sl_adjoint_workspace_size(total_paths, n_sets, n_steps, ckpt_k, p);
    if (!ws || ws_bytes < need) return set_error(SL_ERR_WORKSPACE, "workspace %zu < %zu", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* w = static_cast<unsigned char*>(ws);
    const int n_ckpt = (n_steps + ckpt_k - 1) / ckpt_k;
    AdjArgs A{};
    SimArgs& a = A.s;
    if (model == SL_MODEL_MLP) {
        a.params = net->params;
        a.d_in = net->d_in;
        a.act = net->act;
    }
    a.theta = theta;
    a.p = p;
    a.Y0 = Y0;
    a.offsets = path_offsets;
    a.n_sets = n_sets;
    a.total = total_paths;
    a.dt = T / static_cast<float>(n_steps);
    a.n_steps = n_steps;
    a.seed = seed;
    a.m = m;
    a.status = reinterpret_cast<unsigned*>(w);
    int rc = make_gh_const(m, &a.gh);
    if (rc) return rc;
    A.K = K;
    A.k = ckpt_k;
    A.n_ckpt = n_ckpt;
    size_t off = kStatusBytes;
    A.ckpt = reinterpret_cast<float*>(w + off);
    off += align256(static_cast<size_t>(n_ckpt + 1) * total_paths * 4);
    A.pv = out_paths ? out_paths : reinterpret_cast<float*>(w + off);
    off += align256(static_cast<size_t>(2 + p) * total_paths * 4);
    float* yt = reinterpret_cast<float*>(w + off);
    off += align256(static_cast<size_t>(total_paths) * 4);
    uint32_t* list = reinterpret_cast<uint32_t*>(w + off);
    off += align256(static_cast<size_t>(total_paths) * 4);
    unsigned* count = reinterpret_cast<unsigned*>(w + off);
    off += 256;
    void* part = w + off;
    rc = cuda_error(cudaMemsetAsync(a.status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (total_paths > 0) {
        if (model == SL_MODEL_GBM_EXACT) rc = launch_adj<SL_MODEL_GBM_EXACT, 0>(A, st);
        else if (model == SL_MODEL_OU_EXACT) rc = launch_adj<SL_MODEL_OU_EXACT, 0>(A, st);
        else if (net->prec == SL_PREC_BF16)
            rc = launch_tc_adjoint(a, K, ckpt_k, n_ckpt, A.ckpt, A.pv, yt, list, count, st);
        else if (net->act == SL_ACT_SOFTPLUS) rc = launch_adj<SL_MODEL_MLP, SL_ACT_SOFTPLUS>(A, st);
        else rc = launch_adj<SL_MODEL_MLP, SL_ACT_RELU>(A, st);
        if (rc) return rc;
    }
    if (out_value) {
        rc = launch_set_moments(A.pv, path_offsets, n_sets, total_paths, out_value, nullptr, part, st);
        if (rc) return rc;
    }
    if (out_dY0) {
        rc = launch_set_moments(A.pv + total_paths, path_offsets, n_sets, total_paths, out_dY0, nullptr,
                                part, st, 1, seed_grad);
        if (rc) return rc;
    }
    if (out_dtheta) {
        for (int k = 0; k < p; ++k) {
            rc = launch_set_moments(A.pv + static_cast<int64_t>(2 + k) * total_paths, path_offsets, n_sets,
                                    total_paths, out_dtheta + k, nullptr, part, st, p, seed_grad);
            if (rc) return rc;
        }
    }
    return SL_OK;
}

}  // extern "C"
