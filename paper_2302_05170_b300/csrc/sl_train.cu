// sl_train.cu -- GPU training of the collocation network H (Eq. 6.3/6.4):
// FP32 batched forward, mean-squared-error gradient by back-propagation, and
// Adam (the optimiser, batch size 1024 and learning rate 1e-3 named in the
// experiments section), all in the library's kernels.
//
// BF16-aware training (prec = SL_PREC_BF16): the forward and backward passes
// use the weights and biases rounded to BF16 (nearest, ties to even), as the
// tensor-core sampler evaluates them, and the gradient so obtained updates the
// FP32 parameters (a straight-through step), so the BF16 network is the one
// trained.
//
// Gradient: CTA c takes kRows rows of the minibatch, runs the forward pass
// with every layer's pre-activations kept in shared memory, back-propagates
// the loss 1/(B m) sum (H(f) - y)^2, and writes its partial gradient (one
// value per parameter) and partial loss to the workspace.  A second kernel
// adds the partials of each parameter in CTA order (deterministic), and, for
// training, applies the Adam update in the same pass.
#include <cuda_bf16.h>
#include <math.h>

#include "sl_internal.cuh"

namespace sl {
namespace {

constexpr int W = SL_WIDTH;
constexpr int kRows = 8;               // minibatch rows per CTA
constexpr int kThreads = 512;
constexpr int kMaxParams = W * SL_MAX_DIN + W + 3 * (W * W + W) + SL_MAX_M * W + SL_MAX_M;

struct Layer {
    int n_in, n_out;
    int w_off, b_off;   // offsets in the flat parameter array
};

__device__ __forceinline__ void layer_table(int d_in, int m, Layer (&L)[5]) {
    int o = 0;
    for (int l = 0; l < 5; ++l) {
        const int ni = (l == 0) ? d_in : W, no = (l == 4) ? m : W;
        L[l].n_in = ni;
        L[l].n_out = no;
        L[l].w_off = o;
        L[l].b_off = o + ni * no;
        o += ni * no + no;
    }
}

__device__ __forceinline__ float act_f(int act, float z) {
    if (act == SL_ACT_SOFTPLUS) return z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
    return fmaxf(z, 0.0f);
}
__device__ __forceinline__ float act_df(int act, float z) {
    if (act == SL_ACT_SOFTPLUS) return 1.0f / (1.0f + expf(-z));
    return z > 0.0f ? 1.0f : 0.0f;
}

struct GradSmem {
    float P[kMaxParams];
    float h[5][kRows][W + 2];      // h[0] = features, h[l] = output of hidden layer l (l=1..4)
    float z[5][kRows][W + 2];      // pre-activations of layers 1..5 (z[4] = network output)
    float g[2][kRows][W + 2];      // back-propagated gradient (ping-pong)
    float lossp[kThreads / 32];
};

// Partial MSE gradient of CTA blockIdx.x over rows rows[c*kRows ...] of the batch.
__global__ void __launch_bounds__(kThreads)
grad_partial_kernel(const float* __restrict__ P, int d_in, int m, int act, int bf16,
                    const float* __restrict__ feats, const float* __restrict__ labels,
                    const int32_t* __restrict__ rows, int n_rows, float inv_bm,
                    float* __restrict__ part, float* __restrict__ loss_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem& s = *reinterpret_cast<GradSmem*>(smem_raw);
    const int tid = threadIdx.x;
    Layer L[5];
    layer_table(d_in, m, L);
    const int n_params = L[4].b_off + m;
    for (int i = tid; i < n_params; i += kThreads)
        s.P[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(P[i])) : P[i];
    const int r0 = blockIdx.x * kRows;
    const int nr = min(kRows, n_rows - r0);
    for (int i = tid; i < kRows * d_in; i += kThreads) {
        const int r = i / d_in, k = i % d_in;
        float v = 0.0f;
        if (r < nr) {
            const int64_t row = rows ? rows[r0 + r] : (r0 + r);
            v = feats[row * d_in + k];
        }
        s.h[0][r][k] = v;
    }
    __syncthreads();
    // forward
    for (int l = 0; l < 5; ++l) {
        const int ni = L[l].n_in, no = L[l].n_out;
        const float* Wl = s.P + L[l].w_off;
        const float* bl = s.P + L[l].b_off;
        for (int i = tid; i < kRows * no; i += kThreads) {
            const int r = i / no, o = i % no;
            float acc = bl[o];
            for (int k = 0; k < ni; ++k) acc = fmaf(Wl[o * ni + k], s.h[l][r][k], acc);
            s.z[l][r][o] = acc;
            if (l < 4) s.h[l + 1][r][o] = act_f(act, acc);
        }
        __syncthreads();
    }
    // loss and dL/dout
    float lsum = 0.0f;
    for (int i = tid; i < kRows * m; i += kThreads) {
        const int r = i / m, j = i % m;
        float gv = 0.0f;
        if (r < nr) {
            const int64_t row = rows ? rows[r0 + r] : (r0 + r);
            const float e = s.z[4][r][j] - labels[row * m + j];
            lsum = fmaf(e * e, inv_bm, lsum);
            gv = 2.0f * e * inv_bm;
        }
        s.g[0][r][j] = gv;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) s.lossp[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) t += s.lossp[w];
        loss_part[blockIdx.x] = t;
    }
    // backward: g holds dL/dz of layer l (after the activation derivative)
    float* gp = part + static_cast<int64_t>(blockIdx.x) * n_params;
    int cur = 0;
    for (int l = 4; l >= 0; --l) {
        const int ni = L[l].n_in, no = L[l].n_out;
        if (l < 4) {   // dL/dz = dL/dh * act'(z)
            for (int i = tid; i < kRows * no; i += kThreads) {
                const int r = i / no, o = i % no;
                s.g[cur][r][o] *= act_df(act, s.z[l][r][o]);
            }
            __syncthreads();
        }
        // parameter gradients of layer l
        for (int i = tid; i < no * ni; i += kThreads) {
            const int o = i / ni, k = i % ni;
            float acc = 0.0f;
            for (int r = 0; r < kRows; ++r) acc = fmaf(s.g[cur][r][o], s.h[l][r][k], acc);
            gp[L[l].w_off + i] = acc;
        }
        for (int o = tid; o < no; o += kThreads) {
            float acc = 0.0f;
            for (int r = 0; r < kRows; ++r) acc += s.g[cur][r][o];
            gp[L[l].b_off + o] = acc;
        }
        if (l > 0) {   // dL/dh of the layer below
            const float* Wl = s.P + L[l].w_off;
            for (int i = tid; i < kRows * ni; i += kThreads) {
                const int r = i / ni, k = i % ni;
                float acc = 0.0f;
                for (int o = 0; o < no; ++o) acc = fmaf(Wl[o * ni + k], s.g[cur][r][o], acc);
                s.g[cur ^ 1][r][k] = acc;
            }
            __syncthreads();
            cur ^= 1;
        }
    }
}

// Sum the partials of every parameter into grad, and optionally apply Adam; block 0
// also sums the partial losses.  A block takes kRedParams parameters; kRedSplit
// threads per parameter add the partials c = c0, c0 + kRedSplit, .. in order and the
// kRedSplit sub-sums are added in a fixed order (deterministic).
constexpr int kRedParams = 64, kRedSplit = 4, kRedThreads = kRedParams * kRedSplit;

__global__ void __launch_bounds__(kRedThreads)
reduce_adam_kernel(const float* __restrict__ part, const float* __restrict__ loss_part, int n_parts,
                   int n_params, float* __restrict__ grad, float* __restrict__ loss_out,
                   float* __restrict__ params, float* __restrict__ am, float* __restrict__ av, float lr,
                   float b1, float b2, float eps, float c1, float c2) {
    __shared__ float sub[kRedSplit][kRedParams];
    const int pl = threadIdx.x % kRedParams, c0 = threadIdx.x / kRedParams;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kRedParams + pl;
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss_out) {
        float t = 0.0f;
        for (int c = 0; c < n_parts; ++c) t += loss_part[c];
        *loss_out = t;
    }
    float s = 0.0f;
    if (i < n_params)
        for (int c = c0; c < n_parts; c += kRedSplit) s += part[static_cast<int64_t>(c) * n_params + i];
    sub[c0][pl] = s;
    __syncthreads();
    if (c0 != 0 || i >= n_params) return;
    const float gsum = ((sub[0][pl] + sub[1][pl]) + sub[2][pl]) + sub[3][pl];
    if (grad) grad[i] = gsum;
    if (params) {
        const float mi = b1 * am[i] + (1.0f - b1) * gsum;
        const float vi = b2 * av[i] + (1.0f - b2) * gsum * gsum;
        am[i] = mi;
        av[i] = vi;
        params[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

unsigned reduce_blocks(int64_t n_params) { return static_cast<unsigned>((n_params + kRedParams - 1) / kRedParams); }

// FP32 batched forward pass, one thread per row.
__global__ void __launch_bounds__(kThreads)
forward_kernel(const float* __restrict__ P, int d_in, int m, int act, const float* __restrict__ feats,
               int64_t n_rows, float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sP = reinterpret_cast<float*>(smem_raw);
    Layer L[5];
    layer_table(d_in, m, L);
    const int n_params = L[4].b_off + m;
    for (int i = threadIdx.x; i < n_params; i += kThreads) sP[i] = P[i];
    __syncthreads();
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; r < n_rows;
         r += static_cast<int64_t>(gridDim.x) * kThreads) {
        float a[W + 2], b[W + 2];
        for (int k = 0; k < d_in; ++k) a[k] = feats[r * d_in + k];
        for (int l = 0; l < 5; ++l) {
            const float* Wl = sP + L[l].w_off;
            const float* bl = sP + L[l].b_off;
            for (int o = 0; o < L[l].n_out; ++o) {
                float acc = bl[o];
                for (int k = 0; k < L[l].n_in; ++k) acc = fmaf(Wl[o * L[l].n_in + k], a[k], acc);
                b[o] = (l < 4) ? act_f(act, acc) : acc;
            }
            for (int o = 0; o < L[l].n_out; ++o) a[o] = b[o];
        }
        for (int j = 0; j < m; ++j) out[r * m + j] = a[j];
    }
}

int check_net_shape(int d_in, int m, int act) {
    if (d_in < 1 || d_in > SL_MAX_DIN) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d outside [1,%d]", d_in, SL_MAX_DIN);
    if (m < 1 || m > SL_MAX_M) return set_error(SL_ERR_UNSUPPORTED, "m=%d outside [1,%d]", m, SL_MAX_M);
    if (act != SL_ACT_RELU && act != SL_ACT_SOFTPLUS) return set_error(SL_ERR_ARG, "act=%d", act);
    return SL_OK;
}

size_t part_bytes(int d_in, int m, int batch) {
    const int64_t np = sl_n_params(d_in, m);
    const int64_t nc = (batch + kRows - 1) / kRows;
    return align256(static_cast<size_t>(nc * np) * 4) + align256(static_cast<size_t>(nc) * 4);
}

int launch_grad(const float* P, int d_in, int m, int act, int bf16, const float* feats, const float* labels,
                const int32_t* rows, int n_rows, void* ws, cudaStream_t st, float** part_out,
                float** loss_part_out, int* n_parts) {
    const int64_t np = sl_n_params(d_in, m);
    const int nc = (n_rows + kRows - 1) / kRows;
    float* part = static_cast<float*>(ws);
    float* loss_part = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) +
                                                align256(static_cast<size_t>(nc * np) * 4));
    const size_t smem = sizeof(GradSmem);
    int rc = cuda_error(cudaFuncSetAttribute(grad_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)), "grad attribute");
    if (rc) return rc;
    grad_partial_kernel<<<nc, kThreads, smem, st>>>(P, d_in, m, act, bf16, feats, labels, rows, n_rows,
                                                     1.0f / (static_cast<float>(n_rows) * m), part, loss_part);
    rc = cuda_error(cudaGetLastError(), "grad_partial launch");
    *part_out = part;
    *loss_part_out = loss_part;
    *n_parts = nc;
    return rc;
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" {

size_t sl_train_workspace_size(int d_in, int m, int batch) {
    if (batch < 1) batch = 1;
    return part_bytes(d_in, m, batch);
}

int sl_mlp_forward(const sl_net* net, const float* feats, int64_t n_rows, float* out, void* stream) {
    if (!net || !net->params || !feats || !out) return set_error(SL_ERR_ARG, "NULL argument");
    int rc = check_net_shape(net->d_in, net->m, net->act);
    if (rc) return rc;
    if (n_rows < 0) return set_error(SL_ERR_ARG, "n_rows < 0");
    if (n_rows == 0) return SL_OK;
    const size_t smem = static_cast<size_t>(sl_n_params(net->d_in, net->m)) * 4;
    rc = cuda_error(cudaFuncSetAttribute(forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)), "forward attribute");
    if (rc) return rc;
    int64_t blocks = (n_rows + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 4;
    if (blocks > cap) blocks = cap;
    forward_kernel<<<static_cast<unsigned>(blocks), kThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        net->params, net->d_in, net->m, net->act, feats, n_rows, out);
    return cuda_error(cudaGetLastError(), "forward launch");
}

int sl_mse_grad(const sl_net* net, const float* feats, const float* labels, const int32_t* rows,
                int n_rows, float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
    if (!net || !net->params || !feats || !labels || !grad) return set_error(SL_ERR_ARG, "NULL argument");
    int rc = check_net_shape(net->d_in, net->m, net->act);
    if (rc) return rc;
    if (n_rows < 1) return set_error(SL_ERR_ARG, "n_rows < 1");
    if (!ws || ws_bytes < part_bytes(net->d_in, net->m, n_rows))
        return set_error(SL_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *part, *lp;
    int nc;
    if (net->prec != SL_PREC_FP32 && net->prec != SL_PREC_BF16) return set_error(SL_ERR_ARG, "prec=%d", net->prec);
    rc = launch_grad(net->params, net->d_in, net->m, net->act, net->prec == SL_PREC_BF16, feats, labels, rows,
                     n_rows, ws, st, &part, &lp, &nc);
    if (rc) return rc;
    const int np = static_cast<int>(sl_n_params(net->d_in, net->m));
    reduce_adam_kernel<<<reduce_blocks(np), kRedThreads, 0, st>>>(part, lp, nc, np, grad, loss, nullptr, nullptr,
                                                         nullptr, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
    return cuda_error(cudaGetLastError(), "reduce launch");
}

int sl_adam_step(float* params, float* adam_m, float* adam_v, const float* grad, int64_t n, int64_t t,
                 float lr, float b1, float b2, float eps, void* stream) {
    if (!params || !adam_m || !adam_v || !grad) return set_error(SL_ERR_ARG, "NULL argument");
    if (n < 0 || n > (int64_t(1) << 30) || t < 1) return set_error(SL_ERR_ARG, "n or t out of range");
    if (n == 0) return SL_OK;
    const float c1 = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b1), static_cast<double>(t))));
    const float c2 = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b2), static_cast<double>(t))));
    // one "partial" = the gradient itself
    reduce_adam_kernel<<<reduce_blocks(n), kRedThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        grad, grad, 1, static_cast<int>(n), nullptr, nullptr, params, adam_m, adam_v, lr, b1, b2, eps, c1, c2);
    return cuda_error(cudaGetLastError(), "adam launch");
}

int sl_train(float* params, int d_in, int m, int act, int prec, float* adam_m, float* adam_v, int64_t t0,
             const float* feats, const float* labels, const int32_t* batch_rows, int n_batches,
             int batch, float lr, float b1, float b2, float eps, float* losses, void* ws,
             size_t ws_bytes, void* stream) {
    if (!params || !adam_m || !adam_v || !feats || !labels || !batch_rows)
        return set_error(SL_ERR_ARG, "NULL argument");
    int rc = check_net_shape(d_in, m, act);
    if (rc) return rc;
    if (prec != SL_PREC_FP32 && prec != SL_PREC_BF16) return set_error(SL_ERR_ARG, "prec=%d", prec);
    if (n_batches < 0 || batch < 1 || t0 < 0) return set_error(SL_ERR_ARG, "n_batches/batch/t0 out of range");
    if (!ws || ws_bytes < part_bytes(d_in, m, batch)) return set_error(SL_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = static_cast<int>(sl_n_params(d_in, m));
    for (int b = 0; b < n_batches; ++b) {
        float *part, *lp;
        int nc;
        rc = launch_grad(params, d_in, m, act, prec == SL_PREC_BF16, feats, labels,
                         batch_rows + static_cast<int64_t>(b) * batch, batch, ws, st, &part, &lp, &nc);
        if (rc) return rc;
        const double t = static_cast<double>(t0 + b + 1);
        const float c1 = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b1), t)));
        const float c2 = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b2), t)));
        reduce_adam_kernel<<<reduce_blocks(np), kRedThreads, 0, st>>>(part, lp, nc, np, nullptr,
                                                             losses ? losses + b : nullptr, params,
                                                             adam_m, adam_v, lr, b1, b2, eps, c1, c2);
        rc = cuda_error(cudaGetLastError(), "reduce_adam launch");
        if (rc) return rc;
    }
    return SL_OK;
}

}  // extern "C"
