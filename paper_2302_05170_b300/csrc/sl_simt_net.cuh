// sl_simt_net.cuh -- the network H of Eq. (6.4) for FP32 CUDA-core kernels:
// shared-memory staging of the FP32 parameters, the broadcast dot product and
// the forward pass of one feature row per thread.
#pragma once

#include "sl_internal.cuh"

namespace sl {
namespace simt {

constexpr int W = SL_WIDTH;   // 50
constexpr int WS = 52;        // padded row stride (16-byte aligned rows)
constexpr int DS = 8;         // padded input width of layer 1

// Shared-memory image of the network (floats).
struct SmemNet {
    float W1[W * DS];
    float b1[WS];
    float Wh[3][W * WS];
    float bh[3][WS];
    float W5[SL_MAX_M * WS];
    float b5[SL_MAX_M];
};

// dst[i] = src_of(i) for i < n by the whole block, eight independent loads in flight
// per thread (the weights are cold in a small launch: a load at a time would leave the
// staging latency-bound).
template <class F>
__device__ __forceinline__ void stage_loop(float* dst, int n, F src_of) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int base = 0; base < n; base += 8 * nt) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * nt + tid;
            v[u] = i < n ? src_of(i) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * nt + tid;
            if (i < n) dst[i] = v[u];
        }
    }
}

__device__ inline void stage_net(SmemNet& s, const float* __restrict__ P, int d_in, int m) {
    const float* p = P;
    stage_loop(s.W1, W * DS, [&](int i) { const int o = i / DS, k = i % DS; return k < d_in ? __ldg(p + o * d_in + k) : 0.0f; });
    p += W * d_in;
    stage_loop(s.b1, WS, [&](int i) { return i < W ? __ldg(p + i) : 0.0f; });
    p += W;
    for (int l = 0; l < 3; ++l) {
        stage_loop(s.Wh[l], W * WS, [&](int i) { const int o = i / WS, k = i % WS; return k < W ? __ldg(p + o * W + k) : 0.0f; });
        p += W * W;
        stage_loop(s.bh[l], WS, [&](int i) { return i < W ? __ldg(p + i) : 0.0f; });
        p += W;
    }
    stage_loop(s.W5, SL_MAX_M * WS, [&](int i) {
        const int o = i / WS, k = i % WS;
        return (o < m && k < W) ? __ldg(p + o * W + k) : 0.0f;
    });
    p += m * W;
    stage_loop(s.b5, SL_MAX_M, [&](int i) { return i < m ? __ldg(p + i) : 0.0f; });
}

template <int ACT>
__device__ __forceinline__ float activation(float z) {
    if (ACT == SL_ACT_SOFTPLUS) return z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
    return fmaxf(z, 0.0f);
}

// sum_k row[k] * in[k] over the 50 inputs (row: 16-byte aligned, stride WS).
__device__ __forceinline__ float dot50(const float* __restrict__ row, const float (&in)[W], float acc) {
#pragma unroll
    for (int k = 0; k < 48; k += 4) {
        const float4 w4 = *reinterpret_cast<const float4*>(row + k);
        acc = fmaf(w4.x, in[k], acc);
        acc = fmaf(w4.y, in[k + 1], acc);
        acc = fmaf(w4.z, in[k + 2], acc);
        acc = fmaf(w4.w, in[k + 3], acc);
    }
    const float2 w2 = *reinterpret_cast<const float2*>(row + 48);
    acc = fmaf(w2.x, in[48], acc);
    return fmaf(w2.y, in[49], acc);
}

// The network H: features f -> collocation points y (Eq. 6.4).  The inputs of
// a layer live in registers; its outputs go to the thread's column of `act`
// (element k at act[k * nt], conflict-free across a warp) and are reloaded as
// the next layer's inputs.
template <int ACT>
__device__ __forceinline__ void mlp_forward(const SmemNet& s, float* act, int nt,
                                            const float (&f)[DS], float (&y)[SL_MAX_M]) {
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
        act[o * nt] = activation<ACT>(acc);
    }
    float h[W];
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int k = 0; k < W; ++k) h[k] = act[k * nt];
#pragma unroll 2
        for (int o = 0; o < W; ++o) act[o * nt] = activation<ACT>(dot50(s.Wh[l] + o * WS, h, s.bh[l][o]));
    }
#pragma unroll
    for (int k = 0; k < W; ++k) h[k] = act[k * nt];
#pragma unroll
    for (int o = 0; o < SL_MAX_M; ++o) y[o] = dot50(s.W5 + o * WS, h, s.b5[o]);
}

}  // namespace simt
}  // namespace sl
