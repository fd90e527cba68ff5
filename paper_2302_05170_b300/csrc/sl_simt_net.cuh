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

// acc = (w, w) * (h0, h1) + acc for two paths in one packed FP32x2 FMA (each half rounds like
// fmaf: the same results as two scalar FMAs).
__device__ __forceinline__ void fma2w(float w, float h0, float h1, float& a0, float& a1) {
    asm("{\n.reg .b64 ww, hh, aa;\nmov.b64 ww, {%2, %2};\nmov.b64 hh, {%3, %4};\nmov.b64 aa, {%0, %1};\n"
        "fma.rn.f32x2 aa, ww, hh, aa;\nmov.b64 {%0, %1}, aa;\n}"
        : "+f"(a0), "+f"(a1)
        : "f"(w), "f"(h0), "f"(h1));
}

// Two paths per thread with packed FMAs (the same arithmetic per path as mlp_forward).
template <int ACT>
__device__ __forceinline__ void mlp_forward_x2(const SmemNet& s, float* act, int nt,
                                               const float (&f)[2][DS], float (&y)[2][SL_MAX_M]) {
#pragma unroll 2
    for (int o = 0; o < W; ++o) {
        const float4 a = *reinterpret_cast<const float4*>(s.W1 + o * DS);
        const float4 b = *reinterpret_cast<const float4*>(s.W1 + o * DS + 4);
        float a0 = s.b1[o], a1 = a0;
        fma2w(a.x, f[0][0], f[1][0], a0, a1);
        fma2w(a.y, f[0][1], f[1][1], a0, a1);
        fma2w(a.z, f[0][2], f[1][2], a0, a1);
        fma2w(a.w, f[0][3], f[1][3], a0, a1);
        fma2w(b.x, f[0][4], f[1][4], a0, a1);
        fma2w(b.y, f[0][5], f[1][5], a0, a1);
        fma2w(b.z, f[0][6], f[1][6], a0, a1);
        fma2w(b.w, f[0][7], f[1][7], a0, a1);
        act[o * nt] = activation<ACT>(a0);
        act[(W + o) * nt] = activation<ACT>(a1);
    }
    float h0[W], h1[W];
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            h0[k] = act[k * nt];
            h1[k] = act[(W + k) * nt];
        }
#pragma unroll 2
        for (int o = 0; o < W; ++o) {
            const float* row = s.Wh[l] + o * WS;
            float a0 = s.bh[l][o], a1 = a0;
#pragma unroll
            for (int k = 0; k < 48; k += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(row + k);
                fma2w(w4.x, h0[k], h1[k], a0, a1);
                fma2w(w4.y, h0[k + 1], h1[k + 1], a0, a1);
                fma2w(w4.z, h0[k + 2], h1[k + 2], a0, a1);
                fma2w(w4.w, h0[k + 3], h1[k + 3], a0, a1);
            }
            const float2 w2 = *reinterpret_cast<const float2*>(row + 48);
            fma2w(w2.x, h0[48], h1[48], a0, a1);
            fma2w(w2.y, h0[49], h1[49], a0, a1);
            act[o * nt] = activation<ACT>(a0);
            act[(W + o) * nt] = activation<ACT>(a1);
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        h0[k] = act[k * nt];
        h1[k] = act[(W + k) * nt];
    }
#pragma unroll
    for (int o = 0; o < SL_MAX_M; ++o) {
        const float* row = s.W5 + o * WS;
        float a0 = s.b5[o], a1 = a0;
#pragma unroll
        for (int k = 0; k < 48; k += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(row + k);
            fma2w(w4.x, h0[k], h1[k], a0, a1);
            fma2w(w4.y, h0[k + 1], h1[k + 1], a0, a1);
            fma2w(w4.z, h0[k + 2], h1[k + 2], a0, a1);
            fma2w(w4.w, h0[k + 3], h1[k + 3], a0, a1);
        }
        const float2 w2 = *reinterpret_cast<const float2*>(row + 48);
        fma2w(w2.x, h0[48], h1[48], a0, a1);
        fma2w(w2.y, h0[49], h1[49], a0, a1);
        y[0][o] = a0;
        y[1][o] = a1;
    }
}

}  // namespace simt
}  // namespace sl
