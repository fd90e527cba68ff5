// sl_simt.cu -- FP32 CUDA-core form of the 7L online sampler (Algorithm I,
// steps 2-8) and the deterministic FP64 per-set moments.
//
// A thread owns its paths for the whole time loop: two per thread for the network
// (Eq. 6.4, FP32 FMAs against weights staged once per CTA in shared memory, every
// lane of a warp reading the same weight: a broadcast), one per thread for the
// exact-collocation models (GBM lognormal map, OU map of Eq. 6.6), which replace
// the network by their closed form.  The state, the normals and the collocation
// vector stay in registers.
#include <math.h>

#include "sl_internal.cuh"
#include "sl_simt_net.cuh"

namespace sl {
namespace {

using namespace simt;

// The exact-collocation models, MODEL: SL_MODEL_GBM_EXACT / SL_MODEL_OU_EXACT.
template <int MODEL>
__global__ void __launch_bounds__(256) simt_7l_kernel(const SimArgs a) {
    const int m = a.m;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < a.total;
         g += stride) {
        int s = 0;
        const int64_t gg = a.first + g;   // index in the whole batch (g: in this call)
        int64_t q = gg;
        if (a.offsets) {
            s = owning_set(a.offsets, a.n_sets, gg);
            q = gg - __ldg(a.offsets + s);
            if (!path_in_set(a.offsets, s, gg, a.status)) continue;
        }
        const float* th = a.theta + static_cast<int64_t>(s) * a.p;
        float Y = a.Y0 ? __ldg(a.Y0 + s) : a.y0_scalar;
        if (a.out_grid) a.out_grid[g] = Y;

        // Per-path constants of the exact maps (theta is fixed along the path).
        float ex[SL_MAX_M];   // GBM: y_j = Y * ex[j];  OU: y_j = c1 * Y + ex[j]
        float c1 = 0.0f;
        if (MODEL == SL_MODEL_GBM_EXACT) {
            const float mu = __ldg(th), sg = __ldg(th + 1);
            const float am = (mu - 0.5f * sg * sg) * a.dt, bm = sg * sqrtf(a.dt);
#pragma unroll
            for (int j = 0; j < SL_MAX_M; ++j) ex[j] = (j < m) ? expf(fmaf(bm, a.gh.x[j], am)) : 0.0f;
        } else {
            const float yb = __ldg(th), sg = __ldg(th + 1), lam = __ldg(th + 2);
            c1 = expf(-lam * a.dt);
            const float sd = sg * sqrtf(-expm1f(-2.0f * lam * a.dt) / (2.0f * lam));
            const float c0 = yb * (-expm1f(-lam * a.dt));
#pragma unroll
            for (int j = 0; j < SL_MAX_M; ++j) ex[j] = fmaf(sd, a.gh.x[j], c0);
        }

        float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = 0; i < a.n_steps; ++i) {
            if ((i & 3) == 0)
                z4 = normal4(a.seed, 0u, static_cast<uint32_t>(s), static_cast<uint32_t>(q),
                             static_cast<uint32_t>(i >> 2));
            const float X = pick4(z4, i & 3);
            float y[SL_MAX_M];
            if (MODEL == SL_MODEL_GBM_EXACT) {
#pragma unroll
                for (int j = 0; j < SL_MAX_M; ++j) y[j] = Y * ex[j];
            } else {
#pragma unroll
                for (int j = 0; j < SL_MAX_M; ++j) y[j] = fmaf(c1, Y, ex[j]);
            }
            Y = lagrange_eval_m(y, X, a.gh, m);
            if (a.out_grid) a.out_grid[static_cast<int64_t>(i + 1) * a.total + g] = Y;
        }
        if (a.out_YT) a.out_YT[g] = Y;
        if (!isfinite(Y)) raise_status(a.status, SL_DEV_NONFINITE);
    }
}

// The network form: two neighbouring paths per thread, every weight load feeding one packed
// FP32x2 FMA for both (mlp_forward_x2: per path the arithmetic of mlp_forward, so the same
// results as one path per thread, 1.47x faster on the 16 x 1e6 x 16 workload).  The parameters
// (42 KB) and each thread's two activation columns sit in shared memory.
constexpr int kMlpThreads = 128;
template <int ACT>
__global__ void __launch_bounds__(kMlpThreads) simt_7l_mlp_kernel(const SimArgs a) {
    constexpr int NP = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemNet& net = *reinterpret_cast<SmemNet*>(smem_raw);
    float* act = reinterpret_cast<float*>(smem_raw + sizeof(SmemNet)) + threadIdx.x;
    const int m = a.m;
    stage_net(net, a.params, a.d_in, m);
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * NP;
    for (int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * NP; g0 < a.total;
         g0 += stride) {
        int s[NP];
        int64_t q[NP], g[NP];
        bool live[NP];
        float Y[NP], f[NP][DS];
        float4 z4[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            live[p] = g0 + p < a.total;           // a path past the end runs and is not stored
            g[p] = live[p] ? g0 + p : g0;
            const int64_t gg = a.first + g[p];    // index in the whole batch (g: in this call)
            s[p] = 0;
            q[p] = gg;
            if (a.offsets) {
                s[p] = owning_set(a.offsets, a.n_sets, gg);
                q[p] = gg - __ldg(a.offsets + s[p]);
                if (live[p]) live[p] = path_in_set(a.offsets, s[p], gg, a.status);
            }
            const float* th = a.theta + static_cast<int64_t>(s[p]) * a.p;
            Y[p] = a.Y0 ? __ldg(a.Y0 + s[p]) : a.y0_scalar;
            if (a.out_grid && live[p]) a.out_grid[g[p]] = Y[p];
#pragma unroll
            for (int k = 0; k < DS; ++k) f[p][k] = 0.0f;
            f[p][1] = a.dt;
            for (int k = 0; k < a.p && k < DS - 2; ++k) f[p][2 + k] = __ldg(th + k);
            z4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int i = 0; i < a.n_steps; ++i) {
            float X[NP], y[NP][SL_MAX_M];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                if ((i & 3) == 0)
                    z4[p] = normal4(a.seed, 0u, static_cast<uint32_t>(s[p]), static_cast<uint32_t>(q[p]),
                                    static_cast<uint32_t>(i >> 2));
                X[p] = pick4(z4[p], i & 3);
                f[p][0] = Y[p];
            }
            mlp_forward_x2<ACT>(net, act, blockDim.x, f, y);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                Y[p] = lagrange_eval_m(y[p], X[p], a.gh, m);
                if (a.out_grid && live[p]) a.out_grid[static_cast<int64_t>(i + 1) * a.total + g[p]] = Y[p];
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (!live[p]) continue;
            if (a.out_YT) a.out_YT[g[p]] = Y[p];
            if (!isfinite(Y[p])) raise_status(a.status, SL_DEV_NONFINITE);
        }
    }
}

template <int ACT>
int launch_mlp(const SimArgs& a, cudaStream_t st) {
    auto kern = simt_7l_mlp_kernel<ACT>;
    const size_t smem = sizeof(SmemNet) + static_cast<size_t>(W) * 2 * kMlpThreads * sizeof(float);
    int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)),
                        "simt_7l_mlp attribute");
    if (rc) return rc;
    int per_sm = 0;
    rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMlpThreads, smem),
                    "simt_7l_mlp occupancy");
    if (rc) return rc;
    const int64_t per_block = static_cast<int64_t>(kMlpThreads) * 2;
    const int64_t need = (a.total + per_block - 1) / per_block;
    int64_t blocks = static_cast<int64_t>(sm_count()) * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), kMlpThreads, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "simt_7l_mlp launch");
}
constexpr int kSimtThreads = 256;

template <int MODEL>
int launch_one(const SimArgs& a, cudaStream_t st) {
    auto kern = simt_7l_kernel<MODEL>;
    int per_sm = 0;
    int rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSimtThreads, 0),
                        "simt_7l occupancy");
    if (rc) return rc;
    const int64_t need = (a.total + kSimtThreads - 1) / kSimtThreads;
    int64_t blocks = static_cast<int64_t>(sm_count()) * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), kSimtThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "simt_7l launch");
}

// ---------------------------------------------------------------------------
// Deterministic per-set moments.  Set s is cut into R equal chunks; CTA (s, r)
// accumulates, in FP64, the count, sum and sum of squares of (Y_T - K_s) over
// its chunk (K_s = the set's first value, a shift that keeps the variance
// free of cancellation), in a fixed thread order and a fixed tree.  A second
// kernel adds the R partials of each set in order.
// ---------------------------------------------------------------------------
constexpr int kMomThreads = 256;

__global__ void __launch_bounds__(kMomThreads)
set_moments_partial(const float* __restrict__ y, const int64_t* __restrict__ off, int R,
                    double* __restrict__ part) {
    const int s = blockIdx.x, r = blockIdx.y;
    const int64_t a = off[s], b = off[s + 1], n = b - a;
    const int64_t lo = a + n * r / R, hi = a + n * (r + 1) / R;
    const double K = n > 0 ? static_cast<double>(y[a]) : 0.0;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t g = lo + threadIdx.x; g < hi; g += kMomThreads) {
        const double d = static_cast<double>(y[g]) - K;
        s1 += d;
        s2 = fma(d, d, s2);
    }
    __shared__ double sh1[kMomThreads], sh2[kMomThreads];
    sh1[threadIdx.x] = s1;
    sh2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = kMomThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
            sh2[threadIdx.x] += sh2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = part + (static_cast<int64_t>(s) * R + r) * 2;
        o[0] = sh1[0];
        o[1] = sh2[0];
    }
}

__global__ void set_moments_final(const float* __restrict__ y, const int64_t* __restrict__ off,
                                  int n_sets, int R, const double* __restrict__ part,
                                  double* __restrict__ mean, double* __restrict__ var,
                                  int mean_stride, const double* __restrict__ scale) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sets) return;
    const int64_t a = off[s], n = off[s + 1] - a;
    double s1 = 0.0, s2 = 0.0;
    for (int r = 0; r < R; ++r) {
        s1 += part[(static_cast<int64_t>(s) * R + r) * 2];
        s2 += part[(static_cast<int64_t>(s) * R + r) * 2 + 1];
    }
    const double K = n > 0 ? static_cast<double>(y[a]) : 0.0;
    const double nn = static_cast<double>(n);
    if (mean) mean[static_cast<int64_t>(s) * mean_stride] = (n > 0 ? K + s1 / nn : 0.0) * (scale ? scale[s] : 1.0);
    if (var) var[s] = n > 1 ? fmax(s2 - s1 * s1 / nn, 0.0) / (nn - 1.0) : 0.0;
}

// The offsets of a range call's own paths: set s covers the call's outputs
// [clamp(off[s] - first), clamp(off[s+1] - first)) with clamp to [0, n], and count[s] is their number.
__global__ void range_offsets_kernel(const int64_t* __restrict__ off, int n_sets, int64_t first, int64_t n,
                                     int64_t* __restrict__ local, int64_t* __restrict__ count) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > n_sets) return;
    auto clip = [&](int64_t v) { v -= first; return v < 0 ? int64_t(0) : (v > n ? n : v); };
    local[s] = clip(off[s]);
    if (count && s < n_sets) count[s] = clip(off[s + 1]) - clip(off[s]);
}

int moments_chunks(int n_sets) {
    int R = 4096 / (n_sets > 0 ? n_sets : 1);
    return R < 1 ? 1 : (R > 64 ? 64 : R);
}

}  // namespace

int launch_simt_7l(int model, int m, const SimArgs& a, cudaStream_t st) {
    if (m < SL_MIN_M || m > SL_MAX_M) return set_error(SL_ERR_UNSUPPORTED, "m=%d", m);
    if (model == SL_MODEL_GBM_EXACT) return launch_one<SL_MODEL_GBM_EXACT>(a, st);
    if (model == SL_MODEL_OU_EXACT) return launch_one<SL_MODEL_OU_EXACT>(a, st);
    if (a.act == SL_ACT_SOFTPLUS) return launch_mlp<SL_ACT_SOFTPLUS>(a, st);
    return launch_mlp<SL_ACT_RELU>(a, st);
}

int launch_range_offsets(const int64_t* offsets, int n_sets, int64_t first, int64_t n, int64_t* local,
                         int64_t* count, cudaStream_t st) {
    range_offsets_kernel<<<(n_sets + 1 + 255) / 256, 256, 0, st>>>(offsets, n_sets, first, n, local, count);
    return cuda_error(cudaGetLastError(), "range_offsets launch");
}

size_t set_moments_scratch_bytes(int n_sets) {
    return align256(static_cast<size_t>(n_sets) * moments_chunks(n_sets) * 2 * sizeof(double));
}

int launch_set_moments(const float* y, const int64_t* offsets, int n_sets, int64_t total,
                       double* mean, double* var, void* part, cudaStream_t st, int mean_stride,
                       const double* scale) {
    (void)total;
    const int R = moments_chunks(n_sets);
    set_moments_partial<<<dim3(n_sets, R), kMomThreads, 0, st>>>(y, offsets, R,
                                                                   static_cast<double*>(part));
    int rc = cuda_error(cudaGetLastError(), "set_moments_partial launch");
    if (rc) return rc;
    set_moments_final<<<(n_sets + 127) / 128, 128, 0, st>>>(
        y, offsets, n_sets, R, static_cast<const double*>(part), mean, var, mean_stride, scale);
    return cuda_error(cudaGetLastError(), "set_moments_final launch");
}

}  // namespace sl
