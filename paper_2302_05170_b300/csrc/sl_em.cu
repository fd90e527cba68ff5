// sl_em.cu -- offline stage of the 7L scheme (Algorithm I, step 1):
// fine-step Euler-Maruyama terminal samples (Eq. 6.2) and their empirical
// quantiles at levels Phi(x_j), the collocation labels y_j | (theta, Y_i, dt).
//
// EM: two paths per thread, the whole fine-step loop in registers; the only
// memory traffic is the 4-byte terminal sample; the normals' Box-Muller uses the
// fast logarithm, sine/cosine and square root (normal4_fast).  Select: one CTA per segment,
// exact radix select over the order-preserving 32-bit keys (4 passes of 8
// bits, all requested ranks at once, one histogram per distinct prefix),
// with warp-aggregated shared-memory histogram updates (__match_any_sync) and
// the segment read as float4 where it is 16-byte aligned.
#include <math.h>

#include "sl_internal.cuh"
#include "sl_fastnormal.cuh"

namespace sl {
namespace {

constexpr int kEmThreads = 256;
constexpr int kSelThreads = 512;
constexpr int kMaxK = 16;

// Two paths per thread (q and q + kEmThreads of the CTA's 2 kEmThreads): their independent
// step chains interleave, which keeps the issue slots busier than one chain per thread.
constexpr int kEmPaths = 2;

template <int SDE>
__global__ void __launch_bounds__(kEmThreads)
em_terminal_kernel(const float* __restrict__ theta, const float* __restrict__ Yi,
                   const float* __restrict__ dt, int64_t n_paths, int n_fine, uint64_t seed,
                   float* __restrict__ out) {
    const int r = blockIdx.y;
    const int64_t q0 = static_cast<int64_t>(blockIdx.x) * (kEmPaths * kEmThreads) + threadIdx.x;
    if (q0 >= n_paths) return;
    constexpr int P = (SDE == SL_SDE_GBM) ? 2 : 3;
    const float t0 = __ldg(theta + r * P), t1 = __ldg(theta + r * P + 1);
    const float t2 = (P == 3) ? __ldg(theta + r * P + 2) : 0.0f;
    const float y0 = __ldg(Yi + r);
    const float dtau = __ldg(dt + r) / static_cast<float>(n_fine);
    const float sq = sqrtf(dtau);
    // the drift and diffusion coefficients with the step folded in
    const float t0dt = t0 * dtau, t1sq = t1 * sq, t2dt = t2 * dtau, t2sq = t2 * sq;
    auto step = [&](float& Y, float X) {
        if (SDE == SL_SDE_GBM) {            // (mu, sigma): a = mu Y, b = sigma Y
            Y = fmaf(t1sq * Y, X, fmaf(t0dt, Y, Y));
        } else if (SDE == SL_SDE_OU) {      // (Ybar, sigma, lambda), Eq. 6.5: a = -lambda (Y - Ybar), b = sigma
            Y = fmaf(t1sq, X, fmaf(-t2dt, Y - t0, Y));
        } else {                            // CIR (kappa, ybar, gamma), full truncation
            const float yp = fmaxf(Y, 0.0f);   // a = kappa (ybar - Y+), b = gamma sqrt(Y+)
            Y = fmaf(t2sq * sqrt_approx(yp), X, fmaf(t0dt, t1 - yp, Y));
        }
    };
    float Y[kEmPaths];
    uint32_t qq[kEmPaths];
#pragma unroll
    for (int p = 0; p < kEmPaths; ++p) {
        Y[p] = y0;
        qq[p] = static_cast<uint32_t>(q0 + p * kEmThreads);   // a path past the end runs and is not stored
    }
    // whole blocks of four fine steps (one Philox call per path each), then the remainder
    const int n4 = n_fine >> 2;
    for (int k = 0; k < n4; ++k) {
#pragma unroll
        for (int p = 0; p < kEmPaths; ++p) {
            const float4 z = normal4_fast(seed, 1u, static_cast<uint32_t>(r), qq[p], static_cast<uint32_t>(k));
            step(Y[p], z.x);
            step(Y[p], z.y);
            step(Y[p], z.z);
            step(Y[p], z.w);
        }
    }
    if (n_fine & 3) {
#pragma unroll
        for (int p = 0; p < kEmPaths; ++p) {
            const float4 z = normal4_fast(seed, 1u, static_cast<uint32_t>(r), qq[p], static_cast<uint32_t>(n4));
            for (int u = 0; u < (n_fine & 3); ++u) step(Y[p], pick4(z, u));
        }
    }
#pragma unroll
    for (int p = 0; p < kEmPaths; ++p) {
        const int64_t q = q0 + p * kEmThreads;
        if (q < n_paths) out[static_cast<int64_t>(r) * n_paths + q] = (SDE == SL_SDE_CIR) ? fmaxf(Y[p], 0.0f) : Y[p];
    }
}

struct RankList {
    int64_t r[kMaxK];
    int n;
};

// Order-preserving map float -> uint32 (-0 folded onto +0).
__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t b = __float_as_uint(f + 0.0f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void __launch_bounds__(kSelThreads)
segmented_select_kernel(const float* __restrict__ values, const int64_t* __restrict__ seg_off,
                        int64_t uniform_len, RankList ranks, float* __restrict__ out,
                        unsigned* status) {
    __shared__ uint32_t hist[kMaxK][256];
    __shared__ uint32_t prefix[kMaxK], gprefix[kMaxK];
    __shared__ int64_t rem[kMaxK];
    __shared__ int group_of[kMaxK];
    __shared__ int n_groups;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a = seg_off ? seg_off[s] : static_cast<int64_t>(s) * uniform_len;
    const int64_t n = (seg_off ? seg_off[s + 1] : a + uniform_len) - a;
    const int nk = ranks.n;
    if (n < 0 || n >= (int64_t(1) << 31)) {
        if (tid == 0) raise_status(status, SL_DEV_OFFSETS);
        if (tid < nk) out[static_cast<int64_t>(s) * nk + tid] = __int_as_float(0x7fc00000);
        return;
    }
    if (tid < nk) {
        prefix[tid] = 0u;
        rem[tid] = ranks.r[tid];
    }
    // [a, a + n) = head [a, a4) + body of n4 float4 at 16-byte aligned addresses + tail [e4, a + n)
    const int64_t mis = static_cast<int64_t>((reinterpret_cast<uintptr_t>(values) >> 2) & 3u);
    const int64_t a4 = min(a + ((4 - ((mis + a) & 3)) & 3), a + n);
    const int64_t e4 = max(a4, a + n - ((mis + a + n) & 3));
    const int64_t n4 = (e4 - a4) >> 2;
    const int head = static_cast<int>(a4 - a), tail = static_cast<int>(a + n - e4);
    __syncthreads();
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        const uint32_t hi_mask = pass == 0 ? 0u : ~((1u << (shift + 8)) - 1u);
        if (tid == 0) {   // one histogram per distinct prefix of the still-valid ranks
            int ng = 0;
            for (int j = 0; j < nk; ++j) {
                group_of[j] = -1;
                if (rem[j] >= n) continue;
                int g = 0;
                while (g < ng && gprefix[g] != prefix[j]) ++g;
                if (g == ng) gprefix[ng++] = prefix[j];
                group_of[j] = g;
            }
            n_groups = ng;
        }
        __syncthreads();
        const int ng = n_groups;
        for (int i = tid; i < ng * 256; i += kSelThreads) hist[i >> 8][i & 255] = 0u;
        __syncthreads();
        // One value (warp-converged call): its group g (the rank prefix it extends; none when it
        // matches no prefix), then one shared-memory add per distinct (g, digit) of the warp.
        auto count = [&](float v, bool in) {
            const uint32_t key = float_key(v);
            int g = -1;
            if (in) {
                const uint32_t hk = key & hi_mask;
                for (int j = 0; j < ng; ++j)
                    if (hk == gprefix[j]) {
                        g = j;
                        break;
                    }
            }
            const unsigned act = __ballot_sync(0xffffffffu, g >= 0);
            if (g >= 0) {
                const uint32_t digit = (key >> shift) & 255u;
                const unsigned peers = __match_any_sync(act, (static_cast<uint32_t>(g) << 8) | digit);
                if (lane == __ffs(peers) - 1) atomicAdd(&hist[g][digit], __popc(peers));
            }
        };
        // Aligned body as float4 loads (four values per thread per round); the unaligned head
        // [a, a4) and tail [e4, a + n), at most three values each, by warp 0.
        for (int64_t base = 0; base < n4; base += kSelThreads) {
            const int64_t c = base + tid;
            const bool in = c < n4;
            const float4 v4 = in ? __ldg(reinterpret_cast<const float4*>(values + a4) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            count(v4.x, in);
            count(v4.y, in);
            count(v4.z, in);
            count(v4.w, in);
        }
        if (warp == 0) {
            const int64_t idx = (lane < head) ? a + lane : e4 + (lane - head);
            const bool in = lane < head + tail;
            count(in ? __ldg(values + idx) : 0.0f, in);
        }
        __syncthreads();
        if (warp < nk && group_of[warp] >= 0) {   // warp j resolves rank j's digit
            const uint32_t* h = hist[group_of[warp]];
            uint32_t c[8], local = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                c[i] = h[lane * 8 + i];
                local += c[i];
            }
            uint32_t incl = local;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int64_t rk = rem[warp];
            const unsigned hit = __ballot_sync(0xffffffffu, rk < static_cast<int64_t>(incl));
            const int src = __ffs(hit) - 1;
            if (lane == src) {
                int64_t cum = static_cast<int64_t>(incl - local);
                int bin = 8 * lane;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (rk < cum + c[i]) { bin = 8 * lane + i; break; }
                    cum += c[i];
                }
                rem[warp] = rk - cum;
                prefix[warp] |= static_cast<uint32_t>(bin) << shift;
            }
        }
        __syncthreads();
    }
    if (tid < nk)
        out[static_cast<int64_t>(s) * nk + tid] =
            (ranks.r[tid] < n) ? key_float(prefix[tid]) : __int_as_float(0x7fc00000);
}

int launch_em(int sde, const float* theta, const float* Yi, const float* dt, int n_rows,
              int64_t n_paths, int n_fine, uint64_t seed, float* out, cudaStream_t st) {
    const dim3 grid(static_cast<unsigned>((n_paths + kEmPaths * kEmThreads - 1) / (kEmPaths * kEmThreads)), n_rows);
    if (sde == SL_SDE_GBM)
        em_terminal_kernel<SL_SDE_GBM><<<grid, kEmThreads, 0, st>>>(theta, Yi, dt, n_paths, n_fine, seed, out);
    else if (sde == SL_SDE_OU)
        em_terminal_kernel<SL_SDE_OU><<<grid, kEmThreads, 0, st>>>(theta, Yi, dt, n_paths, n_fine, seed, out);
    else
        em_terminal_kernel<SL_SDE_CIR><<<grid, kEmThreads, 0, st>>>(theta, Yi, dt, n_paths, n_fine, seed, out);
    return cuda_error(cudaGetLastError(), "em_terminal launch");
}

int launch_select(const float* values, const int64_t* seg_off, int64_t uniform_len, int n_seg,
                  const int64_t* ranks, int n_k, float* out, unsigned* status, cudaStream_t st) {
    RankList rl{};
    rl.n = n_k;
    for (int j = 0; j < n_k; ++j) rl.r[j] = ranks[j];
    segmented_select_kernel<<<n_seg, kSelThreads, 0, st>>>(values, seg_off, uniform_len, rl, out, status);
    return cuda_error(cudaGetLastError(), "segmented_select launch");
}

}  // namespace

// Argument checks shared by the label entry points (also the allocation-free one).
int check_em_args(int sde, const float* theta, const float* Yi, const float* dt, int n_rows,
                  int64_t n_paths, int n_fine) {
    if (sde != SL_SDE_GBM && sde != SL_SDE_OU && sde != SL_SDE_CIR)
        return set_error(SL_ERR_ARG, "sde=%d", sde);
    if (!theta || !Yi || !dt) return set_error(SL_ERR_ARG, "theta / Yi / dt == NULL");
    if (n_rows < 0 || n_rows > 65535) return set_error(SL_ERR_UNSUPPORTED, "n_rows=%d outside [0,65535]", n_rows);
    if (n_paths < 0 || n_paths > (int64_t(1) << 31) - 1)
        return set_error(SL_ERR_UNSUPPORTED, "n_paths=%lld outside [0,2^31)", (long long)n_paths);
    if (n_fine < 1) return set_error(SL_ERR_UNSUPPORTED, "n_fine=%d < 1", n_fine);
    return SL_OK;
}

}  // namespace sl

using namespace sl;

extern "C" {

int sl_em_terminal(int sde, const float* theta, const float* Yi, const float* dt, int n_rows,
                   int64_t n_paths, int n_fine, uint64_t seed, float* out, void* stream) {
    int rc = check_em_args(sde, theta, Yi, dt, n_rows, n_paths, n_fine);
    if (rc) return rc;
    if (!out) return set_error(SL_ERR_ARG, "out == NULL");
    if (n_rows == 0 || n_paths == 0) return SL_OK;
    return launch_em(sde, theta, Yi, dt, n_rows, n_paths, n_fine, seed, out,
                     static_cast<cudaStream_t>(stream));
}

size_t sl_select_workspace_size(int n_seg, int n_k) {
    (void)n_seg;
    (void)n_k;
    return kStatusBytes;
}

int sl_segmented_select(const float* values, const int64_t* seg_offsets, int n_seg,
                        const int64_t* ranks, int n_k, float* out, void* ws, size_t ws_bytes,
                        void* stream) {
    if (n_seg < 0) return set_error(SL_ERR_ARG, "n_seg < 0");
    if (n_k < 1 || n_k > kMaxK) return set_error(SL_ERR_UNSUPPORTED, "n_k=%d outside [1,%d]", n_k, kMaxK);
    if (!ranks || !out || !seg_offsets) return set_error(SL_ERR_ARG, "NULL argument");
    for (int j = 0; j < n_k; ++j)
        if (ranks[j] < 0) return set_error(SL_ERR_ARG, "ranks[%d] < 0", j);
    if (!ws || ws_bytes < kStatusBytes) return set_error(SL_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(ws);
    int rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (n_seg == 0) return SL_OK;
    if (!values) return set_error(SL_ERR_ARG, "values == NULL");
    return launch_select(values, seg_offsets, 0, n_seg, ranks, n_k, out, status, st);
}

size_t sl_em_labels_workspace_size(int n_rows, int64_t n_paths, int m) {
    (void)m;
    if (n_rows < 0) n_rows = 0;
    if (n_paths < 0) n_paths = 0;
    return kStatusBytes + align256(static_cast<size_t>(n_rows) * static_cast<size_t>(n_paths) * 4);
}

int em_collocation_labels(int sde, const float* theta, const float* Yi, const float* dt,
                          int n_rows, int64_t n_paths, int n_fine, int m, uint64_t seed,
                          float* labels, void* ws, size_t ws_bytes, void* stream) {
    int rc = check_em_args(sde, theta, Yi, dt, n_rows, n_paths, n_fine);
    if (rc) return rc;
    if (!labels) return set_error(SL_ERR_ARG, "labels == NULL");
    if (n_paths < 1) return set_error(SL_ERR_ARG, "n_paths < 1");
    int64_t ranks[SL_MAX_M];
    rc = sl_quantile_ranks(m, n_paths, ranks);
    if (rc) return rc;
    const size_t need = sl_em_labels_workspace_size(n_rows, n_paths, m);
    if (!ws || ws_bytes < need)
        return set_error(SL_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* w = static_cast<unsigned char*>(ws);
    unsigned* status = reinterpret_cast<unsigned*>(w);
    float* samples = reinterpret_cast<float*>(w + kStatusBytes);
    rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (n_rows == 0) return SL_OK;
    rc = launch_em(sde, theta, Yi, dt, n_rows, n_paths, n_fine, seed, samples, st);
    if (rc) return rc;
    return launch_select(samples, nullptr, n_paths, n_rows, ranks, m, labels, status, st);
}

}  // extern "C"
