// sl_internal.cuh -- shared internals of the B300 Seven-League library
// (device helpers used by every kernel, host helpers used by every entry point).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sevenleague.h"

namespace sl {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int set_error(int status, const char* fmt, ...);   // records text, returns status
int cuda_error(cudaError_t e, const char* where);  // SL_OK if e == cudaSuccess
int sm_count();                                    // SMs of the current device

constexpr size_t kStatusBytes = 256;                // status word region at ws[0]
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Gauss-Hermite points, weights and first-form barycentric weights (FP64, host).
int gauss_hermite_fp64(int m, double* x, double* w, double* bary);

// FP32 copies of the collocation abscissae and barycentric weights, passed to
// kernels by value (kernel parameter space is a constant bank).
struct GHConst {
    float x[SL_MAX_M];
    float bary[SL_MAX_M];
    float dsc[SL_MAX_M];    // X - x_j as fmaf(X, dsc_j, doff_j): (1, -x_j) for j < m,
    float doff[SL_MAX_M];   // (0, 1) for the unused nodes j >= m (a factor 1 in every product)
};
int make_gh_const(int m, GHConst* out);
// Euler-Maruyama label arguments (sde, pointers, sizes): SL_OK or the error code.
int check_em_args(int sde, const float* theta, const float* Yi, const float* dt, int n_rows, int64_t n_paths,
                  int n_fine);

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key bump between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits, exact in FP32.
__device__ __forceinline__ float word_to_uniform(uint32_t w) {
    return (static_cast<float>(w >> 9) + 0.5f) * 0x1p-23f;
}

// Normals 4*block .. 4*block+3 of the stream (seed, tag, set, path):
// Box-Muller on word pairs (0,1) and (2,3); (cos, sin) of each pair.
__device__ __forceinline__ float4 normal4(uint64_t seed, uint32_t tag, uint32_t set,
                                          uint32_t path, uint32_t block) {
    const uint4 w = philox4x32_10(make_uint4(block, path, set, tag), static_cast<uint32_t>(seed),
                                  static_cast<uint32_t>(seed >> 32));
    const float r0 = sqrtf(-2.0f * logf(word_to_uniform(w.x)));
    const float r1 = sqrtf(-2.0f * logf(word_to_uniform(w.z)));
    float s0, c0, s1, c1;
    sincospif(2.0f * word_to_uniform(w.y), &s0, &c0);
    sincospif(2.0f * word_to_uniform(w.w), &s1, &c1);
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

__device__ __forceinline__ float pick4(const float4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// g_m(X) through (x_j, y_j) for a runtime m <= SL_MAX_M: first (modified-Lagrange)
// barycentric form ell(X) sum_j bary_j y_j / (X - x_j), evaluated without division as
// sum_j y_j bary_j prod_{k<j}(X-x_k) prod_{k>j}(X-x_k).  Stable when X lies outside
// [x_0, x_{m-1}] (the second form cancels there).  The unused nodes j >= m contribute a
// factor 1 to every product and a zero term (their barycentric weights are 0).
__device__ __forceinline__ float lagrange_eval_m(const float (&y)[SL_MAX_M], float X,
                                                 const GHConst& gh, int m) {
    float d[SL_MAX_M], pre[SL_MAX_M];
#pragma unroll
    for (int j = 0; j < SL_MAX_M; ++j) d[j] = (j < m) ? X - gh.x[j] : 1.0f;
    pre[0] = 1.0f;
#pragma unroll
    for (int j = 1; j < SL_MAX_M; ++j) pre[j] = pre[j - 1] * d[j - 1];
    float acc = 0.0f, suf = 1.0f;
#pragma unroll
    for (int j = SL_MAX_M - 1; j >= 0; --j) {
        acc = fmaf(y[j] * gh.bary[j], pre[j] * suf, acc);
        suf *= d[j];
    }
    return acc;
}

// The Lagrange basis ell_j(X) for a runtime m <= SL_MAX_M (ell_j = 0 for j >= m),
// so that g_m(X) = sum_j y_j ell_j can be finished with m FMAs once y is known.
__device__ __forceinline__ void lagrange_basis_m(float X, const GHConst& gh, int m, float (&l)[SL_MAX_M]) {
    (void)m;   // the unused nodes are folded into gh.dsc / gh.doff
    float d[SL_MAX_M], pre[SL_MAX_M];
#pragma unroll
    for (int j = 0; j < SL_MAX_M; ++j) d[j] = fmaf(X, gh.dsc[j], gh.doff[j]);
    pre[0] = 1.0f;
#pragma unroll
    for (int j = 1; j < SL_MAX_M; ++j) pre[j] = pre[j - 1] * d[j - 1];
    float suf = 1.0f;
#pragma unroll
    for (int j = SL_MAX_M - 1; j >= 0; --j) {
        l[j] = gh.bary[j] * (pre[j] * suf);
        suf *= d[j];
    }
}

// Largest s with offsets[s] <= g (empty sets are skipped).
__device__ __forceinline__ int owning_set(const int64_t* __restrict__ off, int n_sets, int64_t g) {
    int lo = 0, hi = n_sets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void raise_status(unsigned* status, unsigned bits) {
    if (status) atomicOr(status, bits);
}

// Checked builds (-DSL_CHECKED: libsevenleague_checked.so) verify the indices the kernels
// derive from caller data -- a path's set s must satisfy offsets[s] <= g < offsets[s+1], a
// listed path must lie below the path count -- and on a failure set a status bit and skip
// the path's outputs instead of trusting the index.  The normal build compiles them away.
#ifdef SL_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Flat path g lies in set s (checked builds; always true otherwise).
__device__ __forceinline__ bool path_in_set(const int64_t* off, int s, int64_t g, unsigned* status) {
    if (!kChecked || !off) return true;
    const bool ok = __ldg(off + s) <= g && g < __ldg(off + s + 1);
    if (!ok) raise_status(status, SL_DEV_OFFSETS);
    return ok;
}

// Kernel-side description of a 7L sampling call (shared by all forms).
struct SimArgs {
    const float* params;      // network parameters (FP32, flat)
    int d_in;
    int act;
    const float* theta;       // [n_sets][p]
    int p;
    const float* Y0;          // [n_sets] or NULL -> y0_scalar
    float y0_scalar;
    const int64_t* offsets;   // [n_sets+1] or NULL -> one set of `total` paths
    int n_sets;
    int64_t total;            // paths this call runs (outputs are indexed 0 .. total-1)
    int64_t first;            // flat index, in the batch `offsets` describes, of the call's first path
    float dt;
    int n_steps;
    uint64_t seed;
    float* out_YT;            // [total] or NULL
    float* out_grid;          // [(n_steps+1)][total] or NULL
    int grid_k;               // >1: out_grid keeps only rows Y_0, Y_k, Y_2k, .. (row i/k), BF16 form only
    unsigned* status;         // device status word or NULL
    int m;                    // collocation points
    GHConst gh;
};

// Launchers implemented in the kernel translation units.
int launch_simt_7l(int model, int m, const SimArgs& a, cudaStream_t s);
int launch_tc_7l(int m, const SimArgs& a, cudaStream_t s);
int launch_set_moments(const float* y, const int64_t* offsets, int n_sets, int64_t total,
                       double* mean, double* var, void* part, cudaStream_t s, int mean_stride = 1,
                       const double* scale = nullptr);
size_t set_moments_scratch_bytes(int n_sets);
// local[s] = clamp(offsets[s] - first, 0, n) for s <= n_sets; count[s] = local[s+1] - local[s] (or NULL).
int launch_range_offsets(const int64_t* offsets, int n_sets, int64_t first, int64_t n, int64_t* local,
                         int64_t* count, cudaStream_t st);

}  // namespace sl
