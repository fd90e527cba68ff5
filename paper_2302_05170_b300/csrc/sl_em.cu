// sl_em.cu -- offline stage of the 7L scheme (Algorithm I, step 1):
// fine-step Euler-Maruyama terminal samples (Eq. 6.2) and their empirical
// quantiles at levels Phi(x_j), the collocation labels y_j | (theta, Y_i, dt).
//
// EM: two paths per thread, the whole fine-step loop in registers; the only
// memory traffic is the 4-byte terminal sample; the normals' Box-Muller uses the
// fast logarithm, sine/cosine and square root (normal4_fast).  Select: one CTA per segment,
// exact MSD radix select over the order-preserving 32-bit keys, all requested ranks at once:
// a 14-bit first digit counted in shared memory, then either the ranks' bins copied to shared
// memory and finished there, or two more 9-bit passes over the segment; the segment is read
// as float4 where it is 16-byte aligned.
#include <math.h>

#include "sl_internal.cuh"
#include "sl_fastnormal.cuh"

namespace sl {
namespace {

constexpr int kEmThreads = 256;
constexpr int kSelThreads = 1024;                 // one CTA per SM (see the kernel)
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kMaxK = 16;
constexpr int kD1 = 14;                       // select: first digit, the keys' top 14 bits
constexpr int kBins1 = 1 << kD1;
constexpr int kD2 = 9;                        // refine digits (9 + 9 bits)
constexpr int kBins2 = 1 << kD2;
constexpr int kCandCap = 40960;                // keys the collect step holds in shared memory
// byte table of the ranks' bins, then the histogram, whose space (and 28 KB more) holds the keys
constexpr size_t kSelSmem = static_cast<size_t>(kBins1) + static_cast<size_t>(kCandCap) * 4;
static_assert(kMaxK * kBins2 <= kBins1, "refine histograms reuse the first digit's");
static_assert(kD1 + 2 * kD2 == 32 && (32 - kD1) % 6 == 0, "digits cover the key");
constexpr int kBPT = kBins1 / kSelThreads;     // first-digit bins per thread in the scan
static_assert(kBPT * kSelThreads == kBins1 && kMaxK <= kSelWarps, "first-digit bins per thread, one warp per rank");

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
    // whole blocks of four fine steps (one Philox call per path each), then the remainder; the
    // Philox round keys once per thread (2.3 % of the stage)
    const int n4 = n_fine >> 2;
    const PhiloxKeys K = philox_keys(seed);
    for (int k = 0; k < n4; ++k) {
#pragma unroll
        for (int p = 0; p < kEmPaths; ++p) {
            const float4 z = normal4_fast_keyed(K, 1u, static_cast<uint32_t>(r), qq[p], static_cast<uint32_t>(k));
            step(Y[p], z.x);
            step(Y[p], z.y);
            step(Y[p], z.z);
            step(Y[p], z.w);
        }
    }
    if (n_fine & 3) {
#pragma unroll
        for (int p = 0; p < kEmPaths; ++p) {
            const float4 z = normal4_fast_keyed(K, 1u, static_cast<uint32_t>(r), qq[p], static_cast<uint32_t>(n4));
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

// The select reads a segment with every thread of the CTA: the 16-byte aligned body as float4
// (four per thread per round, so that 16 KB per CTA are in flight), the unaligned head and tail
// (at most three values each) by warp 0.  f(key, in) is called warp-converged; `in` is false for
// the padding lanes.
struct SegSpan {
    int64_t a, a4, n4;
    int head, tail;
};
__device__ __forceinline__ SegSpan seg_span(const float* values, int64_t a, int64_t n) {
    SegSpan sp;
    const int64_t mis = static_cast<int64_t>((reinterpret_cast<uintptr_t>(values) >> 2) & 3u);
    sp.a = a;
    sp.a4 = min(a + ((4 - ((mis + a) & 3)) & 3), a + n);
    const int64_t e4 = max(sp.a4, a + n - ((mis + a + n) & 3));
    sp.n4 = (e4 - sp.a4) >> 2;
    sp.head = static_cast<int>(sp.a4 - a);
    sp.tail = static_cast<int>(a + n - e4);
    return sp;
}
template <class F>
__device__ __forceinline__ void for_each_key(const float* __restrict__ values, const SegSpan& sp, F&& f) {
    const int tid = threadIdx.x, lane = tid & 31;
    const float4* body = reinterpret_cast<const float4*>(values + sp.a4);
    constexpr int U = 4;
    for (int64_t base = 0; base < sp.n4; base += U * kSelThreads) {
        float4 v[U];
        bool in[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = base + u * kSelThreads + tid;
            in[u] = c < sp.n4;
            v[u] = in[u] ? __ldg(body + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            f(float_key(v[u].x), in[u]);
            f(float_key(v[u].y), in[u]);
            f(float_key(v[u].z), in[u]);
            f(float_key(v[u].w), in[u]);
        }
    }
    if ((tid >> 5) == 0) {
        const int64_t idx = (lane < sp.head) ? sp.a + lane : sp.a4 + 4 * sp.n4 + (lane - sp.head);
        const bool in = lane < sp.head + sp.tail;
        f(float_key(in ? __ldg(values + idx) : 0.0f), in);
    }
}

// Exclusive prefix of v over the CTA (returned) and the total; `part` holds kSelWarps words.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* part, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kSelWarps) ? part[lane] : 0u, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kSelWarps) part[lane] = wi - w;   // exclusive prefix of the warp totals
        if (lane == kSelWarps - 1) part[kSelWarps] = wi;
    }
    __syncthreads();
    total = part[kSelWarps];
    const uint32_t r = part[warp] + incl - v;
    __syncthreads();   // part is reused by the caller's next scan
    return r;
}

// Appends to cand (one cursor, *n_cand) the keys of the segment whose first-digit bin is marked in
// `lookup`, in no particular order.  The segment is read last float4 first: its end is the part
// most likely still in L2 from the read just before.  Each thread marks the hits among its 16
// keys of a round in a bit mask; a warp scan of the hit counts places them, with one shared add
// per warp and round.  Slots past cap are not written (the caller has checked that the marked bins
// fit; a segment that changed under the select raises SL_DEV_INDEX).
template <int N>
__device__ __forceinline__ void warp_append(const uint32_t (&k)[N], uint32_t hits, uint32_t* cand,
                                            uint32_t* n_cand, uint32_t cap, unsigned* status) {
    const int lane = threadIdx.x & 31;
    const uint32_t c = static_cast<uint32_t>(__popc(hits));
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tot == 0u) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(n_cand, tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t pos = base + incl - c;
    if (hits) {
        if (pos + c > cap) raise_status(status, SL_DEV_INDEX);
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((hits >> i) & 1u) {
                if (pos < cap) cand[pos] = k[i];
                ++pos;
            }
    }
}

__device__ __forceinline__ void collect_keys(const float* __restrict__ values, const SegSpan& sp,
                                             const uint8_t* lookup, uint32_t* cand, uint32_t* n_cand,
                                             uint32_t cap, unsigned* status) {
    const int tid = threadIdx.x, lane = tid & 31;
    const float4* body = reinterpret_cast<const float4*>(values + sp.a4);
    constexpr int U = 4;
    constexpr int64_t R = static_cast<int64_t>(U) * kSelThreads;
    if (sp.n4 > 0) {
        for (int64_t base = ((sp.n4 - 1) / R) * R; base >= 0; base -= R) {
            float4 v[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t c = base + u * kSelThreads + tid;
                in[u] = c < sp.n4;
                v[u] = in[u] ? __ldg(body + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            uint32_t k[4 * U], hits = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                k[4 * u] = float_key(v[u].x);
                k[4 * u + 1] = float_key(v[u].y);
                k[4 * u + 2] = float_key(v[u].z);
                k[4 * u + 3] = float_key(v[u].w);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (in[u] && lookup[k[4 * u + e] >> (32 - kD1)]) hits |= 1u << (4 * u + e);
            }
            warp_append(k, hits, cand, n_cand, cap, status);
        }
    }
    if ((tid >> 5) == 0) {
        const int64_t idx = (lane < sp.head) ? sp.a + lane : sp.a4 + 4 * sp.n4 + (lane - sp.head);
        const bool in = lane < sp.head + sp.tail;
        const uint32_t k1[1] = {float_key(in ? __ldg(values + idx) : 0.0f)};
        warp_append(k1, (in && lookup[k1[0] >> (32 - kD1)]) ? 1u : 0u, cand, n_cand, cap, status);
    }
}

// One CTA per segment; every requested rank of the segment at once; exact.
//   pass 1:  a histogram of the keys' top 14 bits (16,384 bins in shared memory, one shared add
//            per value) gives each rank its bin and its rank within the bin;
//   collect: when the distinct bins of the ranks hold at most kCandCap values together, a second
//            read of the segment copies those values into shared memory (the histogram's space and
//            more), and the CTA finishes every rank at once with three 6-bit radix passes over
//            them;
//   refine:  otherwise (a value repeated very often, or very narrow data) two more passes over the
//            segment with 9-bit digits, one histogram per distinct prefix.
// A byte table marks the bins of the ranks, so the later passes skip every other value after one
// shared-memory load.  One CTA of 1024 threads per SM (176 KB of shared memory): the 148
// segments in flight (59 MB for 1e5-value segments) stay in the 126 MB L2 between the two
// reads, and the candidate buffer holds 40,960 keys, so narrow rows rarely refine (CIR labels,
// 1024 x 1e5: 0.250 ms against 0.332 ms with two CTAs of 512 threads per SM and 22,528
// candidates; lognormal values: 0.240 against 0.221 ms).
__global__ void __launch_bounds__(kSelThreads, 1)
segmented_select_kernel(const float* __restrict__ values, const int64_t* __restrict__ seg_off,
                        int64_t uniform_len, RankList ranks, float* __restrict__ out,
                        unsigned* status) {
    extern __shared__ __align__(16) uint32_t sel_smem[];
    uint8_t* lookup = reinterpret_cast<uint8_t*>(sel_smem);              // [kBins1] group + 1 of a bin, 0 = none
    uint32_t* hist = sel_smem + kBins1 / 4;                               // [kBins1] pass 1; refine: [kMaxK][kBins2]
    uint32_t* cand = hist;                                                // [kCandCap] collected keys (over hist)
    __shared__ uint32_t fh[kMaxK * 64];                                   // finish: per-rank 6-bit digit counts
    __shared__ uint32_t prefix[kMaxK], gprefix[kMaxK], gcnt[kMaxK], gmask[kMaxK];
    __shared__ uint32_t n_cand;
    __shared__ uint32_t part[kSelWarps + 1];
    __shared__ int64_t rem[kMaxK];
    __shared__ int group_of[kMaxK];
    __shared__ int n_groups, collect;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a = seg_off ? seg_off[s] : static_cast<int64_t>(s) * uniform_len;
    const int64_t n = (seg_off ? seg_off[s + 1] : a + uniform_len) - a;
    const int nk = ranks.n;
    if (n < 0 || n >= (int64_t(1) << 31)) {
        if (tid == 0) raise_status(status, SL_DEV_OFFSETS);
        if (tid < nk) out[static_cast<int64_t>(s) * nk + tid] = __int_as_float(0x7fc00000);
        return;
    }
    const SegSpan sp = seg_span(values, a, n);
    for (int i = tid; i < kBins1; i += kSelThreads) hist[i] = 0u;
    for (int i = tid; i < kBins1 / 4; i += kSelThreads) sel_smem[i] = 0u;   // lookup
    if (tid < nk) {
        prefix[tid] = 0u;
        rem[tid] = ranks.r[tid];
        group_of[tid] = -1;
    }
    __syncthreads();

    // pass 1: top 14 bits
    for_each_key(values, sp, [&](uint32_t key, bool in) {
        if (in) atomicAdd(&hist[key >> (32 - kD1)], 1u);
    });
    __syncthreads();
    {   // thread t owns bins kBPT t .. kBPT t + kBPT - 1 (read rotated by lane)
        uint32_t loc = 0;
#pragma unroll 8
        for (int i = 0; i < kBPT; ++i) loc += hist[kBPT * tid + ((i + lane) & (kBPT - 1))];
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(loc, part, total);
        for (int j = 0; j < nk; ++j) {
            const int64_t r = ranks.r[j];
            if (r >= n || r < static_cast<int64_t>(excl) || r >= static_cast<int64_t>(excl) + loc) continue;
            int64_t cum = excl;
            for (int i = 0; i < kBPT; ++i) {
                const uint32_t c = hist[kBPT * tid + i];
                if (r < cum + c) {
                    prefix[j] = static_cast<uint32_t>(kBPT * tid + i) << (32 - kD1);
                    rem[j] = r - cum;
                    break;
                }
                cum += c;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {   // distinct bins of the valid ranks; collect them if they fit
        int ng = 0;
        uint32_t off = 0;
        for (int j = 0; j < nk; ++j) {
            if (ranks.r[j] >= n) continue;
            int g = 0;
            while (g < ng && gprefix[g] != prefix[j]) ++g;
            if (g == ng) {
                gprefix[ng] = prefix[j];
                gcnt[ng] = hist[prefix[j] >> (32 - kD1)];
                gmask[ng] = 0u;
                off += gcnt[ng];
                lookup[prefix[j] >> (32 - kD1)] = static_cast<uint8_t>(ng + 1);
                ++ng;
            }
            group_of[j] = g;
            gmask[g] |= 1u << j;
        }
        n_groups = ng;
        n_cand = 0u;
        collect = off <= static_cast<uint32_t>(kCandCap);
    }
    __syncthreads();
    const int ng = n_groups;
    if (ng == 0) {
        // no rank below n: every output is NaN
    } else if (collect) {
        collect_keys(values, sp, lookup, cand, &n_cand, static_cast<uint32_t>(kCandCap), status);
        __syncthreads();
        const uint32_t total = min(n_cand, static_cast<uint32_t>(kCandCap));
        for (int shift = 32 - kD1 - 6; shift >= 0; shift -= 6) {
            for (int i = tid; i < nk * 64; i += kSelThreads) fh[i] = 0u;
            __syncthreads();
            for (uint32_t i = tid; i < total; i += kSelThreads) {
                const uint32_t k = cand[i];
                uint32_t msk = gmask[lookup[k >> (32 - kD1)] - 1];
                while (msk) {
                    const int j = __ffs(msk) - 1;
                    msk &= msk - 1u;
                    if ((k >> (shift + 6)) == (prefix[j] >> (shift + 6))) atomicAdd(&fh[j * 64 + ((k >> shift) & 63u)], 1u);
                }
            }
            __syncthreads();
            if (warp < nk && group_of[warp] >= 0) {   // warp j resolves rank j's digit
                const uint32_t* wh = fh + warp * 64;
                const uint32_t rk = static_cast<uint32_t>(rem[warp]);
                const uint32_t c0 = wh[2 * lane], c1 = wh[2 * lane + 1], loc = c0 + c1;
                uint32_t incl = loc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, rk < incl);
                const int src = hit ? __ffs(hit) - 1 : 31;
                if (lane == src) {
                    uint32_t below = incl - loc, digit = 2 * lane;
                    if (rk >= below + c0) {
                        below += c0;
                        digit += 1;
                    }
                    prefix[warp] |= digit << shift;
                    rem[warp] = rk - below;
                }
            }
            __syncthreads();
        }
    } else {
        // refine: 9-bit digits below the 14-bit prefix, hist as [kMaxK][kBins2]
        for (int pass = 0; pass < 2; ++pass) {
            const int shift = 32 - kD1 - kD2 * (pass + 1);
            const uint32_t hi_mask = ~((1u << (shift + kD2)) - 1u);
            if (tid == 0) {
                int g2 = 0;
                for (int j = 0; j < nk; ++j) {
                    group_of[j] = -1;
                    if (ranks.r[j] >= n) continue;
                    int g = 0;
                    while (g < g2 && gprefix[g] != prefix[j]) ++g;
                    if (g == g2) gprefix[g2++] = prefix[j];
                    group_of[j] = g;
                }
                n_groups = g2;
            }
            __syncthreads();
            const int ngr = n_groups;
            for (int i = tid; i < ngr * kBins2; i += kSelThreads) hist[i] = 0u;
            __syncthreads();
            for_each_key(values, sp, [&](uint32_t key, bool in) {
                if (!in || lookup[key >> (32 - kD1)] == 0) return;
                const uint32_t hk = key & hi_mask;
                for (int j = 0; j < ngr; ++j)
                    if (hk == gprefix[j]) {
                        atomicAdd(&hist[j * kBins2 + ((key >> shift) & (kBins2 - 1u))], 1u);
                        break;
                    }
            });
            __syncthreads();
            if (warp < nk && group_of[warp] >= 0) {   // warp j resolves rank j's digit
                const uint32_t* h = hist + group_of[warp] * kBins2;
                constexpr int B = kBins2 / 32;
                uint32_t c[B], loc = 0;
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    c[i] = h[lane * B + i];
                    loc += c[i];
                }
                uint32_t incl = loc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                const int64_t rk = rem[warp];
                const unsigned hit = __ballot_sync(0xffffffffu, rk < static_cast<int64_t>(incl));
                const int src = __ffs(hit) - 1;
                if (lane == src) {
                    int64_t cum = static_cast<int64_t>(incl - loc);
                    int bin = B * lane;
#pragma unroll
                    for (int i = 0; i < B; ++i) {
                        if (rk < cum + c[i]) {
                            bin = B * lane + i;
                            break;
                        }
                        cum += c[i];
                    }
                    rem[warp] = rk - cum;
                    prefix[warp] |= static_cast<uint32_t>(bin) << shift;
                }
            }
            __syncthreads();
        }
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
    const int attr_rc = cuda_error(cudaFuncSetAttribute(segmented_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        static_cast<int>(kSelSmem)),
                                   "segmented_select attribute");
    if (attr_rc) return attr_rc;
    segmented_select_kernel<<<n_seg, kSelThreads, kSelSmem, st>>>(values, seg_off, uniform_len, rl, out, status);
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
