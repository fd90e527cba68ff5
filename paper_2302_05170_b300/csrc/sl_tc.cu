// sl_tc.cu -- BF16 tensor-core (tcgen05) form of the 7L online sampler
// (Algorithm I, steps 2-8) for sm_103a.
//
// The network of Eq. (6.4) is a chain of five GEMMs per coarse step:
//   layer 1:   [128 paths x K=16]  x [K x N=64]      (features, hi+lo split)
//   layers 2-4 [128 paths x K=112] x [K x N=64]      (50 activations hi, 1, lo)
//   layer 5:   [128 paths x K=112] x [K x N=16]      (m <= 8 outputs used)
// A persistent CTA (one per SM) holds S independent path tiles ("slots") of
// 128 paths.  Warp S*4 issues every tcgen05.mma (one elected lane), reading
// A (activations) and B (weights) from shared memory through 128-byte-swizzled
// K-major descriptors and accumulating in FP32 in tensor memory (64 columns
// per slot).  Warpgroup t (warps 4t..4t+3, TMEM lanes 32*(warp%4)..) is the
// epilogue of slot t: it reads the accumulator row of its path with
// tcgen05.ld, applies ReLU, splits every activation h into BF16 hi + lo
// (hi = h truncated to BF16, lo = BF16(h - hi)), and writes the next A tile.
// While one slot's MMAs run, the other slots' epilogues, Philox normals and
// g_m evaluations run, so tensor pipe and CUDA cores overlap.
//
// Numerics: weights and biases are rounded to BF16 (nearest, ties to even);
// the network's inputs and activations carry ~16 significant bits through the
// hi+lo split (a single BF16 rounding of every activation gives ~1e-2 per-path
// error over 16 steps, the split ~1e-5); accumulation is FP32; the state,
// normals and interpolation are FP32.  Biases ride on a constant-1 input column
// (column 50 of the hidden inputs, column 2*d_in of the features), so the
// epilogue adds nothing.
//
// Synchronisation: per slot, mbarrier a_ready (4 arrivals: one per epilogue
// warp, after its shared-memory writes and a proxy fence) and d_ready
// (1 arrival: tcgen05.commit after the layer's MMAs).  Every wait is bounded
// (about one second of global time); on expiry the kernel sets
// SL_DEV_TIMEOUT in the status word, all roles stop, the MMA warp drains its
// own MMAs (bounded) and the tensor memory is released.
#include <cuda_bf16.h>
#include <math.h>

#include "sl_internal.cuh"

namespace sl {
namespace {

constexpr int kTile = 128;                    // paths per slot (MMA M, TMEM lanes)
constexpr int kRowBytes = 128;                // one 128B-swizzle row = 64 BF16
constexpr int kAAtomBytes = kTile * kRowBytes;           // 16 KB: 128 rows x 64 cols
constexpr int kASlotBytes = 2 * kAAtomBytes;             // K = 112 -> two 64-col atoms
constexpr int kB1Bytes = 64 * kRowBytes;                 // layer 1: 64 rows x (16 of 64) cols
constexpr int kBHBytes = 2 * 64 * kRowBytes;             // hidden: 64 rows x 112 cols
constexpr int kB5Bytes = 2 * 16 * kRowBytes;             // output: 16 rows x 112 cols
constexpr int kBBytes = kB1Bytes + 3 * kBHBytes + kB5Bytes;
constexpr int kLoCol = 56;                               // first column of the lo half
constexpr int kBiasCol = 50;                             // constant-1 column
constexpr uint64_t kTimeoutNs = 1000000000ull;           // bounded waits: 1 s

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on abort/timeout.
__device__ __noinline__ bool mbar_wait_slow(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                            unsigned* status) {
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(addr, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > kTimeoutNs) {
            *abort_flag = 1;
            raise_status(status, SL_DEV_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                          unsigned* status) {
#pragma unroll 1
    for (int it = 0; it < 64; ++it)
        if (mbar_try_wait(addr, parity)) return true;
    return mbar_wait_slow(addr, parity, abort_flag, status);
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128 B,
// 8-row atoms 1024 B apart (stride byte offset), fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (static_cast<uint64_t>((saddr >> 4) & 0x3FFFu)) |
           (static_cast<uint64_t>(1u) << 16) |                       // leading byte offset (unused)
           (static_cast<uint64_t>(1024u >> 4) << 32) |               // stride byte offset
           (static_cast<uint64_t>(1u) << 46) |                       // descriptor version
           (static_cast<uint64_t>(2u) << 61);                        // SWIZZLE_128B
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// (lo element, hi element) -> packed BF16x2 with ReLU; lo element in the low half.
__device__ __forceinline__ uint32_t pack_relu(float lo_elem, float hi_elem) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
    return d;
}
__device__ __forceinline__ uint32_t pack_rn(float lo_elem, float hi_elem) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
    return d;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Byte offset of 16-byte chunk `c` (0..7) of row `r` inside a 128B-swizzled atom.
__device__ __forceinline__ uint32_t sw128_chunk(int r, int c) {
    return static_cast<uint32_t>((r >> 3) * 1024 + (r & 7) * kRowBytes + ((c ^ (r & 7)) << 4));
}

// Byte offset of element (row n, column k) of a B tile with `rows` rows.
__device__ __forceinline__ uint32_t b_elem_off(int rows, int n, int k) {
    const int atom = k >> 6, kc = k & 63;
    return static_cast<uint32_t>(atom * rows * kRowBytes) + sw128_chunk(n, kc >> 3) +
           static_cast<uint32_t>((kc & 7) * 2);
}

// Stage the network's weights as BF16 B tiles.
//   B1[n][2i] = B1[n][2i+1] = W1[n][i] (i < d_in), B1[n][2 d_in] = b1[n]
//   Bl[n][k] = Wl[n][k], Bl[n][50] = bl[n], Bl[n][56+k] = Wl[n][k] (k < 50)
__device__ void stage_weights(unsigned char* sB, const float* __restrict__ P, int d_in, int m) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int W = SL_WIDTH;
    for (int i = tid; i < kBBytes / 2; i += nt) reinterpret_cast<uint16_t*>(sB)[i] = 0;
    __syncthreads();
    // layer 1
    const float* W1 = P;
    const float* b1 = P + W * d_in;
    for (int i = tid; i < W * 16; i += nt) {
        const int n = i / 16, k = i % 16;
        float v = 0.0f;
        if (k < 2 * d_in) v = W1[n * d_in + (k >> 1)];
        else if (k == 2 * d_in) v = b1[n];
        else continue;
        *reinterpret_cast<__nv_bfloat16*>(sB + b_elem_off(64, n, k)) = __float2bfloat16_rn(v);
    }
    const float* p = b1 + W;
    unsigned char* dst = sB + kB1Bytes;
    for (int l = 0; l < 4; ++l) {
        const int rows = (l < 3) ? 64 : 16;
        const int n_out = (l < 3) ? W : m;
        const float* Wl = p;
        const float* bl = p + n_out * W;
        for (int i = tid; i < n_out * 112; i += nt) {
            const int n = i / 112, k = i % 112;
            float v;
            if (k < W) v = Wl[n * W + k];
            else if (k == kBiasCol) v = bl[n];
            else if (k >= kLoCol && k < kLoCol + W) v = Wl[n * W + (k - kLoCol)];
            else continue;
            *reinterpret_cast<__nv_bfloat16*>(dst + b_elem_off(rows, n, k)) = __float2bfloat16_rn(v);
        }
        p = bl + n_out;
        dst += (l < 3) ? kBHBytes : kB5Bytes;
    }
}

struct TileState {
    int64_t g;      // flat path index
    int s;          // owning set
    uint32_t q;     // path index within the set
    bool valid;
};

template <int S>
__global__ void __launch_bounds__(32 * (4 * S + 1), 1) tc_7l_kernel(const SimArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* sB = smem;                                  // weights (1024-aligned)
    unsigned char* sA = smem + kBBytes;                        // S slots x 32 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + S * kASlotBytes);   // a_ready[S], d_ready[S], drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mma_warp = 4 * S;
    constexpr uint32_t kCols = (S * 64 <= 32) ? 32 : (S * 64 <= 64) ? 64 : (S * 64 <= 128) ? 128
                               : (S * 64 <= 256) ? 256 : 512;

    if (threadIdx.x == 0) {
        for (int t = 0; t < S; ++t) {
            mbar_init(smem_u32(&bars[t]), 4);        // a_ready: one arrival per epilogue warp
            mbar_init(smem_u32(&bars[S + t]), 1);    // d_ready: tcgen05.commit
        }
        mbar_init(smem_u32(&bars[2 * S]), 1);        // drain
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    stage_weights(sB, a.params, a.d_in, a.m);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int64_t n_tiles = (a.total + kTile - 1) / kTile;
    const int64_t tile_stride = static_cast<int64_t>(gridDim.x) * S;

    if (warp == mma_warp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t sB_u = smem_u32(sB), sA_u = smem_u32(sA);
            int remaining[S];
            int layer[S];
            uint32_t aph[S];
            int64_t left = 0;
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const int64_t first = static_cast<int64_t>(blockIdx.x) * S + t;
                const int64_t ntl = first < n_tiles ? (n_tiles - 1 - first) / tile_stride + 1 : 0;
                remaining[t] = static_cast<int>(ntl * a.n_steps * 5);
                left += remaining[t];
                layer[t] = 0;
                aph[t] = 0;
            }
            uint64_t idle_since = 0;
            while (left > 0) {
                bool issued = false;
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    if (remaining[t] == 0 || !mbar_test(smem_u32(&bars[t]), aph[t])) continue;
                    aph[t] ^= 1u;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(t * 64);
                    const uint32_t a_base = sA_u + static_cast<uint32_t>(t * kASlotBytes);
                    const int l = layer[t];
                    if (l == 0) {
                        mma_bf16(d_tmem, sw128_desc(a_base), sw128_desc(sB_u), idesc_bf16(128, 64), 0u);
                    } else {
                        const uint32_t b_base = (l < 4) ? sB_u + kB1Bytes + (l - 1) * kBHBytes
                                                        : sB_u + kB1Bytes + 3 * kBHBytes;
                        const int rows = (l < 4) ? 64 : 16;
                        const uint32_t idesc = idesc_bf16(128, rows);
#pragma unroll
                        for (int k = 0; k < 7; ++k) {
                            const uint32_t aoff = (k < 4) ? k * 32 : kAAtomBytes + (k - 4) * 32;
                            const uint32_t boff = (k < 4) ? k * 32 : rows * kRowBytes + (k - 4) * 32;
                            mma_bf16(d_tmem, sw128_desc(a_base + aoff), sw128_desc(b_base + boff),
                                     idesc, k > 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(smem_u32(&bars[S + t]));
                    layer[t] = (l == 4) ? 0 : l + 1;
                    --remaining[t];
                    --left;
                    issued = true;
                }
                if (issued) {
                    idle_since = 0;
                } else {   // bounded idling: give up after ~1 s with nothing ready
                    const uint64_t now = global_ns();
                    if (idle_since == 0) idle_since = now;
                    else if (now - idle_since > kTimeoutNs) {
                        *abort_flag = 1;
                        raise_status(a.status, SL_DEV_TIMEOUT);
                        break;
                    }
                    if (*abort_flag) break;
                }
            }
            // Drain: wait until every MMA this thread issued has completed.
            mma_commit(smem_u32(&bars[2 * S]));
            uint64_t t0 = global_ns();
            while (!mbar_try_wait(smem_u32(&bars[2 * S]), 0)) {
                if (global_ns() - t0 > kTimeoutNs) {
                    raise_status(a.status, SL_DEV_TIMEOUT);
                    break;
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue of slot t
        const int t = warp >> 2, wq = warp & 3;
        const int r = wq * 32 + lane;                          // row = TMEM lane = path in tile
        const uint32_t a_slot = smem_u32(sA) + static_cast<uint32_t>(t * kASlotBytes);
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(wq * 32) << 16) +
                               static_cast<uint32_t>(t * 64);
        const uint32_t a_bar = smem_u32(&bars[t]), d_bar = smem_u32(&bars[S + t]);
        uint32_t dph = 0;
        bool ok = true;
        const float dt = a.dt;
        for (int64_t tile = static_cast<int64_t>(blockIdx.x) * S + t; ok && tile < n_tiles;
             tile += tile_stride) {
            TileState ts;
            ts.g = tile * kTile + r;
            ts.valid = ts.g < a.total;
            ts.s = 0;
            int64_t qq = ts.g;
            if (a.offsets) {
                ts.s = owning_set(a.offsets, a.n_sets, ts.valid ? ts.g : a.total - 1);
                qq = ts.g - __ldg(a.offsets + ts.s);
            }
            ts.q = static_cast<uint32_t>(qq);
            const float* th = a.theta + static_cast<int64_t>(ts.s) * a.p;
            float feat[SL_MAX_DIN_TC];
            feat[0] = 0.0f;
            feat[1] = dt;
#pragma unroll
            for (int k = 0; k < SL_MAX_DIN_TC - 2; ++k) feat[2 + k] = (k < a.p) ? __ldg(th + k) : 0.0f;
            float Y = a.Y0 ? __ldg(a.Y0 + ts.s) : a.y0_scalar;
            if (a.out_grid && ts.valid) a.out_grid[ts.g] = Y;
            float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

            for (int i = 0; ok && i < a.n_steps; ++i) {
                // ---- features [Y, dt, theta] as (hi, lo) BF16 pairs + constant 1 (layer-1 A)
                feat[0] = Y;
                uint32_t fw[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) fw[k] = 0u;
#pragma unroll
                for (int k = 0; k < SL_MAX_DIN_TC; ++k) {
                    const float hi = __uint_as_float(__float_as_uint(feat[k]) & 0xFFFF0000u);
                    const uint32_t wv = pack_rn(hi, feat[k] - hi);
                    fw[k] = (k < a.d_in) ? wv : ((k == a.d_in) ? 0x00003F80u : 0u);   // 1.0 after the features
                }
                if (a.d_in == SL_MAX_DIN_TC) fw[7] = 0x00003F80u;
                st_shared_v4(a_slot + sw128_chunk(r, 0), fw[0], fw[1], fw[2], fw[3]);
                st_shared_v4(a_slot + sw128_chunk(r, 1), fw[4], fw[5], fw[6], fw[7]);
                fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(a_bar);

                // ---- hidden layers: accumulator -> ReLU -> hi/lo BF16 -> next A
                for (int l = 0; l < 4; ++l) {
                    ok = mbar_wait(d_bar, dph, abort_flag, a.status);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    dph ^= 1u;
                    tc_fence_after();
                    // columns 0..31: hi words 0..15 (chunks 0-3), lo words 28..43
                    // (chunk 7, atom-1 chunks 0-2)
                    {
                        uint32_t v[32];
                        tmem_ld32(taddr, v);
                        tmem_wait_ld();
                        uint32_t hw[16], lw[16];
#pragma unroll
                        for (int i2 = 0; i2 < 16; ++i2) {
                            const float ha = __uint_as_float(v[2 * i2] & 0xFFFF0000u);
                            const float hb = __uint_as_float(v[2 * i2 + 1] & 0xFFFF0000u);
                            hw[i2] = pack_relu(ha, hb);
                            lw[i2] = pack_relu(__uint_as_float(v[2 * i2]) - ha, __uint_as_float(v[2 * i2 + 1]) - hb);
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            st_shared_v4(a_slot + sw128_chunk(r, c), hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        st_shared_v4(a_slot + sw128_chunk(r, 7), lw[0], lw[1], lw[2], lw[3]);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, c), lw[4 + 4 * c], lw[5 + 4 * c],
                                         lw[6 + 4 * c], lw[7 + 4 * c]);
                    }
                    // columns 32..49: hi words 16..24 (+ the constant-1 word 25), lo words 44..52
                    {
                        uint32_t v[16], u[8];
                        tmem_ld16(taddr + 32, v);
                        tmem_ld8(taddr + 48, u);
                        tmem_wait_ld();
                        uint32_t hw[9], lw[9];
#pragma unroll
                        for (int i2 = 0; i2 < 9; ++i2) {
                            const uint32_t ua = (i2 < 8) ? v[2 * i2] : u[0];
                            const uint32_t ub = (i2 < 8) ? v[2 * i2 + 1] : u[1];
                            const float ha = __uint_as_float(ua & 0xFFFF0000u);
                            const float hb = __uint_as_float(ub & 0xFFFF0000u);
                            hw[i2] = pack_relu(ha, hb);
                            lw[i2] = pack_relu(__uint_as_float(ua) - ha, __uint_as_float(ub) - hb);
                        }
                        st_shared_v4(a_slot + sw128_chunk(r, 4), hw[0], hw[1], hw[2], hw[3]);
                        st_shared_v4(a_slot + sw128_chunk(r, 5), hw[4], hw[5], hw[6], hw[7]);
                        st_shared_v4(a_slot + sw128_chunk(r, 6), hw[8], 0x00003F80u, 0u, 0u);
                        st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 3), lw[0], lw[1], lw[2], lw[3]);
                        st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 4), lw[4], lw[5], lw[6], lw[7]);
                        st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 5), lw[8], 0u, 0u, 0u);
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(a_bar);
                }
                if (!ok) break;
                // ---- output layer: collocation points y_0..y_{m-1}
                ok = mbar_wait(d_bar, dph, abort_flag, a.status);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                dph ^= 1u;
                tc_fence_after();
                uint32_t yv[8];
                tmem_ld8(taddr, yv);
                tmem_wait_ld();
                tc_fence_before();
                float y[SL_MAX_M];
#pragma unroll
                for (int j = 0; j < SL_MAX_M; ++j) y[j] = __uint_as_float(yv[j]);
                // ---- Philox normal and the 7L map g_m (Algorithm I steps 5-6)
                if ((i & 3) == 0)
                    z4 = normal4(a.seed, 0u, static_cast<uint32_t>(ts.s), ts.q, static_cast<uint32_t>(i >> 2));
                Y = lagrange_eval_m(y, pick4(z4, i & 3), a.gh, a.m);
                if (a.out_grid && ts.valid) a.out_grid[static_cast<int64_t>(i + 1) * a.total + ts.g] = Y;
            }
            if (ok && ts.valid) {
                if (a.out_YT) a.out_YT[ts.g] = Y;
                if (!isfinite(Y)) raise_status(a.status, SL_DEV_NONFINITE);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == mma_warp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kCols)
                     : "memory");
    }
}

template <int S>
size_t tc_smem_bytes() {
    return 1024 + kBBytes + static_cast<size_t>(S) * kASlotBytes + (2 * S + 1) * 8 + 16;
}

template <int S>
int launch_s(const SimArgs& a, cudaStream_t st) {
    auto kern = tc_7l_kernel<S>;
    const size_t smem = tc_smem_bytes<S>();
    int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)),
                        "tc_7l attribute");
    if (rc) return rc;
    const int64_t n_tiles = (a.total + kTile - 1) / kTile;
    int64_t grid = sm_count();
    const int64_t need = (n_tiles + S - 1) / S;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    // per-slot MMA-group counters are 32-bit
    const int64_t tiles_per_slot = (n_tiles + grid * S - 1) / (grid * S);
    if (tiles_per_slot * a.n_steps * 5 >= (int64_t(1) << 31))
        return set_error(SL_ERR_UNSUPPORTED, "too many path-steps for one launch (%lld tiles per slot x %d steps)",
                         static_cast<long long>(tiles_per_slot), a.n_steps);
    kern<<<static_cast<unsigned>(grid), 32 * (4 * S + 1), smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "tc_7l launch");
}

int g_slots = 4;   // path tiles in flight per CTA (set by sl_tc_set_slots)

}  // namespace

int launch_tc_7l(int m, const SimArgs& a, cudaStream_t st) {
    (void)m;
    if (a.d_in > SL_MAX_DIN_TC) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d > %d", a.d_in, SL_MAX_DIN_TC);
    switch (g_slots) {
        case 2: return launch_s<2>(a, st);
        case 3: return launch_s<3>(a, st);
        case 5: return launch_s<5>(a, st);
        default: return launch_s<4>(a, st);
    }
}

int tc_set_slots(int s) {
    if (s < 2 || s > 5) return set_error(SL_ERR_ARG, "slots=%d outside [2,5]", s);
    g_slots = s;
    return SL_OK;
}

int tc_get_slots() { return g_slots; }

}  // namespace sl

extern "C" {

int sl_tc_set_slots(int slots) { return sl::tc_set_slots(slots); }
int sl_tc_get_slots(void) { return sl::tc_get_slots(); }

}  // extern "C"
