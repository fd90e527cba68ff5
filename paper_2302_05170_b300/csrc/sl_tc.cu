// sl_tc.cu -- BF16 tensor-core (tcgen05) form of the 7L online sampler
// (Algorithm I, steps 2-8) for sm_103a.
//
// The network of Eq. (6.4) is a chain of five GEMMs per coarse step:
//   layer 1:   [128 paths x K=16]  x [K x N=64]      (features, hi+lo split)
//   layers 2-4 [128 paths x K=112] x [K x N=64]      (50 activations hi, 1, lo)
//   layer 5:   [128 paths x K=112] x [K x N=16]      (m <= 8 outputs used)
// A persistent CTA (one per SM) holds S independent path tiles ("slots") of
// 128 paths.  Warpgroup t (warps 4t..4t+3, TMEM lanes 32*(warp%4)..) owns
// slot t: its warp 0 issues the slot's tcgen05.mma (one elected lane), with B
// (weights) in shared memory through 128-byte-swizzled K-major descriptors, A
// (activations) in tensor memory (or shared memory) and FP32 accumulators in
// tensor memory; all four warps are the slot's epilogue: each thread reads the
// accumulator row of its path with
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
// Synchronisation: the four warps of a slot meet at a named barrier (an AND
// reduction, so a failed wait stops all four together) once the next A operand
// is written; warp 0 then issues the layer's MMAs and commits them to the
// slot's mbarrier d_ready, on which all four warps wait.  Every wait is bounded
// (about one second of global time); on expiry the kernel sets SL_DEV_TIMEOUT
// in the status word, the slot stops, every issuer drains its own MMAs
// (bounded) and the tensor memory is released.
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

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
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

// MMA (A and B from shared memory, or A from tensor memory: row i of A in lane
// i, two BF16 values per 32-bit column, K along the columns) and commit.
// Warp-converged forms: every lane of the issuing warp executes the call with
// the same (warp-uniform) operands and one lane, chosen by elect.sync, issues.
// Keeping the control flow converged lets the descriptors stay in uniform
// registers; issuing from a divergent single-lane branch costs ~2.5x per MMA.
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p, e;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %4, 0;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_ta_w(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p, e;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %4, 0;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit_w(uint32_t mbar) {
    asm volatile(
        "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(mbar)
        : "memory");
}

// The seven K-steps of one layer (K = 112) from tensor-memory A, then the
// commit, in one block with a single elect.sync: A column of step k is
// a_tmem + 8k; B descriptor of step k is db + 2k (k < 4) or db + b_atom1 + 2(k-4).
__device__ __forceinline__ void mma7_ta_commit(uint32_t d_tmem, uint32_t a_tmem, uint64_t db,
                                               uint64_t b_atom1, uint32_t idesc, uint32_t mbar) {
    asm volatile(
        "{\n.reg .pred e, pf, pt;\n.reg .b64 b1, b2, b3, b4, b5, b6;\n.reg .b32 a1, a2, a3, a4, a5, a6;\n"
        "elect.sync _|e, 0xffffffff;\n"
        "setp.ne.b32 pf, %3, %3;\nsetp.eq.b32 pt, %3, %3;\n"
        "add.s64 b1, %2, 2;\nadd.s64 b2, %2, 4;\nadd.s64 b3, %2, 6;\n"
        "add.s64 b4, %2, %4;\nadd.s64 b5, b4, 2;\nadd.s64 b6, b4, 4;\n"
        "add.u32 a1, %1, 8;\nadd.u32 a2, %1, 16;\nadd.u32 a3, %1, 24;\n"
        "add.u32 a4, %1, 32;\nadd.u32 a5, %1, 40;\nadd.u32 a6, %1, 48;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pf;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a4], b4, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a5], b5, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a6], b6, %3, pt;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%5];\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(db), "r"(idesc), "l"(b_atom1), "r"(mbar)
        : "memory");
}

// Layer 1 (K = 16) from tensor-memory A, then the commit.
__device__ __forceinline__ void mma1_ta_commit(uint32_t d_tmem, uint32_t a_tmem, uint64_t db, uint32_t idesc,
                                               uint32_t mbar) {
    asm volatile(
        "{\n.reg .pred e, pf;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 pf, %3, %3;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pf;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%4];\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(db), "r"(idesc), "r"(mbar)
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

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
        "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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

// AND of `v` over the 128 threads of named barrier `id` (also a barrier).
__device__ __forceinline__ bool bar_and(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, 128, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(id)
        : "memory");
    return r != 0;
}

// One path tile ("slot") is owned by one warpgroup: warp w (w = 0..3) reads and
// writes TMEM lanes 32w..32w+31, i.e. paths 32w..32w+31 of the tile, and warp 0
// also issues the tile's MMAs (one elected lane) once all four warps have
// written the next A operand (named barrier 1 + slot).  There is no separate
// MMA warp: a hand-off to a shared issuer costs a round trip per layer.
//
// AT = false: the A operand (features / activations) is staged in shared
// memory (128B-swizzled); AT = true: it lives in tensor memory next to the
// slot's accumulator (columns 64..119 of a 128-column slot).
template <int S, bool AT>
__global__ void __launch_bounds__(128 * S, 1) tc_7l_kernel(const SimArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* sB = smem;                                  // weights (1024-aligned)
    unsigned char* sA = smem + kBBytes;                        // S slots x 32 KB (AT = false)
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (AT ? 0 : S * kASlotBytes));   // d_ready[S], drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = warp >> 2, wq = warp & 3;
    const int r = wq * 32 + lane;                              // row = TMEM lane = path in tile
    constexpr int kSlotCols = AT ? 128 : 64;                   // TMEM columns per slot (D, then A)
    constexpr uint32_t kCols = (S * kSlotCols <= 64) ? 64 : (S * kSlotCols <= 128) ? 128
                               : (S * kSlotCols <= 256) ? 256 : 512;
    static_assert(S * kSlotCols <= 512, "tensor memory holds 512 columns");

    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(smem_u32(&bars[k]), 1);   // d_ready: tcgen05.commit
        mbar_init(smem_u32(&bars[S]), S);                               // drain: one commit per slot
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
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
    const int bar_id = 1 + t;
    const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(t * kSlotCols);   // lane 0 of the slot
    const uint32_t taddr = d_tmem + (static_cast<uint32_t>(wq * 32) << 16);
    const uint32_t a_taddr = taddr + 64;
    const uint32_t a_slot = smem_u32(sA) + static_cast<uint32_t>(t * kASlotBytes);
    const uint32_t d_bar = smem_u32(&bars[t]);
    const bool issuer = (wq == 0);
    // descriptors (warp-uniform)
    const uint32_t sB_u = smem_u32(sB);
    constexpr uint32_t kIdesc64 = idesc_bf16(128, 64), kIdesc16 = idesc_bf16(128, 16);
    const uint64_t da = sw128_desc(a_slot);
    const uint64_t db0 = sw128_desc(sB_u);
    const uint64_t db1 = sw128_desc(sB_u + kB1Bytes);
    const uint64_t db2 = sw128_desc(sB_u + kB1Bytes + kBHBytes);
    const uint64_t db3 = sw128_desc(sB_u + kB1Bytes + 2 * kBHBytes);
    const uint64_t db4 = sw128_desc(sB_u + kB1Bytes + 3 * kBHBytes);

    // MMAs of layer l of this slot (warp-converged, one elected lane issues).
    auto issue = [&](int l) {
        tc_fence_after();
        if (AT) {
            if (l == 0) {
                mma1_ta_commit(d_tmem, d_tmem + 64, db0, kIdesc64, d_bar);
            } else {
                const uint64_t db = (l == 1) ? db1 : (l == 2) ? db2 : (l == 3) ? db3 : db4;
                mma7_ta_commit(d_tmem, d_tmem + 64, db, (l < 4) ? (64 * kRowBytes) >> 4 : (16 * kRowBytes) >> 4,
                               (l < 4) ? kIdesc64 : kIdesc16, d_bar);
            }
            return;
        }
        if (l == 0) {
            if (AT) mma_bf16_ta_w(d_tmem, d_tmem + 64, db0, kIdesc64, 0u);
            else mma_bf16_w(d_tmem, da, db0, kIdesc64, 0u);
        } else {
            const uint64_t db = (l == 1) ? db1 : (l == 2) ? db2 : (l == 3) ? db3 : db4;
            const uint32_t b_atom1 = (l < 4) ? (64 * kRowBytes) >> 4 : (16 * kRowBytes) >> 4;
            const uint32_t idesc = (l < 4) ? kIdesc64 : kIdesc16;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                // K steps 0-3 in the first 64-column atom, 4-6 in the second; descriptor start
                // addresses are in 16-byte units (bits 0-13)
                const uint64_t bk = db + ((k < 4) ? 2u * k : b_atom1 + 2u * (k - 4));
                if (AT) {
                    mma_bf16_ta_w(d_tmem, d_tmem + 64 + 8 * k, bk, idesc, k > 0 ? 1u : 0u);
                } else {
                    const uint64_t ak = da + ((k < 4) ? 2u * k : (kAAtomBytes >> 4) + 2u * (k - 4));
                    mma_bf16_w(d_tmem, ak, bk, idesc, k > 0 ? 1u : 0u);
                }
            }
        }
        mma_commit_w(d_bar);
    };

    uint32_t dph = 0;
    bool ok = true;
    const float dt = a.dt;
    for (int64_t tile = static_cast<int64_t>(blockIdx.x) * S + t; tile < n_tiles; tile += tile_stride) {
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

        for (int i = 0; i < a.n_steps; ++i) {
            // ---- features [Y, dt, theta] as (hi, lo) BF16 pairs + constant 1 (layer-1 A)
            if (ok) {
                feat[0] = Y;
                uint32_t fw[8];
#pragma unroll
                for (int k = 0; k < SL_MAX_DIN_TC; ++k) {
                    const float hi = __uint_as_float(__float_as_uint(feat[k]) & 0xFFFF0000u);
                    const uint32_t wv = pack_rn(hi, feat[k] - hi);
                    fw[k] = (k < a.d_in) ? wv : ((k == a.d_in) ? 0x00003F80u : 0u);   // 1.0 after the features
                }
                fw[7] = (a.d_in == SL_MAX_DIN_TC) ? 0x00003F80u : 0u;
                if (AT) {
                    tmem_st8(a_taddr, fw);
                    tmem_wait_st();
                } else {
                    st_shared_v4(a_slot + sw128_chunk(r, 0), fw[0], fw[1], fw[2], fw[3]);
                    st_shared_v4(a_slot + sw128_chunk(r, 1), fw[4], fw[5], fw[6], fw[7]);
                    fence_proxy_async_smem();
                }
                tc_fence_before();
            }
            ok = bar_and(bar_id, ok);          // slot-uniform from here
            if (!ok) break;
            if (issuer) issue(0);
            // While layer 1 runs: this step's normal and the Lagrange basis at it
            // (independent of the network's output).
            if ((i & 3) == 0)
                z4 = normal4(a.seed, 0u, static_cast<uint32_t>(ts.s), ts.q, static_cast<uint32_t>(i >> 2));
            float lb[SL_MAX_M];
            lagrange_basis_m(pick4(z4, i & 3), a.gh, a.m, lb);

            // ---- hidden layers: accumulator -> ReLU -> hi/lo BF16 -> next A
            // (unrolled: each layer's MMA issue is specialised at compile time)
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
                bool w = mbar_wait(d_bar, dph, abort_flag, a.status);
                dph ^= 1u;
                w = __all_sync(0xffffffffu, w);
                if (w) {
                    tc_fence_after();
                    // Row layout of the next A (BF16 words): hi 0..24 (columns 0..49),
                    // word 25 = {1.0, 0} (bias unit), 26..27 = 0, lo 28..52, 53..55 = 0.
                    // columns 0..31 of the accumulator -> hi words 0..15, lo words 28..43
                    // all three loads in flight before one wait
                    uint32_t v[32], v2[16], u[8];
                    tmem_ld32(taddr, v);
                    tmem_ld16(taddr + 32, v2);
                    tmem_ld8(taddr + 48, u);
                    tmem_wait_ld();
                    uint32_t hw[16], lw[16];
                    {
#pragma unroll
                        for (int i2 = 0; i2 < 16; ++i2) {
                            const float ha = __uint_as_float(v[2 * i2] & 0xFFFF0000u);
                            const float hb = __uint_as_float(v[2 * i2 + 1] & 0xFFFF0000u);
                            hw[i2] = pack_relu(ha, hb);
                            lw[i2] = pack_relu(__uint_as_float(v[2 * i2]) - ha, __uint_as_float(v[2 * i2 + 1]) - hb);
                        }
                    }
                    if (AT) {
                        tmem_st16(a_taddr, hw);
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            st_shared_v4(a_slot + sw128_chunk(r, c), hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        st_shared_v4(a_slot + sw128_chunk(r, 7), lw[0], lw[1], lw[2], lw[3]);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, c), lw[4 + 4 * c], lw[5 + 4 * c],
                                         lw[6 + 4 * c], lw[7 + 4 * c]);
                    }
                    // columns 32..49 -> hi words 16..24, lo words 44..52
                    {
                        uint32_t h9[9], l9[9];
#pragma unroll
                        for (int i2 = 0; i2 < 9; ++i2) {
                            const uint32_t ua = (i2 < 8) ? v2[2 * i2] : u[0];
                            const uint32_t ub = (i2 < 8) ? v2[2 * i2 + 1] : u[1];
                            const float ha = __uint_as_float(ua & 0xFFFF0000u);
                            const float hb = __uint_as_float(ub & 0xFFFF0000u);
                            h9[i2] = pack_relu(ha, hb);
                            l9[i2] = pack_relu(__uint_as_float(ua) - ha, __uint_as_float(ub) - hb);
                        }
                        if (AT) {
                            const uint32_t gb[16] = {h9[0], h9[1], h9[2], h9[3], h9[4], h9[5], h9[6], h9[7],
                                                     h9[8], 0x00003F80u, 0u, 0u, lw[0], lw[1], lw[2], lw[3]};
                            const uint32_t gc[16] = {lw[4], lw[5], lw[6], lw[7], lw[8], lw[9], lw[10], lw[11],
                                                     lw[12], lw[13], lw[14], lw[15], l9[0], l9[1], l9[2], l9[3]};
                            const uint32_t gd[8] = {l9[4], l9[5], l9[6], l9[7], l9[8], 0u, 0u, 0u};
                            tmem_st16(a_taddr + 16, gb);
                            tmem_st16(a_taddr + 32, gc);
                            tmem_st8(a_taddr + 48, gd);
                        } else {
                            st_shared_v4(a_slot + sw128_chunk(r, 4), h9[0], h9[1], h9[2], h9[3]);
                            st_shared_v4(a_slot + sw128_chunk(r, 5), h9[4], h9[5], h9[6], h9[7]);
                            st_shared_v4(a_slot + sw128_chunk(r, 6), h9[8], 0x00003F80u, 0u, 0u);
                            st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 3), l9[0], l9[1], l9[2], l9[3]);
                            st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 4), l9[4], l9[5], l9[6], l9[7]);
                            st_shared_v4(a_slot + kAAtomBytes + sw128_chunk(r, 5), l9[8], 0u, 0u, 0u);
                        }
                    }
                    if (AT) tmem_wait_st();
                    else fence_proxy_async_smem();
                    tc_fence_before();
                }
                ok = bar_and(bar_id, w);
                if (!ok) break;
                if (issuer) issue(l);
            }
            if (!ok) break;
            // ---- output layer: collocation points y_0..y_{m-1}
            bool w = mbar_wait(d_bar, dph, abort_flag, a.status);
            dph ^= 1u;
            w = __all_sync(0xffffffffu, w);
            ok = w;     // combined across the slot at the next barrier
            if (w) {
                tc_fence_after();
                uint32_t yv[8];
                tmem_ld8(taddr, yv);
                tmem_wait_ld();
                tc_fence_before();
                // ---- the 7L map g_m (Algorithm I steps 5-6): Y = sum_j y_j ell_j(X)
                float acc = 0.0f;
#pragma unroll
                for (int j = SL_MAX_M - 1; j >= 0; --j) acc = fmaf(__uint_as_float(yv[j]), lb[j], acc);
                Y = acc;
                if (a.out_grid && ts.valid) a.out_grid[static_cast<int64_t>(i + 1) * a.total + ts.g] = Y;
            }
        }
        if (!ok) break;
        if (ts.valid) {
            if (a.out_YT) a.out_YT[ts.g] = Y;
            if (!isfinite(Y)) raise_status(a.status, SL_DEV_NONFINITE);
        }
    }
    // Drain: each slot's issuer commits once more; the allocating warp waits for all
    // (bounded) before releasing tensor memory.
    if (issuer) mma_commit_w(smem_u32(&bars[S]));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        if (lane == 0) {
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(smem_u32(&bars[S]), 0)) {
                if (global_ns() - t0 > kTimeoutNs) {
                    raise_status(a.status, SL_DEV_TIMEOUT);
                    break;
                }
            }
        }
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kCols)
                     : "memory");
    }
}

template <int S, bool AT>
size_t tc_smem_bytes() {
    return 1024 + kBBytes + (AT ? 0 : static_cast<size_t>(S) * kASlotBytes) + (S + 1) * 8 + 16;
}

template <int S, bool AT>
int launch_s(const SimArgs& a, cudaStream_t st) {
    auto kern = tc_7l_kernel<S, AT>;
    const size_t smem = tc_smem_bytes<S, AT>();
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
    kern<<<static_cast<unsigned>(grid), 128 * S, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "tc_7l launch");
}

int g_slots = 4;   // path tiles in flight per CTA (set by sl_tc_set_slots)
int g_a_tmem = 1;  // 1: A operand in tensor memory (slots <= 4)

}  // namespace

int launch_tc_7l(int m, const SimArgs& a, cudaStream_t st) {
    (void)m;
    if (a.d_in > SL_MAX_DIN_TC) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d > %d", a.d_in, SL_MAX_DIN_TC);
    if (g_a_tmem && g_slots <= 4) {
        switch (g_slots) {
            case 2: return launch_s<2, true>(a, st);
            case 3: return launch_s<3, true>(a, st);
            default: return launch_s<4, true>(a, st);
        }
    }
    switch (g_slots) {
        case 2: return launch_s<2, false>(a, st);
        case 3: return launch_s<3, false>(a, st);
        case 5: return launch_s<5, false>(a, st);
        default: return launch_s<4, false>(a, st);
    }
}

int tc_set_slots(int s) {
    if (s < 2 || s > 5) return set_error(SL_ERR_ARG, "slots=%d outside [2,5]", s);
    g_slots = s;
    return SL_OK;
}

int tc_get_slots() { return g_slots; }

int tc_set_a_tmem(int on) {
    g_a_tmem = on ? 1 : 0;
    return SL_OK;
}

}  // namespace sl

extern "C" {

int sl_tc_set_slots(int slots) { return sl::tc_set_slots(slots); }
int sl_tc_get_slots(void) { return sl::tc_get_slots(); }
int sl_tc_set_a_operand(int in_tensor_memory) { return sl::tc_set_a_tmem(in_tensor_memory); }

}  // extern "C"
