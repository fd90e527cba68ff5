// sl_tc_common.cuh -- building blocks of the tcgen05 (sm_103a) kernels:
// PTX wrappers (mbarrier, tcgen05 MMA/commit/ld/st, fences), shared-memory
// matrix descriptors, BF16 weight staging in 128-byte-swizzled K-major tiles,
// and the per-tile steps of the online sampler (features, MMA issue, normal
// and Lagrange basis, hidden-layer epilogue, output layer).
#pragma once

#include <cuda_bf16.h>
#include <math.h>

#include "sl_internal.cuh"
#include "sl_fastnormal.cuh"

namespace sl {
namespace tc {

constexpr int kTile = 128;                    // paths per slot (MMA M, TMEM lanes)
constexpr int kRowBytes = 128;                // one 128B-swizzle row = 64 BF16
constexpr int kB1Bytes = 64 * kRowBytes;                 // layer 1: 64 rows x (16 of 64) cols
constexpr int kBHBytes = 2 * 64 * kRowBytes;             // hidden: 64 rows x 112 cols
constexpr int kB5Bytes = 2 * 16 * kRowBytes;             // output: 16 rows x 112 cols
constexpr int kBBytes = kB1Bytes + 3 * kBHBytes + kB5Bytes;
constexpr uint64_t kTimeoutNs = 1000000000ull;           // bounded waits: 1 s

// Hidden A row: 112 BF16 values (K) in 56 tensor-memory columns, two per column, the even K
// index in the low half.  Chunk c = 0, 1, 2 covers neurons 16c .. 16c+15: columns 16c .. 16c+7
// hold the hi pairs (neurons 16c+2p, 16c+2p+1 in column 16c+p), columns 16c+8 .. 16c+15 the lo
// pairs.  Column 48 holds the hi pair of neurons 48, 49, column 49 = {1, 0} (the bias unit;
// log2(e) as a hi, lo pair in the base-2 Softplus form),
// column 50 the lo pair of neurons 48, 49, columns 51..55 = 0.  So an epilogue stores each chunk
// with one 16-column store straight from the split's outputs, and columns 49, 51..55 never
// change (tile_init_row writes them once).  The B tiles of the hidden and output layers (and the
// transposed ones of the adjoint) follow the same K order (hid_k_role).
enum KRole { kKNone = 0, kKHi = 1, kKLo = 2, kKBias = 3 };
// The layer-1 A row (the features, K = 16) sits in the slot's last eight columns (120..127,
// after the accumulator 0..63 and the hidden A row 64..119), where no epilogue overwrites it:
// its constant words (dt, theta, the bias unit) are written once per tile, Y's word per step.
constexpr uint32_t kFeatCol = 120;
constexpr uint32_t kBiasWord = 0x00003F80u;              // {1.0, 0} as BF16x2
// The base-2 Softplus form of the sampler (softplus2_fast) carries every pre-activation scaled by
// log2(e): its bias unit is log2(e) as the BF16 pair (hi, lo), both rounded to nearest (their sum
// is log2(e) within 5e-6 of it, relative), against B rows holding the bias at both K indices.
constexpr uint32_t kBiasWordL2 = 0xBB2C3FB9u;
constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLn2 = 0.693147180559945309f;
__host__ __device__ constexpr int hid_k_role(int k, int& n) {
    if (k < 96) {
        n = 16 * (k >> 5) + (k & 15);
        return (k & 16) ? kKLo : kKHi;
    }
    n = 48 + (k & 1);
    return (k == 96 || k == 97) ? kKHi : (k == 100 || k == 101) ? kKLo : (k == 98) ? kKBias : kKNone;
}

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

// One bounded try: the thread may be suspended for up to kSuspendNs waiting for the phase
// (it returns as soon as the phase completes).
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on abort/timeout.
static __device__ __noinline__ bool mbar_wait_slow(uint32_t addr, uint32_t parity, volatile int* abort_flag,
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

// One suspending try inline (it returns when the phase completes, which is the common case);
// the retries, the abort check and the time limit live in the out-of-line slow path.  Every
// instruction counts here: the kernels' time follows their instruction count, and a retry loop
// inline cost 1.3 % of the sampler's launch.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                          unsigned* status) {
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
__device__ __forceinline__ void mma_commit_w(uint32_t mbar) {
    asm volatile(
        "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(mbar)
        : "memory");
}

// The seven K-steps of one layer (K = 112) from tensor-memory A, then the
// commit, in one block with a single elect.sync: A column of step k is
// a_tmem + 8k; B descriptor of step k is db + 2k (k < 4) or db + b_atom1 + 2(k-4).
// The descriptors' start-address field (bits 0..13) stays below 2^14 for every address of
// shared memory, so the K-step offsets are added to the low word alone.
__device__ __forceinline__ void mma7_ta_commit(uint32_t d_tmem, uint32_t a_tmem, uint64_t db,
                                               uint32_t b_atom1, uint32_t idesc, uint32_t mbar) {
    asm volatile(
        "{\n.reg .pred e, pf, pt;\n.reg .b64 b1, b2, b3, b4, b5, b6;\n.reg .b32 a1, a2, a3, a4, a5, a6;\n"
        ".reg .b32 dl, dh, l1, l2, l3, l4, l5, l6;\n"
        "elect.sync _|e, 0xffffffff;\n"
        "setp.ne.b32 pf, %3, %3;\nsetp.eq.b32 pt, %3, %3;\n"
        "mov.b64 {dl, dh}, %2;\n"
        "add.u32 l1, dl, 2;\nadd.u32 l2, dl, 4;\nadd.u32 l3, dl, 6;\n"
        "add.u32 l4, dl, %4;\nadd.u32 l5, l4, 2;\nadd.u32 l6, l4, 4;\n"
        "mov.b64 b1, {l1, dh};\nmov.b64 b2, {l2, dh};\nmov.b64 b3, {l3, dh};\n"
        "mov.b64 b4, {l4, dh};\nmov.b64 b5, {l5, dh};\nmov.b64 b6, {l6, dh};\n"
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
        "r"(a_tmem), "l"(db), "r"(idesc), "r"(b_atom1), "r"(mbar)
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

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t (&v)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(taddr));
}

__device__ __forceinline__ void tmem_st1(uint32_t taddr, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
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
// (lo element, hi element) -> packed BF16x2 truncated toward zero, with ReLU:
// for x > 0 the BF16 value whose bits are the upper half of x's, else 0.
__device__ __forceinline__ uint32_t pack_rz_relu(float lo_elem, float hi_elem) {
    uint32_t d;
    asm("cvt.rz.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
    return d;
}
// (a - ha, b - hb) in one packed FP32x2 subtraction (round to nearest, the same
// result as two scalar subtractions).
__device__ __forceinline__ void sub_f32x2(uint32_t a, uint32_t b, uint32_t ha, uint32_t hb, float& la, float& lb) {
    asm("{\n.reg .b64 x, h, l;\nmov.b64 x, {%2, %3};\nmov.b64 h, {%4, %5};\n"
        "sub.rn.f32x2 l, x, h;\nmov.b64 {%0, %1}, l;\n}"
        : "=f"(la), "=f"(lb)
        : "r"(a), "r"(b), "r"(ha), "r"(hb));
}
// ReLU(x) as BF16 hi + lo for a pair (a, b): hi = truncation (one cvt for the
// pair), unpacked back to FP32 by a shift and a mask; lo = BF16(ReLU(x) - hi),
// where x - hi = x < 0 for negative x, so the ReLU of lo's cvt zeroes it.
__device__ __forceinline__ void split_relu(uint32_t a, uint32_t b, uint32_t& hw, uint32_t& lw) {
    hw = pack_rz_relu(__uint_as_float(a), __uint_as_float(b));
    float la, lb;
    sub_f32x2(a, b, hw << 16, hw & 0xFFFF0000u, la, lb);
    lw = pack_relu(la, lb);
}
// Softplus in base 2.  The tensor-core kernels carry every Softplus pre-activation as
// y = x log2(e) (the features and the bias unit scaled, kBiasWordL2): then
// log2(1 + 2^y) = Softplus(x) log2(e) = max(y, 0) + log2(1 + 2^{-|y|}) takes the exponent and
// logarithm units' own base with no scaling on either side, and a hidden layer whose input and
// output are both in these units needs no change of weights (ln 2 log2(e) = 1).  2^{-|y|} lies in
// (0, 1], so the logarithm's argument lies in (1, 2]; its absolute error stays near 1e-7, far
// below what the BF16 hi + lo split keeps of the result.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float softplus2_fast(float y) {
    return fmaxf(y, 0.0f) + lg2_approx(1.0f + ex2_approx(-fabsf(y)));
}
// The logistic function of the same pre-activation: sigma(x) = 1 / (1 + 2^-y) (0 where 2^-y
// overflows), the derivative of Softplus at x.
__device__ __forceinline__ float sigma2_fast(float y) { return __frcp_rn(1.0f + ex2_approx(-y)); }
__device__ __forceinline__ uint32_t pack_rn(float lo_elem, float hi_elem) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
    return d;
}
// x as BF16 hi + lo for a pair (a, b), no ReLU (cotangents have either sign).
__device__ __forceinline__ void split_rn(uint32_t a, uint32_t b, uint32_t& hw, uint32_t& lw) {
    asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(hw) : "f"(__uint_as_float(b)), "f"(__uint_as_float(a)));
    float la, lb;
    sub_f32x2(a, b, hw << 16, hw & 0xFFFF0000u, la, lb);
    lw = pack_rn(la, lb);
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
//   B1[n][2i] = B1[n][2i+1] = W1[n][i] (i < d_in), B1[n][2 d_in] = B1[n][2 d_in + 1] = b1[n]
//   Bl[n][k] = Wl[n][j] where K index k holds neuron j's hi or lo part, bl[n] at the bias
//   unit's k and at k = 99, 0 elsewhere (the hidden A row's K order, hid_k_role)
// The second bias entries meet the high half of the bias word: 0 in {1.0, 0}, the lo part of
// log2(e) in the base-2 Softplus form's kBiasWordL2.
__device__ inline void stage_weights(unsigned char* sB, const float* __restrict__ P, int d_in, int m) {
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
        else if (k == 2 * d_in || k == 2 * d_in + 1) v = b1[n];
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
            int j = 0;
            const int role = hid_k_role(k, j);
            const bool bias = role == kKBias || k == 99;
            if (role == kKNone && !bias) continue;
            const float v = bias ? bl[n] : Wl[n * W + j];
            *reinterpret_cast<__nv_bfloat16*>(dst + b_elem_off(rows, n, k)) = __float2bfloat16_rn(v);
        }
        p = bl + n_out;
        dst += (l < 3) ? kBHBytes : kB5Bytes;
    }
}

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

// Per-thread state of one path tile (128 paths; this thread owns row `r`).
struct Tile {
    int64_t g;        // path index of this thread's row within the call (its output index)
    int s;            // owning parameter set
    uint32_t q;       // path index within the set (Philox counter)
    bool valid;       // row holds a real path
    float Y;          // state
    float feat[SL_MAX_DIN_TC];
    float4 z4;        // normals of the current block of 4 steps
    float lb[SL_MAX_M];   // Lagrange basis at this step's normal
    uint32_t dph;     // phase of the tile's d_ready barrier
    uint32_t d_tmem;  // accumulator (lane 0 of the tile; A at +64)
    uint32_t taddr;   // accumulator, this warp's lanes
    uint32_t d_bar;   // mbarrier: the tile's MMAs completed
    int bar_id;       // named barrier of the tile's warpgroup
};

// Kernel-wide constants of the issue path.
struct IssueConst {
    uint64_t db0, db1, db2, db3, db4;   // B descriptors of layers 1..5
};

__device__ __forceinline__ void tile_begin(Tile& T, const SimArgs& a, int64_t tile, int r) {
    T.g = tile * kTile + r;
    T.valid = T.g < a.total;
    T.s = 0;
    const int64_t gg = a.first + (T.valid ? T.g : a.total - 1);   // index in the whole batch
    int64_t qq = gg;
    if (a.offsets) {
        T.s = owning_set(a.offsets, a.n_sets, gg);
        qq = gg - __ldg(a.offsets + T.s);
        if (T.valid) T.valid = path_in_set(a.offsets, T.s, gg, a.status);
    }
    T.q = static_cast<uint32_t>(qq);
    const float* th = a.theta + static_cast<int64_t>(T.s) * a.p;
    T.feat[0] = 0.0f;
    T.feat[1] = a.dt;
#pragma unroll
    for (int k = 0; k < SL_MAX_DIN_TC - 2; ++k) T.feat[2 + k] = (k < a.p) ? __ldg(th + k) : 0.0f;
    T.Y = a.Y0 ? __ldg(a.Y0 + T.s) : a.y0_scalar;
    if (a.out_grid && T.valid) a.out_grid[T.g] = T.Y;
    T.z4 = make_float4(0.f, 0.f, 0.f, 0.f);
}

// x as the BF16 pair (hi, lo) of one layer-1 A word: hi = x truncated, lo = BF16(x - hi).
__device__ __forceinline__ uint32_t feature_word(float x) {
    const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFF0000u);
    return pack_rn(hi, x - hi);
}

// Layer-1 A row of a new tile: features [Y, dt, theta] as (hi, lo) BF16 pairs, then the
// constant 1 (columns kFeatCol..kFeatCol+7).  L2: the base-2 Softplus form, features and bias
// unit scaled by log2(e).
template <bool L2 = false>
__device__ __forceinline__ void tile_features_init(Tile& T, const SimArgs& a) {
    T.feat[0] = T.Y;
    constexpr uint32_t bw = L2 ? kBiasWordL2 : kBiasWord;
    uint32_t fw[8];
#pragma unroll
    for (int k = 0; k < SL_MAX_DIN_TC; ++k)
        fw[k] = (k < a.d_in) ? feature_word(L2 ? T.feat[k] * kLog2e : T.feat[k])
                             : ((k == a.d_in) ? bw : 0u);   // the bias unit after the features
    fw[7] = (a.d_in == SL_MAX_DIN_TC) ? bw : 0u;
    tmem_st8(T.taddr + kFeatCol, fw);
    tmem_wait_st();
    tc_fence_before();
}

// Layer-1 A row of the next step: only Y's word changes.
template <bool L2 = false>
__device__ __forceinline__ void tile_features(Tile& T, const SimArgs& a) {
    (void)a;
    tmem_st1(T.taddr + kFeatCol, feature_word(L2 ? T.Y * kLog2e : T.Y));
    tmem_wait_st();
    tc_fence_before();
}

// All four warps agree (named-barrier AND) that the next A is written; the issuing warp
// then issues layer l's MMAs and commits them to the tile's d_ready.
__device__ __forceinline__ bool tile_sync_issue(const Tile& T, const IssueConst& C, int l, bool ok, bool issuer) {
    ok = bar_and(T.bar_id, ok);
    if (ok && issuer) {
        constexpr uint32_t kIdesc64 = idesc_bf16(128, 64), kIdesc16 = idesc_bf16(128, 16);
        tc_fence_after();
        if (l == 0) {
            mma1_ta_commit(T.d_tmem, T.d_tmem + kFeatCol, C.db0, kIdesc64, T.d_bar);
        } else {
            const uint64_t db = (l == 1) ? C.db1 : (l == 2) ? C.db2 : (l == 3) ? C.db3 : C.db4;
            mma7_ta_commit(T.d_tmem, T.d_tmem + 64, db, (l < 4) ? (64 * kRowBytes) >> 4 : (16 * kRowBytes) >> 4,
                           (l < 4) ? kIdesc64 : kIdesc16, T.d_bar);
        }
    }
    return ok;
}

// The hot loop's hand-off: the tile's four warps meet at their named barrier (the next A row is
// written), then the issuing warp issues layer l's MMAs whatever the waits before returned.  A
// failed wait (the abort flag or the time limit) is acted on once per step, at the step's AND
// barrier, so the layers of a step run without per-layer branches (5 % of the sampler's time);
// after a failure the rest of the step runs on stale rows (the status word reports it).
__device__ __forceinline__ void tile_sync_issue_all(const Tile& T, const IssueConst& C, int l, bool issuer) {
    asm volatile("bar.sync %0, 128;" ::"r"(T.bar_id) : "memory");
    if (issuer) {
        constexpr uint32_t kIdesc64 = idesc_bf16(128, 64), kIdesc16 = idesc_bf16(128, 16);
        tc_fence_after();
        if (l == 0) {
            mma1_ta_commit(T.d_tmem, T.d_tmem + kFeatCol, C.db0, kIdesc64, T.d_bar);
        } else {
            const uint64_t db = (l == 1) ? C.db1 : (l == 2) ? C.db2 : (l == 3) ? C.db3 : C.db4;
            mma7_ta_commit(T.d_tmem, T.d_tmem + 64, db, (l < 4) ? (64 * kRowBytes) >> 4 : (16 * kRowBytes) >> 4,
                           (l < 4) ? kIdesc64 : kIdesc16, T.d_bar);
        }
    }
}

// Normal of step i and the Lagrange basis at it (independent of the network).  The normals
// are normal4's Philox words and Box-Muller pairs on the special-function unit (normal4_fast:
// a few 1e-7 of the normal's scale from normal4; 1.3 % of the sampler's time, which follows
// its instruction count); the tensor-core adjoint redraws them the same way.
__device__ __forceinline__ void tile_rng(Tile& T, const SimArgs& a, int i) {
    if ((i & 3) == 0)
        T.z4 = normal4_fast(a.seed, 0u, static_cast<uint32_t>(T.s), T.q, static_cast<uint32_t>(i >> 2));
    lagrange_basis_m(pick4(T.z4, i & 3), a.gh, a.m, T.lb);
}

__device__ __forceinline__ bool tile_wait(Tile& T, volatile int* abort_flag, unsigned* status) {
    bool w = mbar_wait(T.d_bar, T.dph, abort_flag, status);
    T.dph ^= 1u;
    return __all_sync(0xffffffffu, w);
}

// The constant columns of the tile's hidden A row (49 = bias unit, 51..55 = 0), once per
// kernel before the first MMA (the features' wait::st orders it before the issue).
template <bool L2 = false>
__device__ __forceinline__ void tile_init_row(const Tile& T) {
    const uint32_t c[8] = {0u, L2 ? kBiasWordL2 : kBiasWord, 0u, 0u, 0u, 0u, 0u, 0u};
    tmem_st8(T.taddr + 64 + 48, c);
}

// Epilogue frame: the accumulator's columns 0..49 (one FP32 value per neuron) are loaded and
// mapped by pre (all fifty first, so that a long-latency activation has them all in flight),
// f(n, x_n, x_{n+1}, hi_word, lo_word) turns each pair of neurons into a hi and a lo BF16x2
// word, and the words are stored as the next hidden A row (16 columns per chunk).
template <class Pre, class F>
__device__ __forceinline__ void tile_epilogue(const Tile& T, Pre&& pre, F&& f) {
    tc_fence_after();
    uint32_t v0[16], v1[16], v2[16], v3[2];
    tmem_ld16(T.taddr, v0);
    tmem_ld16(T.taddr + 16, v1);
    tmem_ld16(T.taddr + 32, v2);
    tmem_ld2(T.taddr + 48, v3);
    tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v0[k] = pre(v0[k]);
        v1[k] = pre(v1[k]);
        v2[k] = pre(v2[k]);
    }
    v3[0] = pre(v3[0]);
    v3[1] = pre(v3[1]);
    const uint32_t at = T.taddr + 64;
    uint32_t w[16];
#pragma unroll
    for (int p = 0; p < 8; ++p) f(2 * p, v0[2 * p], v0[2 * p + 1], w[p], w[8 + p]);
    tmem_st16(at, w);
#pragma unroll
    for (int p = 0; p < 8; ++p) f(16 + 2 * p, v1[2 * p], v1[2 * p + 1], w[p], w[8 + p]);
    tmem_st16(at + 16, w);
#pragma unroll
    for (int p = 0; p < 8; ++p) f(32 + 2 * p, v2[2 * p], v2[2 * p + 1], w[p], w[8 + p]);
    tmem_st16(at + 32, w);
    uint32_t h, l;
    f(48, v3[0], v3[1], h, l);
    tmem_st1(at + 48, h);
    tmem_st1(at + 50, l);
    tmem_wait_st();
    tc_fence_before();
}

template <class F>
__device__ __forceinline__ void tile_epilogue(const Tile& T, F&& f) {
    tile_epilogue(T, [](uint32_t x) { return x; }, f);
}

// Hidden-layer epilogue: accumulator row -> activation -> BF16 hi + lo -> next A row.
// ReLU is fused into the split's conversions; Softplus is applied to the whole row first, in
// base 2 (L2: the accumulator and the activations scaled by log2(e)).
template <int ACT, bool L2 = false>
__device__ __forceinline__ void tile_hidden_act(const Tile& T) {
    static_assert(ACT != SL_ACT_SOFTPLUS || L2, "the Softplus layers run in base 2");
    if constexpr (ACT == SL_ACT_SOFTPLUS) {
        tile_epilogue(
            T, [](uint32_t x) { return __float_as_uint(softplus2_fast(__uint_as_float(x))); },
            [](int, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) { split_rn(x0, x1, hw, lw); });
    } else {
        tile_epilogue(T, [](int, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) {
            split_relu(x0, x1, hw, lw);
        });
    }
}

__device__ __forceinline__ void tile_hidden(const Tile& T) { tile_hidden_act<SL_ACT_RELU>(T); }

// Output layer: collocation points y_j, then Y_{i+1} = g_m(X) = sum_j y_j ell_j(X)
// (Algorithm I steps 5-6).  L2: the accumulator holds y_j log2(e).
template <bool L2 = false>
__device__ __forceinline__ void tile_out(Tile& T, const SimArgs& a, int i) {
    tc_fence_after();
    uint32_t yv[8];
    tmem_ld8(T.taddr, yv);
    tmem_wait_ld();
    tc_fence_before();
    float acc = 0.0f;
#pragma unroll
    for (int j = SL_MAX_M - 1; j >= 0; --j) acc = fmaf(__uint_as_float(yv[j]), T.lb[j], acc);
    T.Y = L2 ? acc * kLn2 : acc;
    if (a.out_grid && T.valid) {
        const int next = i + 1;
        if (a.grid_k <= 1) a.out_grid[static_cast<int64_t>(next) * a.total + T.g] = T.Y;
        else if (next % a.grid_k == 0) a.out_grid[static_cast<int64_t>(next / a.grid_k) * a.total + T.g] = T.Y;
    }
}

__device__ __forceinline__ void tile_end(const Tile& T, const SimArgs& a) {
    if (!T.valid) return;
    if (a.out_YT) a.out_YT[T.g] = T.Y;
    if (!isfinite(T.Y)) raise_status(a.status, SL_DEV_NONFINITE);
}

}  // namespace tc
}  // namespace sl
