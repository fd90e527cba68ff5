// sl_tc_adjoint.cu -- BF16 tensor-core (tcgen05) form of the pathwise adjoint:
// sensitivities of E[max(Y_T - K, 0)] with respect to Y0 and theta through
// g_m and the network, with Y_i checkpointed every k steps.
//
// Three launches:
//  1. forward: the BF16 sampler itself, with its path grid thinned to the
//     checkpoint rows Y_0, Y_k, Y_2k, .. (the same paths as seven_league_simulate);
//  2. itm_compact_kernel: f(Y_T) for every path, zero sensitivities for the
//     out-of-the-money paths (Y_T <= K), and the list of in-the-money paths;
//  3. tc_adjoint_reverse_kernel over that list only, 128 listed paths per tile
//     (one warpgroup, one of its warps issues the MMAs), lambda = 1 at Y_T; per segment
//     (last first), in blocks of at most 8 steps (last first):
//     a. a forward pass over the block from its first state (the checkpoint,
//        or for a segment longer than 8 steps a state recomputed first) that
//        records the ReLU pattern of every hidden layer at every step as bits
//        in shared memory (pre-activation > 0);
//     then per step i of the block, from its last to its first:
//     b. backward chain with c_j = lambda * ell_j(X_i) (the cotangent of the
//        collocation points: d Y_{i+1} / d y_j = ell_j(X_i)):
//        dh4 = W5^T c, dz_l = dh_l masked, dh_{l-1} = W_l^T dz_l, ...,
//        d/df = W1^T dz1, as tcgen05 MMAs against transposed BF16 weight
//        tiles; the cotangents are split into BF16 hi + lo like the forward
//        activations (A operand in tensor memory);
//     c. lambda <- d/dY_i, g_theta += d/dtheta.
//  Per-set FP64 means come from the shared deterministic reduction.
//
// Softplus networks have no bit pattern to record: dz_l = dh_l * sigma(z_l) needs the
// pre-activation itself.  Per step (last first) and per layer l = 4..1 of the backward
// chain, each thread keeps dh_l of its row in registers while the tile recomputes the
// step's forward up to z_l in the accumulator; sigma(z_l) = 1 / (1 + e^{-z_l}) is then
// taken in FP32 from the accumulator, so nothing is stored and nothing is rounded beyond
// the ReLU form.  Cost per step: 10 forward and 5 backward layer groups (ReLU: 4 + 5), plus
// the segment's states recomputed from its checkpoint.
//
// Tensor memory per tile: 128 columns -- accumulator 0..63, A operand 64..119.
// Shared memory per tile (ReLU): the block's ReLU patterns, 8 steps x 4 layers x 2 words
// per path (32 KB).
#include "sl_tc_common.cuh"

namespace sl {
namespace {

using namespace tc;

constexpr int kMaxCkptK = 32;
constexpr int kB5TBytes = 64 * kRowBytes;          // W5^T: 64 rows (in-neurons) x K = 16 (m hi, m lo)
constexpr int kBHTBytes = 2 * 64 * kRowBytes;      // W_l^T: 64 rows x K = 112
constexpr int kB1TBytes = 2 * 16 * kRowBytes;      // W1^T: 16 rows (features) x K = 112
constexpr int kBTBytes = kB5TBytes + 3 * kBHTBytes + kB1TBytes;

struct AdjTC {
    SimArgs s;
    float K;
    int k;                  // checkpoint interval
    int n_ckpt;             // checkpoints Y_0, Y_k, .., Y_(n_ckpt-1)k
    const float* ckpt;      // [n_ckpt (+1)][total]
    float* pv;              // [(2+p)][total]
    const uint32_t* list;   // in-the-money paths
    const unsigned* count;  // their number
};

// Transposed weights for the backward chain (BF16, 128B-swizzled, K-major):
//   B5T[n][j] = B5T[n][8 + j] = W5[j][n]              (n < 50, j < m)
//   BlT[n][k] = W_l[j][n]   (l = 4, 3, 2; n < 50)     k: the hi or lo part of neuron j
//   B1T[n][k] = W1[j][n]    (n < d_in)                (the hidden A row's K order; 0 at
//                                                      the bias unit and the padding)
__device__ void stage_weights_T(unsigned char* sBT, const float* __restrict__ P, int d_in, int m) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int W = SL_WIDTH;
    for (int i = tid; i < kBTBytes / 2; i += nt) reinterpret_cast<uint16_t*>(sBT)[i] = 0;
    __syncthreads();
    // offsets of W_l in the flat parameter array
    const int o1 = 0;
    const int o2 = W * d_in + W;
    const int o3 = o2 + W * W + W;
    const int o4 = o3 + W * W + W;
    const int o5 = o4 + W * W + W;
    unsigned char* d5 = sBT;
    for (int i = tid; i < W * 16; i += nt) {
        const int n = i / 16, k = i % 16, j = k & 7;
        if (j >= m) continue;
        *reinterpret_cast<__nv_bfloat16*>(d5 + b_elem_off(64, n, k)) = __float2bfloat16_rn(P[o5 + j * W + n]);
    }
    const int offs[3] = {o4, o3, o2};   // W4^T, W3^T, W2^T
    for (int q = 0; q < 3; ++q) {
        unsigned char* d = sBT + kB5TBytes + q * kBHTBytes;
        for (int i = tid; i < W * 112; i += nt) {
            const int n = i / 112, k = i % 112;
            int kk = 0;
            const int role = hid_k_role(k, kk);
            if (role != kKHi && role != kKLo) continue;
            *reinterpret_cast<__nv_bfloat16*>(d + b_elem_off(64, n, k)) = __float2bfloat16_rn(P[offs[q] + kk * W + n]);
        }
    }
    unsigned char* d1 = sBT + kB5TBytes + 3 * kBHTBytes;
    for (int i = tid; i < d_in * 112; i += nt) {
        const int n = i / 112, k = i % 112;
        int kk = 0;
        const int role = hid_k_role(k, kk);
        if (role != kKHi && role != kKLo) continue;
        *reinterpret_cast<__nv_bfloat16*>(d1 + b_elem_off(16, n, k)) = __float2bfloat16_rn(P[o1 + kk * d_in + n]);
    }
}

struct IssueConstT {
    uint64_t db5, db4, db3, db2, db1;   // transposed B descriptors, in chain order
};

// Backward MMAs of chain step lt (0: W5^T, 1: W4^T, 2: W3^T, 3: W2^T, 4: W1^T), issued after the
// warpgroup's named barrier whatever the waits before returned (as tile_sync_issue_all).
__device__ __forceinline__ void tile_sync_issue_T_all(const Tile& T, const IssueConstT& C, int lt, bool issuer) {
    asm volatile("bar.sync %0, 128;" ::"r"(T.bar_id) : "memory");
    if (issuer) {
        constexpr uint32_t kIdesc64 = idesc_bf16(128, 64), kIdesc16 = idesc_bf16(128, 16);
        tc_fence_after();
        if (lt == 0) {
            mma1_ta_commit(T.d_tmem, T.d_tmem + 64, C.db5, kIdesc64, T.d_bar);
        } else {
            const uint64_t db = (lt == 1) ? C.db4 : (lt == 2) ? C.db3 : (lt == 3) ? C.db2 : C.db1;
            mma7_ta_commit(T.d_tmem, T.d_tmem + 64, db, (lt < 4) ? (64 * kRowBytes) >> 4 : (16 * kRowBytes) >> 4,
                           (lt < 4) ? kIdesc64 : kIdesc16, T.d_bar);
        }
    }
}

// Steps of a segment whose ReLU patterns are recorded at once (per tile: 8 steps x 4
// hidden layers x 2 words x 128 rows in shared memory).
constexpr int kMaskSteps = 8;
constexpr int kMaskWordsPerTile = kMaskSteps * 4 * 2 * kTile;

// ReLU pattern of a hidden layer as 64 bits (two words): the pair of neurons (n, n+1),
// n = 32h + 2p + 16c' (h = word, c' = 0 or 1 the chunk inside the word, p = 0..7; the last
// pair, neurons 48 and 49, is p = 8 of word 1), owns bits q = p + 8c' (neuron n) and 16 + q
// (neuron n+1) of word h.
__device__ __forceinline__ constexpr int relu_bit(int n) { return ((n & 15) >> 1) + 8 * ((n >> 4) & 1); }

// Hidden epilogue of a recorded forward step: the sampler's epilogue (ReLU, BF16 hi + lo,
// next A row) plus the layer's ReLU pattern (relu_bit), stored to mrow[0] and mrow[kTile].
// A neuron's bit is "its truncated BF16 hi part is nonzero", i.e. z >= 2^-126: the pair's
// hi word plus 0x7FFF7FFF carries each nonzero half into that half's top bit (halves are at
// most 0x7F80 after the ReLU, so nothing carries across), and one shift and one masked OR
// move the two bits into place.
__device__ __forceinline__ void tile_hidden_rec(const Tile& T, uint32_t* mrow) {
    uint32_t m0 = 0u, m1 = 0u;
    tile_epilogue(T, [&](int n, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) {
        split_relu(x0, x1, hw, lw);
        const int q = relu_bit(n);
        const uint32_t t = (hw + 0x7FFF7FFFu) >> (15 - q);
        const uint32_t sel = (1u << q) | (1u << (16 + q));
        if (n < 32) m0 |= t & sel;
        else m1 |= t & sel;
    });
    mrow[0] = m0;
    mrow[kTile] = m1;
}

// Backward epilogue: dh (accumulator columns 0..49) masked by the recorded ReLU pattern
// (m0: neurons 0..31, m1: neurons 32..49, bits as relu_bit), split into BF16 hi + lo (no
// ReLU: cotangents have either sign) and written as the next A row (the hidden A row's
// layout; the bias unit meets a zero row of the transposed weights).
__device__ __forceinline__ void tile_backward_bits(const Tile& T, uint32_t m0, uint32_t m1) {
    tile_epilogue(T, [&](int n, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) {
        const uint32_t w = (n < 32) ? m0 : m1;
        const int q = relu_bit(n);
        split_rn((w & (1u << q)) ? x0 : 0u, (w & (1u << (16 + q))) ? x1 : 0u, hw, lw);
    });
}

// The accumulator row's columns 0..49 as FP32 values (the cotangent dh of a layer).
__device__ __forceinline__ void tile_acc50(const Tile& T, float (&d)[SL_WIDTH]) {
    tc_fence_after();
    uint32_t v[32], v2[16], u[8];
    tmem_ld32(T.taddr, v);
    tmem_ld16(T.taddr + 32, v2);
    tmem_ld8(T.taddr + 48, u);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = __uint_as_float(v[j]);
#pragma unroll
    for (int j = 0; j < 16; ++j) d[32 + j] = __uint_as_float(v2[j]);
    d[48] = __uint_as_float(u[0]);
    d[49] = __uint_as_float(u[1]);
    tc_fence_before();
}

// Backward epilogue of a Softplus layer: the accumulator holds the layer's pre-activation in
// the sampler's base-2 units, y = z log2(e) (just recomputed); dz = dh * sigma(z),
// sigma(z) = 1 / (1 + 2^{-y}) (sigma2_fast), split into BF16 hi + lo and written as the next A
// row (layout of tile_backward_bits).  The cotangents themselves are in natural units: the
// backward chain runs through the unscaled transposed weights.
__device__ __forceinline__ void tile_backward_sp(const Tile& T, const float (&dh)[SL_WIDTH]) {
    auto dz = [&](int j, uint32_t yb) { return __float_as_uint(dh[j] * sigma2_fast(__uint_as_float(yb))); };
    tile_epilogue(T, [&](int n, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) {
        split_rn(dz(n, x0), dz(n + 1, x1), hw, lw);
    });
}

// Softplus layers whose sigma(z) = 1 / (1 + e^{-z}) the backward chain takes from tensor memory
// instead of recomputing the step's forward pass: the tile's sigma columns (FP32, one column per
// neuron) at kSig4 (layer 4) and kSig3 (layer 3) past its accumulator.  Layers 2 and 1 are still
// recomputed (their sigma would need 100 more columns per tile).
constexpr uint32_t kSig4 = 256, kSig3 = 256 + 64;

__device__ __forceinline__ uint32_t sigma_bits(uint32_t yb) {
    return __float_as_uint(sigma2_fast(__uint_as_float(yb)));
}

// The accumulator row (y = z log2(e) of a Softplus layer): sigma(z) into the sigma columns at
// scol and, with kAct, Softplus(z) log2(e) split into BF16 hi + lo as the next A row
// (tile_hidden_act's output in base 2).
template <bool kAct>
__device__ __forceinline__ void tile_forward_sigma(const Tile& T, uint32_t scol) {
    tc_fence_after();
    uint32_t v0[16], v1[16], v2[16], v3[2];
    tmem_ld16(T.taddr, v0);
    tmem_ld16(T.taddr + 16, v1);
    tmem_ld16(T.taddr + 32, v2);
    tmem_ld2(T.taddr + 48, v3);
    tmem_wait_ld();
    uint32_t s[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = sigma_bits(v0[k]);
    tmem_st16(T.taddr + scol, s);
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = sigma_bits(v1[k]);
    tmem_st16(T.taddr + scol + 16, s);
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = sigma_bits(v2[k]);
    tmem_st16(T.taddr + scol + 32, s);
    tmem_st1(T.taddr + scol + 48, sigma_bits(v3[0]));
    tmem_st1(T.taddr + scol + 49, sigma_bits(v3[1]));
    if constexpr (kAct) {
        auto sp = [](uint32_t x) { return __float_as_uint(softplus2_fast(__uint_as_float(x))); };
        const uint32_t at = T.taddr + 64;
        uint32_t w[16];
#pragma unroll
        for (int p = 0; p < 8; ++p) split_rn(sp(v0[2 * p]), sp(v0[2 * p + 1]), w[p], w[8 + p]);
        tmem_st16(at, w);
#pragma unroll
        for (int p = 0; p < 8; ++p) split_rn(sp(v1[2 * p]), sp(v1[2 * p + 1]), w[p], w[8 + p]);
        tmem_st16(at + 16, w);
#pragma unroll
        for (int p = 0; p < 8; ++p) split_rn(sp(v2[2 * p]), sp(v2[2 * p + 1]), w[p], w[8 + p]);
        tmem_st16(at + 32, w);
        uint32_t h, l;
        split_rn(sp(v3[0]), sp(v3[1]), h, l);
        tmem_st1(at + 48, h);
        tmem_st1(at + 50, l);
    }
    tmem_wait_st();
    tc_fence_before();
}

// Backward epilogue of a Softplus layer whose sigma(z) is in the sigma columns at scol: the
// accumulator holds dh; dz = dh * sigma(z), split into BF16 hi + lo as the next A row (the
// values of tile_backward_sp, without the forward recompute).
__device__ __forceinline__ void tile_backward_sig(const Tile& T, uint32_t scol) {
    uint32_t s0[16], s1[16], s2[16], s3[2];
    tc_fence_after();
    tmem_ld16(T.taddr + scol, s0);
    tmem_ld16(T.taddr + scol + 16, s1);
    tmem_ld16(T.taddr + scol + 32, s2);
    tmem_ld2(T.taddr + scol + 48, s3);
    auto dz = [&](uint32_t db, uint32_t sb) { return __float_as_uint(__uint_as_float(db) * __uint_as_float(sb)); };
    tile_epilogue(T, [&](int n, uint32_t x0, uint32_t x1, uint32_t& hw, uint32_t& lw) {
        const uint32_t sa = (n < 16) ? s0[n] : (n < 32) ? s1[n - 16] : (n < 48) ? s2[n - 32] : s3[n - 48];
        const uint32_t sb = (n + 1 < 16) ? s0[n + 1] : (n + 1 < 32) ? s1[n - 15] : (n + 1 < 48) ? s2[n - 31] : s3[n - 47];
        split_rn(dz(x0, sa), dz(x1, sb), hw, lw);
    });
}

// Cotangent of the collocation points, c_j = lambda * ell_j(X), as the A row
// of W5^T: words 0..3 = hi pairs (c_0, c_1) .. (c_6, c_7), words 4..7 = lo pairs.
__device__ __forceinline__ void tile_cotangent(const Tile& T, float lam) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        split_rn(__float_as_uint(lam * T.lb[2 * q]), __float_as_uint(lam * T.lb[2 * q + 1]), w[q], w[4 + q]);
    }
    tmem_st8(T.taddr + 64, w);
    tmem_wait_st();
    tc_fence_before();
}

// Normal of step i and the Lagrange basis at it, for any order of steps: the
// block of four normals is redrawn whenever step i falls in another block, with
// the forward sweep's generator (normal4_fast, as the sampler's tile_rng).
__device__ __forceinline__ void tile_rng_any(Tile& T, const SimArgs& a, int i, int& blk) {
    if ((i >> 2) != blk) {
        blk = i >> 2;
        T.z4 = normal4_fast(a.seed, 0u, static_cast<uint32_t>(T.s), T.q, static_cast<uint32_t>(blk));
    }
    lagrange_basis_m(pick4(T.z4, i & 3), a.gh, a.m, T.lb);
}

// f(Y_T) for every path; zero sensitivities for the out-of-the-money paths;
// the in-the-money paths (Y_T > K, where f'(Y_T) = 1) appended to `list`
// (warp-aggregated; the order does not matter: every path's result depends on
// its own row only).
__global__ void itm_compact_kernel(const float* __restrict__ yt, int64_t total, float K, int p,
                                   float* __restrict__ pv, uint32_t* __restrict__ list, unsigned* count) {
    const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    bool itm = false;
    if (g < total) {
        const float y = yt[g];
        pv[g] = fmaxf(y - K, 0.0f);
        itm = y > K;
        if (!itm)
            for (int q = 0; q < 1 + p; ++q) pv[static_cast<int64_t>(1 + q) * total + g] = 0.0f;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, itm);
    if (mask) {
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(count, static_cast<unsigned>(__popc(mask)));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (itm) list[base + __popc(mask & ((1u << lane) - 1u))] = static_cast<uint32_t>(g);
    }
}

// Row r of a reverse tile: listed path `g` (or an idle row past the end of the list).
__device__ __forceinline__ void tile_begin_listed(Tile& T, const SimArgs& a, int64_t g, bool valid) {
    T.g = g;
    T.valid = valid;
    T.s = owning_set(a.offsets, a.n_sets, g);
    T.q = static_cast<uint32_t>(g - __ldg(a.offsets + T.s));
    const float* th = a.theta + static_cast<int64_t>(T.s) * a.p;
    T.feat[0] = 0.0f;
    T.feat[1] = a.dt;
#pragma unroll
    for (int k = 0; k < SL_MAX_DIN_TC - 2; ++k) T.feat[2 + k] = (k < a.p) ? __ldg(th + k) : 0.0f;
    T.Y = 0.0f;
    T.z4 = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int ACT>
constexpr int mask_words_per_tile() { return ACT == SL_ACT_RELU ? kMaskWordsPerTile : 0; }

template <int WG, int ACT>
__global__ void __launch_bounds__(128 * WG, 1) tc_adjoint_reverse_kernel(const AdjTC A) {
    constexpr int S = WG;
    // Softplus: two tiles, and past them each tile's sigma columns (kSig4, kSig3)
    constexpr uint32_t kCols = (ACT == SL_ACT_SOFTPLUS) ? 512 : (S * 128 <= 128) ? 128 : (S * 128 <= 256) ? 256 : 512;
    static_assert(S * 128 <= 512 && (ACT != SL_ACT_SOFTPLUS || S <= 2), "tensor memory holds 512 columns");
    constexpr bool L2 = (ACT == SL_ACT_SOFTPLUS);   // the forward recompute in base 2, as the sampler
    const SimArgs& a = A.s;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* sB = smem;
    unsigned char* sBT = smem + kBBytes;
    uint32_t* masks = reinterpret_cast<uint32_t*>(sBT + kBTBytes);     // [S][kMaskSteps][4][2][128]
    uint64_t* bars = reinterpret_cast<uint64_t*>(masks + S * mask_words_per_tile<ACT>());   // d_ready[S], drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wg = warp >> 2, wq = warp & 3;
    const int r = wq * 32 + lane;
    const bool issuer = (wq == (wg & 3));   // one issuing warp per SM sub-partition (as the sampler)

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) mbar_init(smem_u32(&bars[q]), 1);
        mbar_init(smem_u32(&bars[S]), WG);
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
    stage_weights_T(sBT, a.params, a.d_in, a.m);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    IssueConst C;
    const uint32_t sB_u = smem_u32(sB);
    C.db0 = sw128_desc(sB_u);
    C.db1 = sw128_desc(sB_u + kB1Bytes);
    C.db2 = sw128_desc(sB_u + kB1Bytes + kBHBytes);
    C.db3 = sw128_desc(sB_u + kB1Bytes + 2 * kBHBytes);
    C.db4 = sw128_desc(sB_u + kB1Bytes + 3 * kBHBytes);
    IssueConstT CT;
    const uint32_t sBT_u = smem_u32(sBT);
    CT.db5 = sw128_desc(sBT_u);
    CT.db4 = sw128_desc(sBT_u + kB5TBytes);
    CT.db3 = sw128_desc(sBT_u + kB5TBytes + kBHTBytes);
    CT.db2 = sw128_desc(sBT_u + kB5TBytes + 2 * kBHTBytes);
    CT.db1 = sw128_desc(sBT_u + kB5TBytes + 3 * kBHTBytes);

    Tile T;
    T.d_tmem = tmem_base + static_cast<uint32_t>(wg * 128);
    T.taddr = T.d_tmem + (static_cast<uint32_t>(wq * 32) << 16);
    T.d_bar = smem_u32(&bars[wg]);
    T.bar_id = 1 + wg;
    T.dph = 0;
    tile_init_row<L2>(T);
    uint32_t* tmask = masks + wg * mask_words_per_tile<ACT>() + r;   // word (step, layer l, half h) at ((step*4 + l-1)*2 + h)*128

    int64_t n_list = static_cast<int64_t>(*A.count);
    if (kChecked && n_list > a.total) {            // the list holds at most one entry per path
        raise_status(a.status, SL_DEV_INDEX);
        n_list = a.total;
    }
    const int64_t n_tiles = (n_list + kTile - 1) / kTile;
    const int64_t tile_stride = static_cast<int64_t>(gridDim.x) * S;
    const int p = a.p;
    bool ok = true;
    for (int64_t tile = static_cast<int64_t>(blockIdx.x) * S + wg; tile < n_tiles; tile += tile_stride) {
        const int64_t li = tile * kTile + r;
        bool valid = li < n_list;
        int64_t g = A.list[valid ? li : n_list - 1];
        if (kChecked && g >= a.total) {                // a listed path past the path count
            raise_status(a.status, SL_DEV_INDEX);
            g = 0;
            valid = false;
        }
        tile_begin_listed(T, a, g, valid);
        tile_features_init<L2>(T, a);
        if (T.valid) T.valid = path_in_set(a.offsets, T.s, g, a.status);
        int blk = -1;
        float lam = valid ? 1.0f : 0.0f;
        float gth[SL_MAX_DIN_TC - 2];
#pragma unroll
        for (int q = 0; q < SL_MAX_DIN_TC - 2; ++q) gth[q] = 0.0f;
        for (int c = A.n_ckpt - 1; ok && c >= 0; --c) {
            const int i0 = c * A.k;
            const int i1 = min(i0 + A.k, a.n_steps);
            float Ys[kMaxCkptK];
            Ys[0] = A.ckpt[static_cast<int64_t>(c) * a.total + g];
            // ReLU: blocks of kMaskSteps steps recorded at once; Softplus: one step at a time
            constexpr int kBlk = (ACT == SL_ACT_RELU) ? kMaskSteps : 1;
            if (i1 - i0 > kBlk) {
                // a long segment: recompute its states first (Y_{i0+1} .. Y_{i1-1})
                // (one failure check per step, at its AND barrier, as in the sampler)
                for (int i = i0; i < i1 - 1; ++i) {
                    T.Y = Ys[i - i0];
                    tile_features<L2>(T, a);
                    tile_sync_issue_all(T, C, 0, issuer);
                    tile_rng_any(T, a, i, blk);
#pragma unroll
                    for (int l = 1; l <= 4; ++l) {
                        ok &= tile_wait(T, abort_flag, a.status);
                        tile_hidden_act<ACT, L2>(T);
                        tile_sync_issue_all(T, C, l, issuer);
                    }
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_out<L2>(T, a, i);
                    ok = bar_and(T.bar_id, ok);
                    if (!ok) break;
                    Ys[i - i0 + 1] = T.Y;
                }
            }
            if constexpr (ACT == SL_ACT_SOFTPLUS) {
                for (int i = i1 - 1; ok && i >= i0; --i) {
                    tile_rng_any(T, a, i, blk);
                    // the step's forward once, keeping sigma(z_3) and sigma(z_4) in tensor memory
                    // (one failure check per step, at its AND barrier)
                    T.Y = Ys[i - i0];
                    tile_features<L2>(T, a);
                    tile_sync_issue_all(T, C, 0, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_hidden_act<ACT, L2>(T);
                    tile_sync_issue_all(T, C, 1, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_hidden_act<ACT, L2>(T);
                    tile_sync_issue_all(T, C, 2, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_forward_sigma<true>(T, kSig3);
                    tile_sync_issue_all(T, C, 3, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_forward_sigma<false>(T, kSig4);
                    // backward chain with c_j = lambda * ell_j(X_i): dh4 = W5^T c, then dh3, dh2
                    tile_cotangent(T, lam);
                    tile_sync_issue_T_all(T, CT, 0, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_backward_sig(T, kSig4);
                    tile_sync_issue_T_all(T, CT, 1, issuer);
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_backward_sig(T, kSig3);
                    tile_sync_issue_T_all(T, CT, 2, issuer);
                    for (int lt = 3; lt <= 4; ++lt) {
                        const int l = 5 - lt;               // dh_l is in the accumulator
                        ok &= tile_wait(T, abort_flag, a.status);
                        float dh[SL_WIDTH];
                        tile_acc50(T, dh);
                        // the step's forward again, up to z_l (issues 0 .. l-1)
                        T.Y = Ys[i - i0];
                        tile_features<L2>(T, a);
                        tile_sync_issue_all(T, C, 0, issuer);
                        for (int ll = 1; ll < l; ++ll) {
                            ok &= tile_wait(T, abort_flag, a.status);
                            tile_hidden_act<ACT, L2>(T);
                            tile_sync_issue_all(T, C, ll, issuer);
                        }
                        ok &= tile_wait(T, abort_flag, a.status);
                        tile_backward_sp(T, dh);
                        tile_sync_issue_T_all(T, CT, lt, issuer);   // dh_{l-1} = W_l^T dz_l
                    }
                    ok &= tile_wait(T, abort_flag, a.status);
                    {
                        tc_fence_after();
                        uint32_t gf[8];
                        tmem_ld8(T.taddr, gf);
                        tmem_wait_ld();
                        tc_fence_before();
                        lam = __uint_as_float(gf[0]);
#pragma unroll
                        for (int q = 0; q < SL_MAX_DIN_TC - 2; ++q)
                            if (q < p) gth[q] += __uint_as_float(gf[2 + q]);
                    }
                    ok = bar_and(T.bar_id, ok);
                }
            } else {
            // blocks of at most kMaskSteps steps, last first: a forward pass over the block that
            // records every hidden layer's ReLU pattern, then the reverse steps of the block
            for (int j1 = i1; ok && j1 > i0;) {
                const int j0 = max(i0, j1 - kMaskSteps);
                T.Y = Ys[j0 - i0];
                for (int i = j0; i < j1; ++i) {
                    tile_features<L2>(T, a);
                    tile_sync_issue_all(T, C, 0, issuer);
                    tile_rng_any(T, a, i, blk);
#pragma unroll
                    for (int l = 1; l <= 4; ++l) {
                        ok &= tile_wait(T, abort_flag, a.status);
                        tile_hidden_rec(T, tmask + ((i - j0) * 4 + (l - 1)) * 2 * kTile);
                        tile_sync_issue_all(T, C, l, issuer);
                    }
                    ok &= tile_wait(T, abort_flag, a.status);
                    tile_out<L2>(T, a, i);
                    ok = bar_and(T.bar_id, ok);
                    if (!ok) break;
                }
                for (int i = j1 - 1; ok && i >= j0; --i) {
                    // backward chain with c_j = lambda * ell_j(X_i)
                    tile_rng_any(T, a, i, blk);
                    tile_cotangent(T, lam);
                    tile_sync_issue_T_all(T, CT, 0, issuer);
#pragma unroll
                    for (int lt = 1; lt <= 4; ++lt) {   // dh4 -> W4^T, dh3 -> W3^T, dh2 -> W2^T, dh1 -> W1^T
                        ok &= tile_wait(T, abort_flag, a.status);
                        const uint32_t* mr = tmask + ((i - j0) * 4 + (4 - lt)) * 2 * kTile;
                        tile_backward_bits(T, mr[0], mr[kTile]);
                        tile_sync_issue_T_all(T, CT, lt, issuer);
                    }
                    // d/d(features): lambda <- d/dY_i, g_theta += d/dtheta
                    ok &= tile_wait(T, abort_flag, a.status);
                    {
                        tc_fence_after();
                        uint32_t gf[8];
                        tmem_ld8(T.taddr, gf);
                        tmem_wait_ld();
                        tc_fence_before();
                        lam = __uint_as_float(gf[0]);
#pragma unroll
                        for (int q = 0; q < SL_MAX_DIN_TC - 2; ++q)
                            if (q < p) gth[q] += __uint_as_float(gf[2 + q]);
                    }
                    ok = bar_and(T.bar_id, ok);
                }
                j1 = j0;
            }
            }
        }
        if (!ok) break;
        if (valid) {
            A.pv[a.total + g] = lam;
            for (int q = 0; q < p; ++q) A.pv[static_cast<int64_t>(2 + q) * a.total + g] = gth[q];
            if (!isfinite(lam)) raise_status(a.status, SL_DEV_NONFINITE);
        }
    }
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

template <int WG, int ACT>
int launch_reverse(const AdjTC& A, cudaStream_t st) {
    auto kern = tc_adjoint_reverse_kernel<WG, ACT>;
    const size_t smem = 1024 + kBBytes + kBTBytes + static_cast<size_t>(WG) * mask_words_per_tile<ACT>() * 4 +
                        (WG + 1) * 8 + 16;
    int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)),
                        "tc_adjoint attribute");
    if (rc) return rc;
    // The list's length is known on the device only: one persistent CTA per SM
    // (at most as many as the paths could fill); CTAs without a tile exit.
    const int64_t max_tiles = (A.s.total + kTile - 1) / kTile;
    int64_t grid = sm_count();
    const int64_t need = (max_tiles + WG - 1) / WG;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 128 * WG, smem, st>>>(A);
    return cuda_error(cudaGetLastError(), "tc_adjoint launch");
}

}  // namespace

// Tensor-core adjoint: requires an MLP model (ReLU or Softplus), d_in <= 7, m <= 8.
// ckpt: [n_ckpt + 1][total] (the sampler writes rows 0 .. n_steps / k); yt:
// [total]; list: [total]; count: one word.
int launch_tc_adjoint(const SimArgs& s, float K, int k, int n_ckpt, float* ckpt, float* pv, float* yt,
                      uint32_t* list, unsigned* count, cudaStream_t st) {
    if (s.d_in > SL_MAX_DIN_TC) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d > %d", s.d_in, SL_MAX_DIN_TC);
    if (k > kMaxCkptK) return set_error(SL_ERR_UNSUPPORTED, "ckpt_k=%d > %d", k, kMaxCkptK);
    if (s.total > static_cast<int64_t>(UINT32_MAX)) return set_error(SL_ERR_UNSUPPORTED, "total_paths >= 2^32");
    // 1. forward: the sampler, keeping Y_0, Y_k, Y_2k, ..
    SimArgs f = s;
    f.out_YT = yt;
    f.out_grid = ckpt;
    f.grid_k = k;
    int rc = launch_tc_7l(s.m, f, st);
    if (rc) return rc;
    // 2. payoff of every path, list of the in-the-money ones
    rc = cuda_error(cudaMemsetAsync(count, 0, sizeof(unsigned), st), "count clear");
    if (rc) return rc;
    const unsigned blocks = static_cast<unsigned>((s.total + 255) / 256);
    itm_compact_kernel<<<blocks, 256, 0, st>>>(yt, s.total, K, s.p, pv, list, count);
    rc = cuda_error(cudaGetLastError(), "itm_compact launch");
    if (rc) return rc;
    // 3. reverse sweep over the listed paths
    AdjTC A{};
    A.s = s;
    A.s.out_YT = nullptr;
    A.s.out_grid = nullptr;
    A.K = K;
    A.k = k;
    A.n_ckpt = n_ckpt;
    A.ckpt = ckpt;
    A.pv = pv;
    A.list = list;
    A.count = count;
    // Softplus keeps a layer's cotangent (50 floats per thread) live across the forward
    // recompute: two warpgroups per CTA leave 255 registers per thread
    if (s.act == SL_ACT_SOFTPLUS) return launch_reverse<2, SL_ACT_SOFTPLUS>(A, st);
    return launch_reverse<3, SL_ACT_RELU>(A, st);
}

}  // namespace sl
