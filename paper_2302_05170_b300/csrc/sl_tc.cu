// sl_tc.cu -- BF16 tensor-core (tcgen05) form of the 7L online sampler
// (Algorithm I, steps 2-8) for sm_103a.
//
// The network of Eq. (6.4) is a chain of five GEMMs per coarse step:
//   layer 1:   [128 paths x K=16]  x [K x N=64]      (features, hi+lo split)
//   layers 2-4 [128 paths x K=112] x [K x N=64]      (50 activations hi + lo, 1)
//   layer 5:   [128 paths x K=112] x [K x N=16]      (m <= 8 outputs used)
// A persistent CTA (one per SM) holds S independent path tiles ("slots") of
// 128 paths.  Warpgroup t (warps 4t..4t+3, TMEM lanes 32*(warp%4)..) owns
// slot t: its warp t % 4 issues the slot's tcgen05.mma (one elected lane), with B
// (weights) in shared memory through 128-byte-swizzled K-major descriptors, A
// (activations) and FP32 accumulators in tensor memory; all four warps are the
// slot's epilogue: each thread reads the accumulator row of its path with
// tcgen05.ld, applies the activation (ReLU fused into the BF16 conversions, or
// Softplus), splits every activation h into BF16 hi + lo (hi = h truncated to
// BF16, lo = BF16(h - hi)), and writes the next A tile.  Several slots keep
// independent MMA groups in the tensor pipe at once; the Philox normals and the
// Lagrange basis of a step are computed while the step's output-layer MMAs run.
//
// Numerics: weights and biases are rounded to BF16 (nearest, ties to even);
// the network's inputs and activations carry ~16 significant bits through the
// hi+lo split (a single BF16 rounding of every activation gives ~1e-2 per-path
// error over 16 steps, the split ~1e-5); accumulation is FP32; the state,
// normals and interpolation are FP32.  Biases ride on a constant-1 input (K index
// 98 of the hidden inputs, 2*d_in of the features), so the epilogue adds nothing.
// The Softplus form runs in base 2: the features and the bias unit are scaled by
// log2(e) (the bias unit as a BF16 hi + lo pair), so every accumulator holds
// z log2(e), the activation log2(1 + 2^y) = Softplus(z) log2(e) takes the exponent
// and logarithm units without scaling, the hidden weights are unchanged
// (ln 2 log2(e) = 1), and the output layer's sum is scaled back by ln 2.
// The hidden A row keeps each 16-neuron chunk's hi and lo words in 16 adjacent
// columns (one store per chunk); the features sit in the slot's last 8 columns,
// written once per tile except Y's word.
//
// Synchronisation: the four warps of a slot meet at a named barrier once the
// next A operand is written, and the issuing warp then issues the layer's MMAs
// and commits them to the slot's mbarrier d_ready, on which all four warps
// wait.  Warp w runs on SM sub-partition w % 4, so warpgroup t issuing from its
// warp t % 4 spreads the slots' issue work over the four sub-partitions (with
// every slot issuing from its warp 0, sub-partition 0 carried all of it and its
// warps arrived last at every hand-off: 11.5 ms against 11.0 ms on the
// 16 x 1e6 x 16 workload).  Every wait is bounded (about one second of global
// time); on expiry the kernel sets SL_DEV_TIMEOUT in the status word.  The
// waits' results are ANDed over the slot's warps once per step (a bar.red at
// the step's end), where a failure stops the slot; every issuer then drains its
// own MMAs (bounded) and the tensor memory is released.
#include "sl_tc_common.cuh"

namespace sl {
namespace {

using namespace tc;

// WG warpgroups per CTA, TPW path tiles per warpgroup (S = WG * TPW tiles in
// flight).  Warp w of a warpgroup reads and writes TMEM lanes 32(w%4).., i.e.
// paths 32(w%4).. of each of its tiles; warp wg % 4 of the warpgroup also issues the
// tiles' MMAs.  With TPW = 2 the warpgroup alternates between its two tiles
// layer by layer, so one tile's epilogue runs while the other tile's MMAs run
// ("ping-pong"); with TPW = 1 the overlap comes only from other warpgroups.
template <int WG, int TPW, int ACT>
__global__ void __launch_bounds__(128 * WG, 1) tc_7l_kernel(const SimArgs a) {
    constexpr int S = WG * TPW;
    constexpr bool L2 = (ACT == SL_ACT_SOFTPLUS);   // Softplus in base 2 (softplus2_fast)
    constexpr uint32_t kCols = (S * 128 <= 128) ? 128 : (S * 128 <= 256) ? 256 : 512;
    static_assert(S * 128 <= 512, "tensor memory holds 512 columns");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* sB = smem;                                              // weights (1024-aligned)
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kBBytes);            // d_ready[S], drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wg = warp >> 2, wq = warp & 3;
    const int r = wq * 32 + lane;                                          // row = TMEM lane = path in tile
    const bool issuer = (wq == (wg & 3));                                 // sub-partition wg % 4

    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(smem_u32(&bars[k]), 1);   // d_ready: tcgen05.commit
        mbar_init(smem_u32(&bars[S]), WG);                              // drain: one commit per issuer
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

    IssueConst C;
    const uint32_t sB_u = smem_u32(sB);
    C.db0 = sw128_desc(sB_u);
    C.db1 = sw128_desc(sB_u + kB1Bytes);
    C.db2 = sw128_desc(sB_u + kB1Bytes + kBHBytes);
    C.db3 = sw128_desc(sB_u + kB1Bytes + 2 * kBHBytes);
    C.db4 = sw128_desc(sB_u + kB1Bytes + 3 * kBHBytes);

    Tile T[TPW];
#pragma unroll
    for (int j = 0; j < TPW; ++j) {
        const int slot = wg * TPW + j;
        T[j].d_tmem = tmem_base + static_cast<uint32_t>(slot * 128);
        T[j].taddr = T[j].d_tmem + (static_cast<uint32_t>(wq * 32) << 16);
        T[j].d_bar = smem_u32(&bars[slot]);
        T[j].bar_id = 1 + slot;
        T[j].dph = 0;
        tile_init_row<L2>(T[j]);
    }

    const int64_t n_tiles = (a.total + kTile - 1) / kTile;
    const int64_t tile_stride = static_cast<int64_t>(gridDim.x) * S;
    bool ok = true;
    // The warpgroup's tiles are consecutive: tile j of round k is base + j.
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * S + wg * TPW; base < n_tiles; base += tile_stride) {
#pragma unroll
        for (int j = 0; j < TPW; ++j) {   // a tile past the end computes garbage rows and stores nothing
            tile_begin(T[j], a, base + j, r);
            if (base + j >= n_tiles) T[j].valid = false;
            if (ok) tile_features_init<L2>(T[j], a);
            ok = tile_sync_issue(T[j], C, 0, ok, issuer);
            if (!ok) break;
        }
        if (!ok) break;
        for (int i = 0; i < a.n_steps; ++i) {
#pragma unroll
            for (int l = 1; l <= 4; ++l) {
#pragma unroll
                for (int j = 0; j < TPW; ++j) {
                    ok &= tile_wait(T[j], abort_flag, a.status);
                    tile_hidden_act<ACT, L2>(T[j]);
                    tile_sync_issue_all(T[j], C, l, issuer);
                    // the step's normal and Lagrange basis while the output layer's MMAs run
                    if (l == 4) tile_rng(T[j], a, i);
                }
            }
#pragma unroll
            for (int j = 0; j < TPW; ++j) {
                ok &= tile_wait(T[j], abort_flag, a.status);
                tile_out<L2>(T[j], a, i);
                if (i + 1 < a.n_steps) {
                    tile_features<L2>(T[j], a);
                    tile_sync_issue_all(T[j], C, 0, issuer);
                }
            }
            // Every warp of the warpgroup must take the same branch below and meet the
            // same named barriers afterwards: agree on `ok` (also after the last step).
            ok = bar_and(T[0].bar_id, ok);
            if (!ok) break;
        }
        if (!ok) break;
#pragma unroll
        for (int j = 0; j < TPW; ++j) tile_end(T[j], a);
    }
    // Drain: each issuer commits once more; the allocating warp waits for all
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

template <int WG, int TPW>
size_t tc_smem_bytes() {
    return 1024 + kBBytes + (WG * TPW + 1) * 8 + 16;
}

template <int WG, int TPW, int ACT = SL_ACT_RELU>
int launch_cfg(const SimArgs& a, cudaStream_t st) {
    constexpr int S = WG * TPW;
    auto kern = tc_7l_kernel<WG, TPW, ACT>;
    const size_t smem = tc_smem_bytes<WG, TPW>();
    int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)),
                        "tc_7l attribute");
    if (rc) return rc;
    const int64_t n_tiles = (a.total + kTile - 1) / kTile;
    int64_t grid = sm_count();
    const int64_t need = (n_tiles + S - 1) / S;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 128 * WG, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "tc_7l launch");
}

int g_slots = 4;   // path tiles in flight per CTA (sl_tc_set_slots)
int g_tpw = 1;     // tiles per warpgroup (sl_tc_set_pipeline)

}  // namespace

int launch_tc_7l(int m, const SimArgs& a, cudaStream_t st) {
    (void)m;
    if (a.d_in > SL_MAX_DIN_TC) return set_error(SL_ERR_UNSUPPORTED, "d_in=%d > %d", a.d_in, SL_MAX_DIN_TC);
    if (a.act == SL_ACT_SOFTPLUS) {   // one tile per warpgroup
        switch (g_slots) {
            case 2: return launch_cfg<2, 1, SL_ACT_SOFTPLUS>(a, st);
            case 3: return launch_cfg<3, 1, SL_ACT_SOFTPLUS>(a, st);
            default: return launch_cfg<4, 1, SL_ACT_SOFTPLUS>(a, st);
        }
    }
    if (g_tpw == 2) return (g_slots == 2) ? launch_cfg<1, 2>(a, st) : launch_cfg<2, 2>(a, st);
    switch (g_slots) {
        case 2: return launch_cfg<2, 1>(a, st);
        case 3: return launch_cfg<3, 1>(a, st);
        default: return launch_cfg<4, 1>(a, st);
    }
}

int tc_set_slots(int s) {
    if (s < 2 || s > 4) return set_error(SL_ERR_ARG, "slots=%d outside [2,4]", s);
    if (g_tpw == 2 && s == 3) return set_error(SL_ERR_ARG, "slots=3 needs one tile per warpgroup");
    g_slots = s;
    return SL_OK;
}

int tc_get_slots() { return g_slots; }

int tc_set_pipeline(int tpw) {
    if (tpw != 1 && tpw != 2) return set_error(SL_ERR_ARG, "tiles per warpgroup=%d (1 or 2)", tpw);
    if (tpw == 2 && g_slots == 3) return set_error(SL_ERR_ARG, "slots=3 needs one tile per warpgroup");
    g_tpw = tpw;
    return SL_OK;
}

int tc_get_pipeline() { return g_tpw; }

}  // namespace sl

extern "C" {

int sl_tc_set_slots(int slots) { return sl::tc_set_slots(slots); }
int sl_tc_get_slots(void) { return sl::tc_get_slots(); }
int sl_tc_set_pipeline(int tiles_per_warpgroup) { return sl::tc_set_pipeline(tiles_per_warpgroup); }
int sl_tc_get_pipeline(void) { return sl::tc_get_pipeline(); }

}  // extern "C"
