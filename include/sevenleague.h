/*
 * sevenleague.h -- C ABI of the B300 (sm_103a) Seven-League (7L) library.
 *
 * The 7L scheme (Liu, Colonna, Grzelak, Oosterlee, arXiv:2302.05170) samples
 * an Ito SDE dY = a dt + b dW (Eq. 6.1) with large time steps: for every
 * Monte Carlo path and coarse step a small network H maps (Y_i, dt, theta) to
 * m conditional collocation points y_j (Eq. 6.3/6.4), a standard normal X is
 * drawn and Y_{i+1} = g_m(X) is the Lagrange interpolant through
 * (x_j, y_j) at the Gauss-Hermite points x_j (Algorithm I, steps 2-8).  The
 * offline stage (Algorithm I step 1) produces the training labels from
 * fine-step Euler-Maruyama paths (Eq. 6.2).
 *
 * Conventions (every entry point):
 *  - Array arguments are caller-owned DEVICE pointers (e.g. a torch tensor's
 *    data_ptr()) unless the comment says HOST.  The library never frees or
 *    keeps them after the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream; host-side argument
 *    checks happen before anything is enqueued.
 *  - Scratch memory comes from a caller buffer `ws` of `ws_bytes` bytes,
 *    sized by the matching *_workspace_size() query, 256-byte aligned.  The
 *    library allocates no device memory.
 *  - Every function returns an sl_status; on failure nothing was enqueued
 *    (SL_ERR_CUDA: a launch failed) and sl_last_error_string() says why.
 *  - Kernels that meet non-finite state or out-of-range indices set bits of a
 *    device status word in the first 256 bytes of `ws`; sl_workspace_status()
 *    synchronises the stream and reports them as SL_ERR_DEVICE.
 *  - Random numbers: X for (seed, tag, set s, path q, step i) is normal
 *    number i of the Philox4x32-10 stream with key (seed low, seed high) and
 *    counter (i/4, q, s, tag); Box-Muller on word pairs (0,1)/(2,3) of the
 *    block, uniforms ((w>>9)+1/2)/2^23.  Tags: 0 = 7L online, 1 = EM fine
 *    steps.  Results are therefore independent of launch shape and batching.
 */
#ifndef SEVENLEAGUE_H
#define SEVENLEAGUE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Network shape (Section "Numerical Results": 4 hidden layers of 50). */
#define SL_WIDTH 50
#define SL_N_HIDDEN 4
#define SL_MIN_M 2         /* supported collocation counts m */
#define SL_MAX_M 8
#define SL_MAX_DIN 8       /* FP32 form: d_in = 2 + p <= 8 */
#define SL_MAX_DIN_TC 7    /* BF16 tensor-core form: 2*d_in + 1 <= 16 */
#define SL_MAX_SETS (1 << 24)

typedef enum {
    SL_OK = 0,
    SL_ERR_ARG = 1,          /* NULL pointer, negative size, inconsistent arguments */
    SL_ERR_UNSUPPORTED = 2,  /* m outside [2,8], d_in too large, n_steps < 1, ... */
    SL_ERR_WORKSPACE = 3,    /* ws_bytes below the *_workspace_size() requirement */
    SL_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
    SL_ERR_DEVICE = 5,       /* the device status word is set (NaN/Inf state, bad index) */
    SL_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} sl_status;

/* Device status word bits (read with sl_workspace_status). */
#define SL_DEV_NONFINITE 0x1u   /* a path produced a non-finite state */
#define SL_DEV_OFFSETS 0x2u     /* path_offsets not non-decreasing or total mismatch (the
                                   samplers check a path's set against path_offsets in
                                   checked builds) */
#define SL_DEV_TIMEOUT 0x4u     /* a bounded mbarrier wait expired */
#define SL_DEV_INDEX 0x8u       /* an index derived on the device fell outside its array
                                   (checked builds, libsevenleague_checked.so) */

/* Collocation maps H (Eq. 6.3) */
enum { SL_MODEL_MLP = 0,        /* the network; theta = its parameter inputs (p = d_in - 2) */
       SL_MODEL_GBM_EXACT = 1,  /* exact lognormal quantile map, theta = (mu, sigma) */
       SL_MODEL_OU_EXACT = 2 }; /* exact OU map (Eq. 6.6), theta = (Ybar, sigma, lambda) */
/* SDEs for the offline Euler-Maruyama stage (Eq. 6.2) */
enum { SL_SDE_GBM = 0,          /* theta = (mu, sigma):        a = mu Y, b = sigma Y */
       SL_SDE_OU = 1,           /* theta = (Ybar, sigma, lambda), Eq. 6.5 */
       SL_SDE_CIR = 2 };        /* theta = (kappa, ybar, gamma), full truncation */
enum { SL_ACT_RELU = 0, SL_ACT_SOFTPLUS = 1 };
/* Arithmetic of the network in the online sampler */
enum { SL_PREC_FP32 = 0,        /* FP32 CUDA-core form */
       SL_PREC_BF16 = 1 };      /* tcgen05 BF16 tensor cores, FP32 accumulate, BF16 weights,
                                   activations split hi+lo in BF16; d_in <= SL_MAX_DIN_TC;
                                   ReLU or Softplus (sampler and adjoint) */
enum { SL_PAYOFF_CALL = 0 };    /* f(Y_T) = max(Y_T - K, 0) */

/*
 * The network H of Eq. (6.3)/(6.4): d_in -> 50 -> 50 -> 50 -> 50 -> m, hidden
 * activation `act`, linear output.  `params` (device, FP32) holds, layer by
 * layer, W_l row-major [out][in] followed by b_l; sl_n_params() gives its
 * length.  Input features are [Y_i, dt, theta_0 .. theta_{d_in-3}].
 * Output j is the collocation point at the j-th Gauss-Hermite node in
 * ascending order.  With prec = SL_PREC_BF16 the weights are rounded to BF16
 * (nearest, ties to even) when they are staged on chip.
 */
typedef struct sl_net {
    const float* params;
    int d_in;
    int m;
    int act;
    int prec;
} sl_net;

/* Library version (major*10000 + minor*100 + patch). */
int sl_version(void);
/* Text for the last failing call on this host thread. */
const char* sl_last_error_string(void);
/* Number of parameters of the network for (d_in, m). */
int64_t sl_n_params(int d_in, int m);

/*
 * HOST, FP64.  Gauss-Hermite points of the standard normal (probabilists'
 * Hermite polynomial He_m), ascending, by Golub-Welsch (eigenvalues of the
 * Jacobi matrix with off-diagonal sqrt(k)); w: probability weights
 * (sum 1); bary: first-form barycentric weights 1/prod_{k!=j}(x_j - x_k).
 * Any output pointer may be NULL.  Section "Methodology" (x_j are
 * Gauss-Hermite points of X ~ N(0,1)) and Section "Parallelization"
 * (barycentric Lagrange).  Errors: SL_ERR_UNSUPPORTED for m outside [2,8].
 */
int sl_gauss_hermite(int m, double* x, double* w, double* bary);

/*
 * HOST.  0-based ranks of the empirical quantiles at levels Phi(x_j) among n
 * samples: ceil(n Phi(x_j)) - 1 clamped to [0, n-1] (Algorithm I step 1,
 * labels y_j as quantiles of the fine-step samples).  ranks: HOST [m].
 */
int sl_quantile_ranks(int m, int64_t n, int64_t* ranks);

/* Synchronises `stream`, then reports the device status word of `ws`
 * (SL_OK or SL_ERR_DEVICE / SL_ERR_TIMEOUT).  *bits (HOST, may be NULL)
 * receives the raw SL_DEV_* bits. */
int sl_workspace_status(const void* ws, void* stream, uint32_t* bits);

/*
 * Self-test of the bounded waits (a library facility; the paper has no
 * counterpart).  Clears the status word of `ws` (device, >= 256 bytes) and
 * launches one warp that waits, with the kernels' own bounded mbarrier wait,
 * on a barrier nothing arrives on; after about one second the wait gives up
 * and sets SL_DEV_TIMEOUT, and the kernel returns.  sl_workspace_status then
 * reports SL_ERR_TIMEOUT; the context stays usable.
 */
int sl_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Online stage (Algorithm I, steps 2-8).
 * ---------------------------------------------------------------------- */

/* Bytes of workspace seven_league_simulate_batched needs. */
size_t sl_simulate_workspace_size(int64_t total_paths, int n_sets);

/*
 * Batched 7L sampler.  n_sets parameter sets; set s owns flat paths
 * [path_offsets[s], path_offsets[s+1]) (device int64 [n_sets+1],
 * non-decreasing, path_offsets[0] = 0, path_offsets[n_sets] = total_paths).
 * For every path: Y_0 = Y0[s]; for i < n_steps, y = H(Y_i, dt, theta_s) with
 * dt = T / n_steps, X = normal (seed, tag 0, s, q, i), Y_{i+1} = g_m(X) where
 * q is the path's index within its set.
 *   model      SL_MODEL_*; `net` is required for SL_MODEL_MLP (net->m == m,
 *              p == net->d_in - 2) and ignored otherwise (p = 2 or 3).
 *   theta      device FP32 [n_sets][p];  Y0: device FP32 [n_sets].
 *   out_YT     device FP32 [total_paths] terminal values, or NULL.
 *   out_grid   device FP32 [(n_steps+1)][total_paths] (step-major: all paths
 *              at t_i contiguous, Algorithm I step 7), or NULL.
 *   out_mean   device FP64 [n_sets] path means of Y_T, or NULL.
 *   out_var    device FP64 [n_sets] unbiased sample variances, or NULL.
 * The FP64 per-set reduction is deterministic (fixed order).
 */
int seven_league_simulate_batched(int model, const sl_net* net, const float* theta, int p,
                                  const float* Y0, const int64_t* path_offsets, int n_sets,
                                  int64_t total_paths, float T, int n_steps, int m, uint64_t seed,
                                  float* out_YT, float* out_grid, double* out_mean,
                                  double* out_var, void* ws, size_t ws_bytes, void* stream);

/*
 * Single parameter set, in the order (model, theta, Y0, T, n_steps, m,
 * weights, n_paths, seed, out): theta device FP32 [p], Y0 a HOST value, out
 * device FP32 [n_paths] terminal values.  Needs no workspace.
 */
int seven_league_simulate(int model, const float* theta, int p, float Y0, float T, int n_steps,
                          int m, const sl_net* weights, int64_t n_paths, uint64_t seed,
                          float* out, void* stream);

/*
 * Tuning of the BF16 tensor-core form (process-wide, read at launch time):
 *  - slots: 128-path tiles each persistent CTA keeps in flight (2..4, default 4);
 *  - pipeline: tiles per warpgroup (1 or 2, default 1).  With 2, a warpgroup
 *    alternates between two tiles layer by layer (one tile's epilogue beside
 *    the other's tensor-core work); slots must then be 2 or 4.  On the GBM
 *    workload 4 slots x 1 tile per warpgroup is fastest.
 * Both return SL_ERR_ARG for an unsupported value or combination.
 */
int sl_tc_set_slots(int slots);
int sl_tc_get_slots(void);
int sl_tc_set_pipeline(int tiles_per_warpgroup);
int sl_tc_get_pipeline(void);

/* Bytes of workspace seven_league_simulate_range needs for n_paths paths. */
size_t sl_simulate_range_workspace_size(int64_t n_paths, int n_sets);

/*
 * One contiguous range of a batched call, for splitting a batch across GPUs or
 * calls (the method's paths are independent: Algorithm I steps 4 and 7 run
 * per path).  theta, Y0 and path_offsets describe the WHOLE batch exactly as
 * for seven_league_simulate_batched; this call runs its flat paths
 * first_path .. first_path + n_paths - 1 (first_path + n_paths must not
 * exceed path_offsets[n_sets]).  Each path keeps its set and its index within
 * the set, hence its Philox normals, so out_YT[k] (device FP32 [n_paths]) is
 * bit for bit out_YT[first_path + k] of the whole call, in both network forms;
 * out_grid (or NULL): [(n_steps+1)][n_paths].  Per set, over the set's paths
 * inside the range: out_count (device int64 [n_sets] or NULL) their number,
 * out_mean / out_var (device FP64 [n_sets] or NULL) their mean and unbiased
 * variance (0 for fewer than one / two paths), deterministic as in the batched
 * call; a caller combining ranges weights them by the counts.  Workspace:
 * sl_simulate_range_workspace_size(n_paths, n_sets).  Errors as
 * seven_league_simulate_batched; SL_ERR_ARG for a negative first_path or
 * n_paths.  Allocates nothing.
 */
int seven_league_simulate_range(int model, const sl_net* net, const float* theta, int p, const float* Y0,
                                const int64_t* path_offsets, int n_sets, int64_t first_path, int64_t n_paths,
                                float T, int n_steps, int m, uint64_t seed, float* out_YT, float* out_grid,
                                double* out_mean, double* out_var, int64_t* out_count, void* ws,
                                size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * The 7L-CDC variant (timed beside the 7L scheme in Table 6.1; the remark
 * after Algorithm I): step 3's network evaluation per path is replaced by a
 * global interpolation built from a few network evaluations per parameter
 * set and step.  The paper gives the variant in outline; this library reads
 * it as follows.  For set s and step i (t_i = i dt, dt = T / n_steps):
 *   - marginal collocation points z_k = G_k(Y0[s], t_i, theta_s), k < m: the
 *     collocation map over the horizon t_i from the deterministic start
 *     (features [Y0, t_i, theta]); G = marg_net (NULL: net) for SL_MODEL_MLP,
 *     the exact map for the exact models.  At i = 0, z_k = Y0[s];
 *   - conditional points at the nodes C[k][j] = H_j(z_k, dt, theta_s);
 * and then, by `space`:
 * SL_CDC_SPACE_Y (interpolation in Y through the marginal nodes):
 *   - a path at Y_i takes yhat_j = sum_k C[k][j] L_k(Y_i), L_k the Lagrange
 *     basis in Y through the z_k, while min z <= Y_i <= max z; beyond the
 *     outermost node on a side, the line through the two outermost nodes on
 *     that side (degree m-1 extrapolation grows without bound); yhat = C[0]
 *     when all z_k coincide, as at i = 0.  Then Y_{i+1} = g_m(X) through
 *     (x_j, yhat_j), with the normals of the 7L sampler (tag 0).
 *   With a conditional map that is affine in Y (the exact GBM and OU maps)
 *   the chain equals the 7L chain.  Lagrange interpolation through the
 *   quantiles of a wide marginal (a lognormal with sigma sqrt(t) ~ 0.7) is
 *   ill-conditioned: a network's errors in C are magnified up to ~1e3-1e5.
 * SL_CDC_SPACE_QUANTILE (interpolation in the marginal's quantile coordinate):
 *   - G_i(xi) = sum_k z^(i)_k L_k(xi) through the Gauss-Hermite points x_k
 *     (continued beyond them by the lines through the two outermost nodes)
 *     is the marginal collocation map of t_i; a path carries xi_i (xi_0 = 0)
 *     with Y_i = G_i(xi_i);
 *   - eta[k][j] = G_{i+1}^{-1}(C[k][j]) (beyond [z_0, z_{m-1}] the lines;
 *     inside, the smallest root of G = y in the first node interval
 *     [x_k, x_{k+1}] with z_k <= y <= z_{k+1}, however close later crossings
 *     lie; see sl_cdcq_inverse); xi_{i+1} = sum_k sum_j eta[k][j]
 *     L_k(xi_i) L_j(X) for xi_i in [x_0, x_{m-1}] (beyond, the line in xi
 *     through the two outermost node rows sum_j eta[k][j] L_j(X)),
 *     Gauss-Hermite points in both variables (as well conditioned as g_m);
 *   - G_{i+1} must increase from its first to its last node (else the paths
 *     are NaN: SL_DEV_NONFINITE); coinciding nodes give Y_{i+1} = z_0.
 *   With the exact OU map the chain equals the 7L chain.
 * The network evaluations ((m + 1) per set and step; m + 2 in the quantile
 * coordinate) run in FP32 on CUDA cores whatever net->prec says; the paths
 * run in FP32; the inverses and the interpolants' coefficients in FP64.
 * ---------------------------------------------------------------------- */
#define SL_CDC_SPACE_Y 0
#define SL_CDC_SPACE_QUANTILE 1

/* Bytes of workspace seven_league_cdc_simulate_batched needs. */
size_t sl_cdc_workspace_size(int64_t total_paths, int n_sets, int n_steps);

/*
 * Batched 7L-CDC sampler.  Arguments, outputs and errors as
 * seven_league_simulate_batched, plus marg_net (SL_MODEL_MLP only; NULL = use
 * net; same d_in and m as net, its own activation) and space
 * (SL_CDC_SPACE_Y or SL_CDC_SPACE_QUANTILE; SL_ERR_ARG otherwise).  The
 * workspace holds, at byte offset 256, the tables of the call: FP32
 * [n_sets][n_steps][224].  SL_CDC_SPACE_QUANTILE, per (set, step): [0,8) the
 * marginal nodes of t_{i+1}; [8,16) the monomial coefficients of G_{i+1}
 * (FP64, rounded once); [16] x_0, [17] x_{m-1}, [18] the slope of the line
 * below x_0, [19] above x_{m-1}, [20] z_0, [21] z_{m-1}, [22] x_1, [23]
 * x_{m-2}; [24,88) eta[8][8]; [88,152) B[a][b] with xi_{i+1} = sum_a xi_i^a
 * sum_b B[a][b] X^b (FP64, rounded once); [152,184) the monomial rows in X of
 * the node rows 0, 1, m-2, m-1 (for xi beyond the hull); zero elsewhere and
 * beyond m.  SL_CDC_SPACE_Y, per (set,
 * step): [0,8) z (the marginal nodes, zero beyond m); [8,16) w
 * (their barycentric weights 1/prod_{l!=k}(z_k - z_l), computed in FP64 from
 * the FP32 nodes; all zero when the nodes coincide); [16,80) C[8][8] (row k =
 * the conditional points at z_k, zero beyond m); [80,88) S_lo and [88,96)
 * S_hi, the slopes (C[b][j] - C[a][j]) / (z_b - z_a) of the lines through the
 * two smallest and the two largest nodes (ties to the lower index; FP64,
 * rounded once; 0 if the two nodes coincide); [96,104) C_lo and [104,112)
 * C_hi, the rows of the smallest and the largest node; [112] z_lo, [113]
 * z_hi; [114,120) zero; then monomial coefficients (a = 0..m-1, FP64 sums
 * rounded once) of g_m through a row y, sum_j y_j b_j prod_{l!=j}(X - x_l)
 * (b_j the Gauss-Hermite points' barycentric weights): [120,128) D of row
 * C[0]; [128,192) A[k][a] of w_k times row k of C (zero when the nodes
 * coincide); [192,200) of C_lo, [200,208) of S_lo, [208,216) of C_hi,
 * [216,224) of S_hi.  Nodes that
 * coincide only in part give non-finite paths (SL_DEV_NONFINITE).
 */
int seven_league_cdc_simulate_batched(int model, const sl_net* net, const sl_net* marg_net, int space,
                                      const float* theta, int p, const float* Y0,
                                      const int64_t* path_offsets, int n_sets, int64_t total_paths,
                                      float T, int n_steps, int m, uint64_t seed, float* out_YT,
                                      float* out_grid, double* out_mean, double* out_var, void* ws,
                                      size_t ws_bytes, void* stream);

/*
 * G^{-1} of the quantile-coordinate 7L-CDC scheme (the step that moves the
 * conditional points into the next step's coordinate, eta = G^{-1}(C)) on
 * caller-given marginal nodes, by the table kernel's own device routine.
 * zn: device FP32 [n_maps][m], the nodes z_k of each map G(xi) = sum_k z_k
 * L_k(xi) through the Gauss-Hermite points (continued beyond them by the
 * lines through the two outermost nodes); y: device FP64 [n_maps][n_y];
 * out: device FP64 [n_maps][n_y], G^{-1}(y) of its row's map.  Inside
 * [z_0, z_{m-1}] the result is the smallest root of G = y in the first node
 * interval with z_k <= y <= z_{k+1}: the sign variations of the Bernstein
 * coefficients (FP64) of G - y on that interval isolate it (one variation:
 * one root; more: a left-first search over dyadic sub-intervals, down to
 * 2^-40 of the interval, for the first with one), then it is refined in FP32
 * and by one FP64 Newton step.  Roots closer together than 2^-40 of a node
 * interval, and a G that comes within rounding of y without crossing it,
 * are the cases where the choice can differ from the exact first root.
 * Nodes that all coincide give 0; a G that does not increase from its
 * first to its last node gives NaN.  Asynchronous on `stream`; allocates
 * nothing.  SL_ERR_UNSUPPORTED for m outside [2, 8], SL_ERR_ARG for
 * negative counts or NULL pointers, SL_ERR_CUDA if the launch fails.
 */
int sl_cdcq_inverse(int m, const float* zn, int n_maps, const double* y, int n_y, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Offline stage (Algorithm I, step 1).
 * ---------------------------------------------------------------------- */

/*
 * Euler-Maruyama terminal samples (Eq. 6.2): row r starts at Yi[r] and takes
 * n_fine steps of dt[r]/n_fine with normals (seed, tag 1, r, q, k); CIR uses
 * full truncation and returns max(Y,0).  theta device FP32 [n_rows][p]
 * (p = 2 for GBM, 3 for OU/CIR); Yi, dt device FP32 [n_rows];
 * out device FP32 [n_rows][n_paths].
 */
int sl_em_terminal(int sde, const float* theta, const float* Yi, const float* dt, int n_rows,
                   int64_t n_paths, int n_fine, uint64_t seed, float* out, void* stream);

/* Bytes of workspace sl_segmented_select needs. */
size_t sl_select_workspace_size(int n_seg, int n_k);

/*
 * Order statistics of ragged segments: out[s*n_k + j] = the ranks[j]-th
 * smallest (0-based) value of values[seg_offsets[s] .. seg_offsets[s+1]),
 * NaN where ranks[j] >= the segment's length.  Values must not be NaN.
 * seg_offsets device int64 [n_seg+1]; ranks HOST int64 [n_k], n_k <= 16.
 * Exact (radix select on the order-preserving 32-bit keys).
 */
int sl_segmented_select(const float* values, const int64_t* seg_offsets, int n_seg,
                        const int64_t* ranks, int n_k, float* out, void* ws, size_t ws_bytes,
                        void* stream);

/* Bytes of workspace em_collocation_labels needs. */
size_t sl_em_labels_workspace_size(int n_rows, int64_t n_paths, int m);

/*
 * Collocation labels y_j | (theta_r, Yi_r, dt_r): the empirical quantiles at
 * levels Phi(x_j) (ranks from sl_quantile_ranks) of n_paths Euler-Maruyama
 * terminal samples per row (sl_em_terminal), labels device FP32 [n_rows][m].
 */
int em_collocation_labels(int sde, const float* theta, const float* Yi, const float* dt,
                          int n_rows, int64_t n_paths, int n_fine, int m, uint64_t seed,
                          float* labels, void* ws, size_t ws_bytes, void* stream);

/*
 * em_collocation_labels for callers that cannot allocate device memory (the
 * paper has no counterpart: this is a deployment convenience).  A plugin
 * inside a host application that owns all device allocations, a service with
 * a memory budget fixed at start-up, or code that must not enter the CUDA
 * allocator at a given point can pass its inputs and the label output but not
 * a scratch buffer.  This entry point uses instead a fixed 16 MiB array that
 * the library keeps in device memory (a file-scope __device__ variable, held
 * on every GPU that loads the library until the process exits) and calls no
 * allocation routine.  Limits and behaviour:
 *  - n_rows * n_paths must not exceed sl_em_labels_noalloc_max_samples()
 *    (4,194,240 samples); larger calls return SL_ERR_WORKSPACE;
 *  - the first call on a device looks the array's address up
 *    (cudaGetSymbolAddress, with that device current) and caches it: make that
 *    first call before any stream capture on that device;
 *  - every call uses the same array, so calls whose work overlaps on the GPU
 *    (different streams, or different host threads) race; order them on one
 *    stream.  The array keeps the previous call's contents; the call clears
 *    its status word and overwrites every sample it reads;
 *  - the device status word (SL_DEV_* bits: a negative segment length, a
 *    non-finite sample) lives in the array, which no caller can address, so
 *    those bits are not reported: a caller that needs them uses
 *    em_collocation_labels with its own workspace and sl_workspace_status.
 * Arguments are checked as em_collocation_labels checks them (SL_ERR_ARG,
 * SL_ERR_UNSUPPORTED) before the size limit (SL_ERR_WORKSPACE); results and
 * the other errors are those of em_collocation_labels.
 */
int em_collocation_labels_noalloc(int sde, const float* theta, const float* Yi, const float* dt,
                                  int n_rows, int64_t n_paths, int n_fine, int m, uint64_t seed,
                                  float* labels, void* stream);
/* Largest n_rows * n_paths em_collocation_labels_noalloc accepts. */
size_t sl_em_labels_noalloc_max_samples(void);

/* ------------------------------------------------------------------------
 * Pathwise sensitivities (adjoint) of E[f(Y_T)], f(Y) = max(Y - K, 0).
 * ---------------------------------------------------------------------- */

/* Bytes of workspace seven_league_adjoint needs: the status word, ceil(n_steps /
 * ckpt_k) + 1 checkpoint rows of total_paths FP32, the per-path values, Y_T and
 * the in-the-money path list (BF16 form), and the per-set reduction scratch. */
size_t sl_adjoint_workspace_size(int64_t total_paths, int n_sets, int n_steps, int ckpt_k, int p);

/*
 * Same sampling as seven_league_simulate_batched (same arguments, normals and
 * paths); then, per path, f(Y_T) and its derivatives f'(Y_T) dY_T/dY0 and
 * f'(Y_T) dY_T/dtheta by reverse-mode differentiation through g_m and the
 * collocation map (network input gradient, or the exact map's derivative),
 * with Y_i checkpointed every ckpt_k steps (1..32) in the workspace and
 * recomputed between checkpoints.  Out-of-the-money paths (Y_T <= K) have
 * zero sensitivities.  Per set, FP64 means (deterministic reduction):
 *   out_value  [n_sets]       E[f(Y_T)]                      (or NULL)
 *   out_dY0    [n_sets]       dE/dY0   * seed_grad[s]        (or NULL)
 *   out_dtheta [n_sets][p]    dE/dtheta * seed_grad[s]       (or NULL)
 * seed_grad: device FP64 [n_sets] upstream factors (NULL = 1), for use as the
 * backward of an autograd function.  out_paths: device FP32 [(2+p)][total]
 * per-path (f, df/dY0, df/dtheta_0..) or NULL (kept in the workspace).
 * Network forms: net->prec = SL_PREC_FP32 runs the FP32 CUDA-core form (one
 * launch). SL_PREC_BF16 (ReLU or Softplus, d_in <= SL_MAX_DIN_TC) runs the
 * tcgen05 form in three launches on `stream`: the BF16 sampler (the same paths
 * as seven_league_simulate_batched) keeping the checkpoint rows, a compaction
 * of the in-the-money paths, and a reverse sweep over those paths only that
 * back-propagates through the same BF16 weights (hi + lo BF16 cotangents, FP32
 * accumulation; ReLU patterns recorded as bits, Softplus derivatives taken from
 * the pre-activations recomputed layer by layer). total_paths < 2^32 for the
 * BF16 form.
 */
int seven_league_adjoint(int model, const sl_net* net, const float* theta, int p, const float* Y0,
                         const int64_t* path_offsets, int n_sets, int64_t total_paths, float T,
                         int n_steps, int m, uint64_t seed, int payoff, float K, int ckpt_k,
                         double* out_value, double* out_dY0, double* out_dtheta,
                         const double* seed_grad, float* out_paths, void* ws, size_t ws_bytes,
                         void* stream);

/* ------------------------------------------------------------------------
 * Training of the network H (Algorithm I step 1: learn the map from
 * (Y_i, dt, theta) to the collocation labels; Section "Numerical Results":
 * Adam, batch 1024, learning rate 1e-3).  FP32 throughout.
 * ---------------------------------------------------------------------- */

/* Bytes of workspace sl_mse_grad / sl_train need for a minibatch of `batch` rows. */
size_t sl_train_workspace_size(int d_in, int m, int batch);

/* out[r][j] = H_j(feats[r]) (device FP32 [n_rows][d_in] -> [n_rows][m]); net->prec ignored. */
int sl_mlp_forward(const sl_net* net, const float* feats, int64_t n_rows, float* out, void* stream);

/*
 * Gradient of L = 1/(n_rows*m) sum_r sum_j (H_j(f_r) - y_rj)^2 over the rows
 * rows[0..n_rows) (device int32, NULL = 0..n_rows-1) of feats [N][d_in] and
 * labels [N][m]: grad device FP32 [sl_n_params], *loss device FP32 (may be
 * NULL).  Deterministic (fixed reduction order).  net->prec = SL_PREC_BF16:
 * H is the network with every weight and bias rounded to BF16 (nearest, ties
 * to even), the one the tensor-core sampler evaluates, and grad is its
 * gradient (applied to the FP32 parameters, a straight-through update).
 */
int sl_mse_grad(const sl_net* net, const float* feats, const float* labels, const int32_t* rows,
                int n_rows, float* grad, float* loss, void* ws, size_t ws_bytes, void* stream);

/*
 * One Adam step (Kingma & Ba) with step counter t >= 1 on n parameters:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 */
int sl_adam_step(float* params, float* adam_m, float* adam_v, const float* grad, int64_t n,
                 int64_t t, float lr, float b1, float b2, float eps, void* stream);

/*
 * n_batches Adam steps (t = t0+1 .. t0+n_batches) of the MSE loss on the
 * minibatches batch_rows[b*batch .. (b+1)*batch) (device int32): params,
 * adam_m, adam_v device FP32 [sl_n_params(d_in, m)] updated in place;
 * losses device FP32 [n_batches] (loss of each minibatch before its update,
 * may be NULL).  prec = SL_PREC_BF16 trains the BF16-rounded network (as
 * sl_mse_grad), SL_PREC_FP32 the FP32 one; SL_ERR_ARG otherwise.  Only kernel
 * launches on `stream`: capturable in a CUDA graph.
 */
int sl_train(float* params, int d_in, int m, int act, int prec, float* adam_m, float* adam_v, int64_t t0,
             const float* feats, const float* labels, const int32_t* batch_rows, int n_batches,
             int batch, float lr, float b1, float b2, float eps, float* losses, void* ws,
             size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SEVENLEAGUE_H */
