// sl_simulate.cu -- C-ABI entry points of the online 7L sampler (Algorithm I,
// steps 2-8): argument checks, workspace layout, dispatch to the FP32 CUDA-core
// form or the BF16 tcgen05 form, and the FP64 per-set moments.
#include <math.h>

#include "sl_check.cuh"
#include "sl_internal.cuh"

using namespace sl;

namespace sl {

int model_p(int model) { return model == SL_MODEL_GBM_EXACT ? 2 : 3; }

int check_net(const sl_net* net, int m, int p) {
    if (!net || !net->params) return set_error(SL_ERR_ARG, "network (params) required for SL_MODEL_MLP");
    if (net->m != m) return set_error(SL_ERR_ARG, "net->m=%d but m=%d", net->m, m);
    if (net->d_in != p + 2) return set_error(SL_ERR_ARG, "net->d_in=%d but p=%d (d_in = p + 2)", net->d_in, p);
    if (net->d_in < 2 || net->d_in > SL_MAX_DIN)
        return set_error(SL_ERR_UNSUPPORTED, "d_in=%d outside [2,%d]", net->d_in, SL_MAX_DIN);
    if (net->act != SL_ACT_RELU && net->act != SL_ACT_SOFTPLUS)
        return set_error(SL_ERR_ARG, "act=%d", net->act);
    if (net->prec != SL_PREC_FP32 && net->prec != SL_PREC_BF16)
        return set_error(SL_ERR_ARG, "prec=%d", net->prec);
    if (net->prec == SL_PREC_BF16) {
        if (net->d_in > SL_MAX_DIN_TC)
            return set_error(SL_ERR_UNSUPPORTED, "BF16 tensor-core form needs d_in <= %d", SL_MAX_DIN_TC);
    }
    return SL_OK;
}

int check_common(int model, const sl_net* net, const float* theta, int p, float T, int n_steps,
                 int m) {
    if (model != SL_MODEL_MLP && model != SL_MODEL_GBM_EXACT && model != SL_MODEL_OU_EXACT)
        return set_error(SL_ERR_ARG, "model=%d", model);
    if (m < SL_MIN_M || m > SL_MAX_M)
        return set_error(SL_ERR_UNSUPPORTED, "m=%d outside [%d,%d]", m, SL_MIN_M, SL_MAX_M);
    if (n_steps < 1) return set_error(SL_ERR_UNSUPPORTED, "n_steps=%d < 1", n_steps);
    if (!(T > 0.0f) || !isfinite(T)) return set_error(SL_ERR_ARG, "T must be finite and > 0");
    if (!theta && p > 0) return set_error(SL_ERR_ARG, "theta == NULL");
    if (model == SL_MODEL_MLP) return check_net(net, m, p);
    if (p != model_p(model))
        return set_error(SL_ERR_ARG, "model %d needs p=%d, got %d", model, model_p(model), p);
    return SL_OK;
}

}  // namespace sl

namespace {

int dispatch(int model, const sl_net* net, int m, const SimArgs& a, cudaStream_t st) {
    if (model == SL_MODEL_MLP && net->prec == SL_PREC_BF16) return launch_tc_7l(m, a, st);
    return launch_simt_7l(model, m, a, st);
}

}  // namespace

extern "C" {

size_t sl_simulate_workspace_size(int64_t total_paths, int n_sets) {
    if (total_paths < 0) total_paths = 0;
    if (n_sets < 1) n_sets = 1;
    return kStatusBytes + align256(static_cast<size_t>(total_paths) * sizeof(float)) +
           set_moments_scratch_bytes(n_sets);
}

int seven_league_simulate_batched(int model, const sl_net* net, const float* theta, int p,
                                  const float* Y0, const int64_t* path_offsets, int n_sets,
                                  int64_t total_paths, float T, int n_steps, int m, uint64_t seed,
                                  float* out_YT, float* out_grid, double* out_mean,
                                  double* out_var, void* ws, size_t ws_bytes, void* stream) {
    int rc = check_common(model, net, theta, p, T, n_steps, m);
    if (rc) return rc;
    if (n_sets < 1 || n_sets > SL_MAX_SETS) return set_error(SL_ERR_ARG, "n_sets=%d", n_sets);
    if (total_paths < 0) return set_error(SL_ERR_ARG, "total_paths < 0");
    if (total_paths > (int64_t(1) << 40)) return set_error(SL_ERR_UNSUPPORTED, "total_paths too large");
    if (!Y0 || !path_offsets) return set_error(SL_ERR_ARG, "Y0 / path_offsets == NULL");
    if (!out_YT && !out_grid && !out_mean && !out_var)
        return set_error(SL_ERR_ARG, "no output requested");
    if (!ws) return set_error(SL_ERR_WORKSPACE, "ws == NULL");
    const bool moments = out_mean || out_var;
    const size_t need = kStatusBytes +
                        ((moments && !out_YT) ? align256(static_cast<size_t>(total_paths) * 4) : 0) +
                        (moments ? set_moments_scratch_bytes(n_sets) : 0);
    if (ws_bytes < need)
        return set_error(SL_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* w = static_cast<unsigned char*>(ws);
    unsigned* status = reinterpret_cast<unsigned*>(w);
    size_t off = kStatusBytes;
    float* yt = out_YT;
    if (moments && !out_YT) {
        yt = reinterpret_cast<float*>(w + off);
        off += align256(static_cast<size_t>(total_paths) * 4);
    }
    void* part = w + off;

    SimArgs a{};
    if (model == SL_MODEL_MLP) {
        a.params = net->params;
        a.d_in = net->d_in;
        a.act = net->act;
    }
    a.theta = theta;
    a.p = p;
    a.Y0 = Y0;
    a.offsets = path_offsets;
    a.n_sets = n_sets;
    a.total = total_paths;
    a.dt = T / static_cast<float>(n_steps);
    a.n_steps = n_steps;
    a.seed = seed;
    a.out_YT = yt;
    a.out_grid = out_grid;
    a.status = status;
    a.m = m;
    rc = make_gh_const(m, &a.gh);
    if (rc) return rc;
    rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (total_paths > 0) {
        rc = dispatch(model, net, m, a, st);
        if (rc) return rc;
    }
    if (moments) return launch_set_moments(yt, path_offsets, n_sets, total_paths, out_mean, out_var, part, st);
    return SL_OK;
}

size_t sl_simulate_range_workspace_size(int64_t n_paths, int n_sets) {
    if (n_sets < 1) n_sets = 1;
    return sl_simulate_workspace_size(n_paths, n_sets) + align256(static_cast<size_t>(n_sets + 1) * sizeof(int64_t));
}

int seven_league_simulate_range(int model, const sl_net* net, const float* theta, int p, const float* Y0,
                                const int64_t* path_offsets, int n_sets, int64_t first_path, int64_t n_paths,
                                float T, int n_steps, int m, uint64_t seed, float* out_YT, float* out_grid,
                                double* out_mean, double* out_var, int64_t* out_count, void* ws,
                                size_t ws_bytes, void* stream) {
    int rc = check_common(model, net, theta, p, T, n_steps, m);
    if (rc) return rc;
    if (n_sets < 1 || n_sets > SL_MAX_SETS) return set_error(SL_ERR_ARG, "n_sets=%d", n_sets);
    if (first_path < 0 || n_paths < 0) return set_error(SL_ERR_ARG, "first_path / n_paths < 0");
    if (first_path + n_paths > (int64_t(1) << 40)) return set_error(SL_ERR_UNSUPPORTED, "paths beyond 2^40");
    if (!Y0 || !path_offsets) return set_error(SL_ERR_ARG, "Y0 / path_offsets == NULL");
    if (!out_YT && !out_grid && !out_mean && !out_var && !out_count)
        return set_error(SL_ERR_ARG, "no output requested");
    if (!ws) return set_error(SL_ERR_WORKSPACE, "ws == NULL");
    const bool moments = out_mean || out_var;
    const size_t need = kStatusBytes +
                        ((moments && !out_YT) ? align256(static_cast<size_t>(n_paths) * 4) : 0) +
                        align256(static_cast<size_t>(n_sets + 1) * sizeof(int64_t)) +
                        (moments ? set_moments_scratch_bytes(n_sets) : 0);
    if (ws_bytes < need)
        return set_error(SL_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* w = static_cast<unsigned char*>(ws);
    unsigned* status = reinterpret_cast<unsigned*>(w);
    size_t off = kStatusBytes;
    float* yt = out_YT;
    if (moments && !out_YT) {
        yt = reinterpret_cast<float*>(w + off);
        off += align256(static_cast<size_t>(n_paths) * 4);
    }
    int64_t* local = reinterpret_cast<int64_t*>(w + off);
    off += align256(static_cast<size_t>(n_sets + 1) * sizeof(int64_t));
    void* part = w + off;

    SimArgs a{};
    if (model == SL_MODEL_MLP) {
        a.params = net->params;
        a.d_in = net->d_in;
        a.act = net->act;
    }
    a.theta = theta;
    a.p = p;
    a.Y0 = Y0;
    a.offsets = path_offsets;
    a.n_sets = n_sets;
    a.total = n_paths;
    a.first = first_path;
    a.dt = T / static_cast<float>(n_steps);
    a.n_steps = n_steps;
    a.seed = seed;
    a.out_YT = yt;
    a.out_grid = out_grid;
    a.status = status;
    a.m = m;
    rc = make_gh_const(m, &a.gh);
    if (rc) return rc;
    rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    if (n_paths > 0) {
        rc = dispatch(model, net, m, a, st);
        if (rc) return rc;
    }
    if (!moments && !out_count) return SL_OK;
    rc = launch_range_offsets(path_offsets, n_sets, first_path, n_paths, local, out_count, st);
    if (rc) return rc;
    if (moments) return launch_set_moments(yt, local, n_sets, n_paths, out_mean, out_var, part, st);
    return SL_OK;
}

int seven_league_simulate(int model, const float* theta, int p, float Y0, float T, int n_steps,
                          int m, const sl_net* weights, int64_t n_paths, uint64_t seed,
                          float* out, void* stream) {
    int rc = check_common(model, weights, theta, p, T, n_steps, m);
    if (rc) return rc;
    if (n_paths < 0 || n_paths > (int64_t(1) << 32)) return set_error(SL_ERR_ARG, "n_paths=%lld", (long long)n_paths);
    if (!out) return set_error(SL_ERR_ARG, "out == NULL");
    if (n_paths == 0) return SL_OK;
    SimArgs a{};
    if (model == SL_MODEL_MLP) {
        a.params = weights->params;
        a.d_in = weights->d_in;
        a.act = weights->act;
    }
    a.theta = theta;
    a.p = p;
    a.Y0 = nullptr;
    a.y0_scalar = Y0;
    a.offsets = nullptr;
    a.n_sets = 1;
    a.total = n_paths;
    a.dt = T / static_cast<float>(n_steps);
    a.n_steps = n_steps;
    a.seed = seed;
    a.out_YT = out;
    a.status = nullptr;
    a.m = m;
    rc = make_gh_const(m, &a.gh);
    if (rc) return rc;
    return dispatch(model, weights, m, a, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
