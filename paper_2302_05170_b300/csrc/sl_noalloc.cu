// sl_noalloc.cu -- a variant of em_collocation_labels for callers that cannot
// allocate device memory.
//
// Some callers have no allocator to hand: a plugin running inside a host
// application that owns every cudaMalloc, a real-time or embedded service
// whose memory budget is fixed at start-up, or code that must not touch the
// CUDA allocator between two points (for example while another component is
// capturing or replaying work).  They can still pass their inputs and the
// label output, but not the scratch buffer em_collocation_labels needs for the
// Euler-Maruyama terminal samples.  This file gives them an entry point whose
// scratch is a fixed-size array in the library's own device memory.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library's module is loaded holds it until the process exits.  In host code
// its name only stands for the symbol, not for a device address, so the
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached.  The entry point allocates nothing itself: it
// clears the status word and hands the array to em_collocation_labels as its
// workspace.
#include <mutex>

#include "sl_internal.cuh"

namespace sl {
namespace {

// Status word (256 B) + up to kNoAllocMaxSamples FP32 terminal samples: 16 MiB.
constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_ws on the current device (looked up on first use).
int noalloc_address(void** out) {
    int dev = 0;
    int rc = cuda_error(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return set_error(SL_ERR_UNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        rc = cuda_error(cudaGetSymbolAddress(&p, g_noalloc_ws), "cudaGetSymbolAddress");
        if (rc) return rc;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SL_OK;
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" {

size_t sl_em_labels_noalloc_max_samples(void) { return (kNoAllocBytes - kStatusBytes) / sizeof(float); }

int em_collocation_labels_noalloc(int sde, const float* theta, const float* Yi, const float* dt, int n_rows,
                                  int64_t n_paths, int n_fine, int m, uint64_t seed, float* labels,
                                  void* stream) {
    // the arguments first, as em_collocation_labels checks them, then the buffer's size
    int rc = check_em_args(sde, theta, Yi, dt, n_rows, n_paths, n_fine);
    if (rc) return rc;
    if (!labels) return set_error(SL_ERR_ARG, "labels == NULL");
    if (n_paths < 1) return set_error(SL_ERR_ARG, "n_paths < 1");
    int64_t ranks[SL_MAX_M];
    rc = sl_quantile_ranks(m, n_paths, ranks);
    if (rc) return rc;
    const size_t need = sl_em_labels_workspace_size(n_rows, n_paths, m);
    if (need > kNoAllocBytes)
        return set_error(SL_ERR_WORKSPACE,
                         "n_rows * n_paths = %lld samples exceeds the fixed no-allocation buffer (%zu samples); "
                         "use em_collocation_labels with a caller workspace",
                         static_cast<long long>(n_rows) * n_paths, sl_em_labels_noalloc_max_samples());
    void* ws = nullptr;
    rc = noalloc_address(&ws);
    if (rc) return rc;
    // em_collocation_labels clears the status word and overwrites every sample it reads.
    return em_collocation_labels(sde, theta, Yi, dt, n_rows, n_paths, n_fine, m, seed, labels, ws,
                                 kNoAllocBytes, stream);
}

}  // extern "C"
