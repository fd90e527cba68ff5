// sl_selftest.cu -- a self-test of the kernels' bounded waits.
//
// Every mbarrier wait in the tensor-core kernels gives up after about one
// second of global time, records SL_DEV_TIMEOUT in the workspace status word
// and lets the kernel finish, so a lost completion becomes an error status on
// the host instead of a hung GPU.  This entry point exercises that path on
// purpose: one warp waits, with the kernels' own wait routine, on a shared
// memory mbarrier that nothing ever arrives on.
#include "sl_tc_common.cuh"

namespace sl {
namespace {

using namespace tc;

__global__ void wait_timeout_kernel(unsigned* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // phase 0 never completes: no thread arrives and no MMA commits to it
    const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, status);
    if (__all_sync(0xffffffffu, !ok) == 0 && threadIdx.x == 0) raise_status(status, SL_DEV_NONFINITE);
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" {

int sl_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < kStatusBytes) return set_error(SL_ERR_WORKSPACE, "workspace %zu < %zu", ws_bytes, kStatusBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(ws);
    int rc = cuda_error(cudaMemsetAsync(status, 0, kStatusBytes, st), "status clear");
    if (rc) return rc;
    wait_timeout_kernel<<<1, 32, 0, st>>>(status);
    return cuda_error(cudaGetLastError(), "wait_timeout launch");
}

}  // extern "C"
