// sl_tc.cu -- placeholder until the tcgen05 form lands.
#include "sl_internal.cuh"
namespace sl {
int launch_tc_7l(int m, const SimArgs& a, cudaStream_t s) {
    (void)m; (void)a; (void)s;
    return set_error(SL_ERR_UNSUPPORTED, "BF16 tensor-core form not built");
}
}  // namespace sl
