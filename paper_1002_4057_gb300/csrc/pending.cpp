// Entry points whose kernels are not in this build yet.
#include "../../include/spdinv.h"
#include "api_internal.h"

namespace spdinv {
spdinv_status run_mixed(int64_t, double*, int64_t, const spdinv_opts*, int*, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
}  // namespace spdinv
