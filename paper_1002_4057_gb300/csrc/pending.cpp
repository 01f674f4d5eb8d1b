// Entry points whose kernels are not in this build yet.
#include "../../include/spdinv.h"
#include "api_internal.h"

namespace spdinv {
spdinv_status run_mixed(int64_t, double*, int64_t, const spdinv_opts*, int*, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
}  // namespace spdinv

extern "C" {
spdinv_status spdinv_potri_batched(int, const int*, double* const*, const int*, int*, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
spdinv_status spdinv_spotri_batched(int, const int*, float* const*, const int*, int*, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
spdinv_status spdinv_potri_backward(int, int64_t, const double*, int64_t, int64_t, const double*, int64_t, int64_t,
                                    double*, int64_t, int64_t, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
spdinv_status spdinv_spotri_backward(int, int64_t, const float*, int64_t, int64_t, const float*, int64_t, int64_t,
                                     float*, int64_t, int64_t, cudaStream_t) {
    return SPDINV_ERR_UNSUPPORTED;
}
}
