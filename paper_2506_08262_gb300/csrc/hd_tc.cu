// Tensor-core halfspace path (placeholder until the tcgen05 kernel lands).
#include "rrs_internal.h"

namespace rrs {

float band_gamma_tc(int d) { (void)d; return 1e-4f; }
bool hd_tc_supported(int d) { (void)d; return false; }

cudaError_t launch_build_bf16_planes(const float*, int64_t, int, int, int, uint16_t*, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t launch_hd_tc(const TaskDev*, int, const SlotDev*, const DsDev*, const float*, const double*,
                         const double*, ResDev*, int64_t*, int*, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace rrs
