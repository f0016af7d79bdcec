// Tensor-core power step for the complex64 Taylor series (placeholder until
// the tcgen05 kernel is in: the FP64 GEMM serves both paths meanwhile).
#include "internal.h"

bool tc_gemm_available() { return false; }

hw_status launch_tc_power_step(int, const float *, const float *, float, float *, double *, double, int,
                               cudaStream_t)
{
    return hw_fail(HW_EUNSUPPORTED, "tensor-core power step not built");
}
