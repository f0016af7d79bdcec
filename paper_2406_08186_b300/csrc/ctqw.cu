// Continuous-time walk (Sec. 3.1): placeholder until the kernels land.
#include "internal.h"

extern "C" hw_status hw_ctqw_expm(const hw_graph *, double, const int32_t *, int32_t, double, hw_dtype,
                                  void *, const hw_opts *, void *)
{
    hw_clear_error();
    return hw_fail(HW_EUNSUPPORTED, "hw_ctqw_expm not built yet");
}

extern "C" hw_status hw_ctqw_evolve(const void *, int64_t, hw_dtype, int32_t, int64_t, const void *, void *,
                                    const int32_t *, int32_t, double *, const hw_opts *, void *)
{
    hw_clear_error();
    return hw_fail(HW_EUNSUPPORTED, "hw_ctqw_evolve not built yet");
}
