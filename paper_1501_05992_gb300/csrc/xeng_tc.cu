// X-engine, tcgen05 FP8 form (K2c).  Placeholder until the tensor-core
// kernel lands: reports the path as unsupported.
#include "internal.cuh"

namespace corr {

bool tc_supported(int, int) { return false; }

cudaError_t launch_xeng_tc(const uint8_t *, int, int, int, bool, int32_t *, bool,
                           DeviceStatus *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace corr
