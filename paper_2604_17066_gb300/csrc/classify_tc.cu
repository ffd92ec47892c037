// classify_tc.cu -- placeholder until the tcgen05 path lands.
#include "rsr_launch.h"
namespace rsr {
bool tc_supported() { return false; }
cudaError_t launch_encode_tc(const uint8_t *, int64_t, int64_t, int, int, int, bool, uint8_t *, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_classify_tc(const ClassifyParams &, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace rsr
