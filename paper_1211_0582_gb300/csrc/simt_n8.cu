// FP32 fused stage kernels for polynomial order 8.
#include "simt_stage.cuh"

namespace dgmx {
template cudaError_t launch_simt_order<8>(int, const StageArgs &, cudaStream_t);
} // namespace dgmx
