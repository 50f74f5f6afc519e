// FP32 fused stage kernels for polynomial order 3.
#include "simt_stage.cuh"

namespace dgmx {
template cudaError_t launch_simt_order<3>(int, const StageArgs &, cudaStream_t);
} // namespace dgmx
