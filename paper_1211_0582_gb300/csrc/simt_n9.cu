// FP32 fused stage kernels for polynomial order 9.
#include "simt_stage.cuh"

namespace dgmx {
template cudaError_t launch_simt_order<9>(int, const StageArgs &, cudaStream_t);
} // namespace dgmx
