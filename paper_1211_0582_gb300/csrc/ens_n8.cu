// Persistent ensemble kernels (autotuner candidates) for polynomial order 8.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<8>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n8(int i) { return EnsembleCandidates<8>::c(i); }
} // namespace dgmx
