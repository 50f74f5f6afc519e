// Persistent ensemble kernels (autotuner candidates) for polynomial order 6.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<6>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n6(int i) { return EnsembleCandidates<6>::c(i); }
} // namespace dgmx
