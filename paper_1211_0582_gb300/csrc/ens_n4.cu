// Persistent ensemble kernels (autotuner candidates) for polynomial order 4.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<4>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n4(int i) { return EnsembleCandidates<4>::c(i); }
} // namespace dgmx
