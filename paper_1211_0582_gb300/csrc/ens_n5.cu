// Persistent ensemble kernels (autotuner candidates) for polynomial order 5.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<5>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n5(int i) { return EnsembleCandidates<5>::c(i); }
} // namespace dgmx
