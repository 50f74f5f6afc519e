// Persistent ensemble kernels (autotuner candidates) for polynomial order 3.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<3>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n3(int i) { return EnsembleCandidates<3>::c(i); }
} // namespace dgmx
