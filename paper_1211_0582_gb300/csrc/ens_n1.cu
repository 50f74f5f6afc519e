// Persistent ensemble kernels (autotuner candidates) for polynomial order 1.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<1>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n1(int i) { return EnsembleCandidates<1>::c(i); }
} // namespace dgmx
