// Persistent ensemble kernels (autotuner candidates) for polynomial order 2.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<2>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n2(int i) { return EnsembleCandidates<2>::c(i); }
} // namespace dgmx
