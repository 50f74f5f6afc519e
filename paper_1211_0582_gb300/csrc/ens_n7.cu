// Persistent ensemble kernels (autotuner candidates) for polynomial order 7.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<7>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n7(int i) { return EnsembleCandidates<7>::c(i); }
} // namespace dgmx
