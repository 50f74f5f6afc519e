// Persistent ensemble kernels (autotuner candidates) for polynomial order 9.
#include "ensemble.cuh"

namespace dgmx {
template cudaError_t launch_ensemble_order<9>(int, const StageArgs &, const StageCoeffs &, float *, float *, int,
                                               GridBarrier *, int *, cudaStream_t, int, int *);
int ensemble_candidate_eb_n9(int i) { return EnsembleCandidates<9>::c(i); }
} // namespace dgmx
