// Grid-wide synchronisation of a persistent cooperative launch (all blocks
// resident), shared by the ensemble kernels: a generation barrier with a
// bounded wait, and the LSERK4 stage coefficients those kernels loop over.
#pragma once
#include <cuda_runtime.h>

namespace dgmx {

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Sense-free generation barrier over all blocks of a cooperative launch.
// Gives up after `limit` cycles and returns false.
__device__ __forceinline__ bool grid_barrier(GridBarrier *gb, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *vgen = &gb->gen;
    const unsigned int my_gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      gb->count = 0u;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == my_gen) {
        if (clock64() - t0 > limit) {
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct StageCoeffs {
  float a[5], b[5];
};

} // namespace dgmx
