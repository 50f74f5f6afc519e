// Discrete electromagnetic energy 1/2 sum_k J_k (eps_k E^T M E + mu_k H^T M H),
// reduced in FP64 on the device (one warp per element and field, the mass
// matrix in shared memory, warp-shuffle reduction, one FP64 atomic per warp).
// The row products (M q)_i are formed in FP32 (the fields are FP32); every
// sum over nodes, fields and elements is carried in FP64.
#include "common.cuh"

namespace dgmx {

namespace {

__global__ void k_energy(int Np, int Npad, int64_t K, const float *__restrict__ u, const float *__restrict__ geo,
                         const double *__restrict__ M, double *out) {
  extern __shared__ float s_M[];
  for (int i = threadIdx.x; i < Np * Np; i += blockDim.x) s_M[i] = float(M[i]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int64_t pairs = 6 * K;
  double total = 0.0;
  for (int64_t p = int64_t(blockIdx.x) * warps + (threadIdx.x >> 5); p < pairs; p += int64_t(gridDim.x) * warps) {
    int c = int(p / K);
    int64_t k = p - int64_t(c) * K;
    const float *q = u + (int64_t(c) * K + k) * Npad;
    double acc = 0.0;
    for (int i = lane; i < Np; i += 32) {
      float mi = 0.f;
      for (int j = 0; j < Np; ++j) mi = fmaf(s_M[i * Np + j], __ldg(q + j), mi);
      acc += double(mi) * double(q[i]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float *g = geo + k * G_STRIDE;
    double w = c < 3 ? 1.0 / double(g[G_IEPS]) : 1.0 / double(g[G_IMU]);
    total += 0.5 * double(g[G_J]) * w * acc;
  }
  if (lane == 0) atomicAdd(out, total);
}

} // namespace

cudaError_t launch_energy(int N, int64_t K, int Npad, const float *u, const float *geo, const double *M, double *out,
                          cudaStream_t s) {
  int Np = num_nodes(N);
  size_t smem = size_t(Np) * Np * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (6 * K + 7) / 8;
  unsigned blocks = unsigned(want < int64_t(sms) * 4 ? want : int64_t(sms) * 4);
  if (blocks == 0) blocks = 1;
  k_energy<<<blocks, 256, smem, s>>>(Np, Npad, K, u, geo, M, out);
  return cudaGetLastError();
}

} // namespace dgmx
