// Discrete electromagnetic energy 1/2 sum_k J_k (eps_k E^T M E + mu_k H^T M H),
// reduced in FP64 on the device. The (field, element) rows of the field vector
// are processed in tiles of PB consecutive rows (one contiguous span of memory,
// staged in shared memory with 16-byte loads); a thread forms four entries
// (M q)_i, i = 4t..4t+3, of one row from the transposed mass matrix in shared
// memory, multiplies them with q_i, and the row's partial sums are added up per
// tile in shared memory (FP64) before one FP64 atomic per tile. The products
// (M q)_i are formed in FP32 (the fields are FP32); every sum over nodes,
// fields and elements is carried in FP64.
#include "common.cuh"

namespace dgmx {

namespace {

constexpr int kEnergyThreads = 256;

__global__ void __launch_bounds__(kEnergyThreads)
    k_energy(int Np, int Npad, int64_t K, const float *__restrict__ u, const float *__restrict__ geo,
             const double *__restrict__ M, double *out) {
  extern __shared__ float4 s_mem4[];
  const int NQ = Npad / 4;
  const int PB = kEnergyThreads / NQ; // rows per tile
  float *s_MT = reinterpret_cast<float *>(s_mem4);                 // [Np][Npad]: s_MT[j][i] = M[i][j]
  float *s_q = s_MT + Np * Npad;                                  // [PB][Npad]
  double *s_part = reinterpret_cast<double *>(s_q + PB * Npad);   // [kEnergyThreads]
  for (int t = threadIdx.x; t < Np * Npad; t += blockDim.x) {
    const int j = t / Npad, i = t - j * Npad;
    s_MT[t] = i < Np ? float(M[i * Np + j]) : 0.f;
  }
  const int tid = threadIdx.x;
  const int ps = tid / NQ, q = tid - (tid / NQ) * NQ;
  const int64_t rows = 6 * K;
  double total = 0.0;
  for (int64_t p0 = int64_t(blockIdx.x) * PB; p0 < rows; p0 += int64_t(gridDim.x) * PB) {
    const int nr = int(rows - p0 < PB ? rows - p0 : PB);
    __syncthreads(); // the previous tile's rows are no longer read
    const float4 *src = reinterpret_cast<const float4 *>(u + p0 * Npad);
    for (int t = tid; t < nr * NQ; t += blockDim.x) reinterpret_cast<float4 *>(s_q)[t] = __ldg(src + t);
    __syncthreads();
    double part = 0.0;
    if (ps < nr) {
      const float *qr = s_q + ps * Npad;
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
      for (int j = 0; j < Np; ++j) {
        const float4 mt = *reinterpret_cast<const float4 *>(s_MT + j * Npad + 4 * q);
        const float qj = qr[j];
        m0 = fmaf(mt.x, qj, m0);
        m1 = fmaf(mt.y, qj, m1);
        m2 = fmaf(mt.z, qj, m2);
        m3 = fmaf(mt.w, qj, m3);
      }
      const float mv[4] = {m0, m1, m2, m3};
      for (int r = 0; r < 4; ++r)
        if (4 * q + r < Np) part += double(mv[r]) * double(qr[4 * q + r]);
    }
    s_part[tid] = part;
    __syncthreads();
    if (tid < nr) {
      double acc = 0.0;
      for (int t = 0; t < NQ; ++t) acc += s_part[tid * NQ + t];
      const int64_t p = p0 + tid;
      const int c = int(p / K);
      const int64_t k = p - int64_t(c) * K;
      const float *g = geo + k * G_STRIDE;
      const double w = c < 3 ? 1.0 / double(g[G_IEPS]) : 1.0 / double(g[G_IMU]);
      total += 0.5 * double(g[G_J]) * w * acc;
    }
  }
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if ((tid & 31) == 0 && total != 0.0) atomicAdd(out, total);
}

// Sets *flag to 1 if any of the n4 float4 values holds a NaN or an infinity.
__global__ void __launch_bounds__(256) k_nonfinite(const float4 *__restrict__ u, int64_t n4, int *flag) {
  bool bad = false;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
    const float4 v = __ldg(u + i);
    bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

} // namespace

cudaError_t launch_nonfinite_check(const float *u, int64_t nfloats, int *flag, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n4 = nfloats / 4;
  int64_t blocks = (n4 + 255) / 256;
  if (blocks > int64_t(sms) * 8) blocks = int64_t(sms) * 8;
  if (blocks < 1) blocks = 1;
  k_nonfinite<<<unsigned(blocks), 256, 0, s>>>(reinterpret_cast<const float4 *>(u), n4, flag);
  return cudaGetLastError();
}

cudaError_t launch_energy(int N, int64_t K, int Npad, const float *u, const float *geo, const double *M, double *out,
                          cudaStream_t s) {
  const int Np = num_nodes(N);
  const int NQ = Npad / 4, PB = kEnergyThreads / NQ;
  const size_t smem = size_t(Np) * Npad * sizeof(float) + size_t(PB) * Npad * sizeof(float) +
                      size_t(kEnergyThreads) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (6 * K + PB - 1) / PB;
  const int64_t cap = int64_t(sms) * 4;
  unsigned blocks = unsigned(tiles < cap ? tiles : cap);
  if (blocks == 0) blocks = 1;
  k_energy<<<blocks, kEnergyThreads, smem, s>>>(Np, Npad, K, u, geo, M, out);
  return cudaGetLastError();
}

} // namespace dgmx
