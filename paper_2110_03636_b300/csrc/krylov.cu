// FP64 vector kernels of the flexible-GMRES refinement on K_delta: several
// inner products against one vector in one pass (fixed summation order, so
// every run adds in the same order), and linear combinations of stored basis
// vectors. All are HBM-bound streams over vectors of n + m doubles.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace kkt {

constexpr int kKrylovThreads = 256;

// part[b * cnt + i] = sum over block b's share of k of w[k] * V[i * ld + k]
__global__ void __launch_bounds__(kKrylovThreads) k_multidot(const double* __restrict__ w,
                                                             const double* __restrict__ V, int64_t ld, int64_t N,
                                                             int cnt, double* __restrict__ part) {
  __shared__ double red[kKrylovThreads / 32][kMaxKrylov];
  double acc[kMaxKrylov];
#pragma unroll
  for (int i = 0; i < kMaxKrylov; i++) acc[i] = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const double wk = w[k];
#pragma unroll
    for (int i = 0; i < kMaxKrylov; i++)
      if (i < cnt) acc[i] += wk * V[i * ld + k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kMaxKrylov; i++) {
    if (i >= cnt) break;
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < kKrylovThreads / 32; q++) s += red[q][threadIdx.x];
    part[blockIdx.x * cnt + threadIdx.x] = s;
  }
}

// out[i] = sum over blocks of part[b * cnt + i], blocks in ascending order
__global__ void k_multidot_final(const double* __restrict__ part, int blocks, int cnt, double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= cnt) return;
  double s = 0.0;
  for (int b = 0; b < blocks; b++) s += part[b * cnt + i];
  out[i] = s;
}

// y[k] = alpha * y[k] + sum_{i < cnt} c[i] * V[i * ld + k]   (k < N)
__global__ void __launch_bounds__(kKrylovThreads) k_lincomb(double* __restrict__ y, double alpha,
                                                            const double* __restrict__ V, int64_t ld, int64_t N,
                                                            int cnt, const double* __restrict__ c) {
  __shared__ double cs[kMaxKrylov];
  if (threadIdx.x < cnt) cs[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    double v = alpha == 0.0 ? 0.0 : alpha * y[k];
    for (int i = 0; i < cnt; i++) v += cs[i] * V[i * ld + k];
    y[k] = v;
  }
}

static unsigned krylov_grid(int64_t N) {
  const int64_t b = (N + kKrylovThreads - 1) / kKrylovThreads;
  return (unsigned)(b < 296 ? (b < 1 ? 1 : b) : 296);
}

cudaError_t launch_multidot(const double* w, const double* V, int64_t ld, int64_t N, int cnt, double* part,
                            double* out, cudaStream_t st) {
  if (cnt < 1 || cnt > kMaxKrylov) return cudaErrorInvalidValue;
  const unsigned g = krylov_grid(N);
  k_multidot<<<g, kKrylovThreads, 0, st>>>(w, V, ld, N, cnt, part);
  k_multidot_final<<<1, 32, 0, st>>>(part, (int)g, cnt, out);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(double* y, double alpha, const double* V, int64_t ld, int64_t N, int cnt, const double* c,
                           cudaStream_t st) {
  if (cnt < 0 || cnt > kMaxKrylov) return cudaErrorInvalidValue;
  k_lincomb<<<krylov_grid(N), kKrylovThreads, 0, st>>>(y, alpha, V, ld, N, cnt, c);
  return cudaGetLastError();
}

}  // namespace kkt
