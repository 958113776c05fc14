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

// ------------------------------------------------ Krylov variants on S (FP64)
// out = beta * out + alpha * J^T y   (J^T by column, original labels; no atomics)
__global__ void k_jt_mult(int64_t n, const int64_t* __restrict__ tp, const int32_t* __restrict__ trow,
                          const int32_t* __restrict__ tv, const double* __restrict__ Jv, const double* __restrict__ y,
                          double alpha, double beta, double* __restrict__ out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t q = tp[c]; q < tp[c + 1]; q++) s += Jv[tv[q]] * y[trow[q]];
    out[c] = (beta == 0.0 ? 0.0 : beta * out[c]) + alpha * s;
  }
}
// out = beta * out + alpha * J x
__global__ void k_j_mult(int64_t m, const int64_t* __restrict__ jp, const int32_t* __restrict__ jc,
                         const double* __restrict__ Jv, const double* __restrict__ x, double alpha, double beta,
                         double* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t q = jp[r]; q < jp[r + 1]; q++) s += Jv[q] * x[jc[q]];
    out[r] = (beta == 0.0 ? 0.0 : beta * out[r]) + alpha * s;
  }
}
// out = H~ x + delta x (H~ from its full symmetric pattern, original labels)
__global__ void k_hsym_mult(int64_t n, const int64_t* __restrict__ hp, const int32_t* __restrict__ hc,
                            const int32_t* __restrict__ hv, const double* __restrict__ Hv, const double* __restrict__ x,
                            double delta, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = delta * x[i];
    for (int64_t q = hp[i]; q < hp[i + 1]; q++) s += Hv[hv[q]] * x[hc[q]];
    out[i] = s;
  }
}
// y = a * x + b * y
__global__ void k_axpby(int64_t N, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = a * x[k] + (b == 0.0 ? 0.0 : b * y[k]);
}
// lower values of J J^T: entry e = sum of J[qa] J[qb] over its pairs
__global__ void k_jjt_values(int64_t ne, const int64_t* __restrict__ pp, const int32_t* __restrict__ pa,
                             const int32_t* __restrict__ pb, const double* __restrict__ Jv, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t q = pp[e]; q < pp[e + 1]; q++) s += Jv[pa[q]] * Jv[pb[q]];
    out[e] = s;
  }
}

// ------------------------------------------------ FGMRES coefficients on the device
// State (doubles): H[(R+1) x R] row-major with row stride R, cs[R], sn[R],
// g[R+1], hcol[R+1], then flag (1.0 when the cycle may stop). One thread.
//   mode 0: hcol = dots;            coef = -dots       (first Gram-Schmidt pass)
//   mode 1: hcol += dots;           coef = -dots       (reorthogonalisation)
//   mode 2: hn = sqrt(max(dots[0], 0)); column k of H = -hcol, H[k+1][k] = hn;
//           previous rotations, new rotation, g update; coef[0] = -1/hn (0 if
//           hn = 0); flag = |g[k+1]| <= tol or hn = 0
//   mode 3: coef = the solution y of the k x k upper triangle H y = g
//   mode 4: start of a cycle: g = (rnorm, 0, ...), coef[0] = 1/rnorm, flag = 0
__global__ void k_fgmres_coef(int mode, int k, int R, const double* __restrict__ dots, const DevStatus* st,
                              double tol, double* __restrict__ gs, double* __restrict__ coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* H = gs;
  double* cs = H + (R + 1) * R;
  double* sn = cs + R;
  double* g = sn + R;
  double* hcol = g + R + 1;
  double* flag = hcol + R + 1;
  if (mode == 0 || mode == 1) {
    for (int i = 0; i <= k; i++) {
      hcol[i] = mode == 0 ? dots[i] : hcol[i] + dots[i];
      coef[i] = -dots[i];
    }
  } else if (mode == 2) {
    const double hn = sqrt(fmax(dots[0], 0.0));
    for (int i = 0; i <= k; i++) H[i * R + k] = -hcol[i];
    H[(k + 1) * R + k] = hn;
    for (int i = 0; i < k; i++) {
      const double t = cs[i] * H[i * R + k] + sn[i] * H[(i + 1) * R + k];
      H[(i + 1) * R + k] = -sn[i] * H[i * R + k] + cs[i] * H[(i + 1) * R + k];
      H[i * R + k] = t;
    }
    const double den = hypot(H[k * R + k], H[(k + 1) * R + k]);
    cs[k] = den > 0 ? H[k * R + k] / den : 1.0;
    sn[k] = den > 0 ? H[(k + 1) * R + k] / den : 0.0;
    H[k * R + k] = den;
    H[(k + 1) * R + k] = 0.0;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    coef[0] = hn > 0 ? -1.0 / hn : 0.0;
    *flag = (fabs(g[k + 1]) <= tol || hn == 0.0) ? 1.0 : 0.0;
    flag[1] = fabs(sn[k]);   // this step's residual contraction |g[k+1]| / |g[k]|
  } else if (mode == 3) {
    for (int i = k - 1; i >= 0; i--) {
      double t = g[i];
      for (int j = i + 1; j < k; j++) t -= H[i * R + j] * coef[j];
      coef[i] = H[i * R + i] != 0.0 ? t / H[i * R + i] : 0.0;
    }
  } else {
    const double rn = st->res_norm;
    for (int i = 0; i <= R; i++) g[i] = 0.0;
    g[0] = rn;
    coef[0] = rn > 0 ? 1.0 / rn : 0.0;
    *flag = 0.0;
  }
}

cudaError_t launch_fgmres_coef(int mode, int k, int R, const double* dots, const DevStatus* st, double tol, double* gs,
                               double* coef, cudaStream_t s) {
  k_fgmres_coef<<<1, 32, 0, s>>>(mode, k, R, dots, st, tol, gs, coef);
  return cudaGetLastError();
}

cudaError_t launch_jt_mult(int64_t n, const int64_t* tp, const int32_t* trow, const int32_t* tv, const double* Jv,
                           const double* y, double alpha, double beta, double* out, cudaStream_t st) {
  k_jt_mult<<<krylov_grid(n), kKrylovThreads, 0, st>>>(n, tp, trow, tv, Jv, y, alpha, beta, out);
  return cudaGetLastError();
}
cudaError_t launch_j_mult(int64_t m, const int64_t* jp, const int32_t* jc, const double* Jv, const double* x,
                          double alpha, double beta, double* out, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  k_j_mult<<<krylov_grid(m), kKrylovThreads, 0, st>>>(m, jp, jc, Jv, x, alpha, beta, out);
  return cudaGetLastError();
}
cudaError_t launch_hsym_mult(int64_t n, const int64_t* hp, const int32_t* hc, const int32_t* hv, const double* Hv,
                             const double* x, double delta, double* out, cudaStream_t st) {
  k_hsym_mult<<<krylov_grid(n), kKrylovThreads, 0, st>>>(n, hp, hc, hv, Hv, x, delta, out);
  return cudaGetLastError();
}
cudaError_t launch_axpby(int64_t N, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_axpby<<<krylov_grid(N), kKrylovThreads, 0, st>>>(N, a, x, b, y);
  return cudaGetLastError();
}
cudaError_t launch_jjt_values(int64_t ne, const int64_t* pp, const int32_t* pa, const int32_t* pb, const double* Jv,
                              double* out, cudaStream_t st) {
  if (ne == 0) return cudaSuccess;
  k_jjt_values<<<krylov_grid(ne), kKrylovThreads, 0, st>>>(ne, pp, pa, pb, Jv, out);
  return cudaGetLastError();
}

}  // namespace kkt
