// Symmetrized Ruiz scaling of the 2x2 KKT system (Sec. 4.1: the system is
// scaled before gamma and delta are judged against it; D. Ruiz, "A scaling
// algorithm to equilibrate both rows and columns norms in matrices",
// RAL-TR-2001-034, 2001).
//
// K = [H~, J^T; J, 0] is symmetric, so one diagonal D = diag(D_x, D_y)
// scales rows and columns alike: D = I, then per iteration every row's
// infinity norm r_i = max_j (D_i |K_ij|) D_j of the current D K D is taken
// (all rows from the same D) and D_i <- D_i / sqrt(r_i) where r_i > 0. The
// products are formed in that order (row factor first) and only multiplied,
// maxed, square-rooted and divided, so the result does not depend on the
// summation order: it is the same on any device. The handle then holds the
// scaled values D_x H~ D_x and D_y J D_x; right-hand sides are scaled by D
// and solutions unscaled by D.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace kkt {

// one row of K per thread: H~ rows from the full symmetric pattern (original
// labels) and the J^T part, J rows from the CSR
__global__ void k_ruiz_rows(RuizArgs a, const double* __restrict__ Dold, double* __restrict__ Dnew) {
  const int64_t N = a.n + a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double di = Dold[i];
    double r = 0.0;
    if (i < a.n) {
      for (int64_t q = a.Hs_ptr[i]; q < a.Hs_ptr[i + 1]; q++)
        r = fmax(r, (di * fabs(a.Hv[a.Hs_vidx[q]])) * Dold[a.Hs_col[q]]);
      for (int64_t q = a.JT_ptr[i]; q < a.JT_ptr[i + 1]; q++)
        r = fmax(r, (di * fabs(a.Jv[a.JT_vidx[q]])) * Dold[a.n + a.JT_row[q]]);
    } else {
      const int64_t row = i - a.n;
      for (int64_t q = a.J_rowptr[row]; q < a.J_rowptr[row + 1]; q++)
        r = fmax(r, (di * fabs(a.Jv[q])) * Dold[a.J_colidx[q]]);
    }
    Dnew[i] = r > 0.0 ? di / sqrt(r) : di;
  }
}

// H~ (lower CSC, one column per thread) and J (one row per thread) scaled in place
__global__ void k_scale_values(RuizArgs a, const double* __restrict__ D, double* __restrict__ Hv,
                               double* __restrict__ Jv) {
  const int64_t N = a.n + a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < a.n) {
      const double dj = D[t];
      for (int64_t q = a.H_colptr[t]; q < a.H_colptr[t + 1]; q++) Hv[q] = (D[a.H_rowidx[q]] * Hv[q]) * dj;
    } else {
      const int64_t row = t - a.n;
      const double dr = D[t];
      for (int64_t q = a.J_rowptr[row]; q < a.J_rowptr[row + 1]; q++) Jv[q] = (dr * Jv[q]) * D[a.J_colidx[q]];
    }
  }
}

// y = D .* x over [x (n); x (m)] given as two parts
__global__ void k_scale_vec(int64_t n, int64_t m, const double* __restrict__ D, const double* __restrict__ xx,
                            const double* __restrict__ xy, double* __restrict__ yx, double* __restrict__ yy) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) yx[i] = D[i] * xx[i];
    else yy[i - n] = D[i] * xy[i - n];
  }
}

// D (n + m doubles) from the values in a.Hv / a.Jv, then the values scaled
// in place (Hv, Jv are the same arrays as a.Hv, a.Jv); Dtmp is scratch.
cudaError_t launch_ruiz(const RuizArgs& a, int iters, double* D, double* Dtmp, double* Hv, double* Jv,
                        cudaStream_t st) {
  const int64_t N = a.n + a.m;
  const int threads = 256;
  int64_t blocks = (N + threads - 1) / threads;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (blocks < 1) blocks = 1;
  cudaError_t e = cudaMemcpyAsync(D, a.ones, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  if (e) return e;
  double* cur = D;
  double* nxt = Dtmp;
  for (int k = 0; k < iters; k++) {
    k_ruiz_rows<<<(unsigned)blocks, threads, 0, st>>>(a, cur, nxt);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != D && (e = cudaMemcpyAsync(D, cur, sizeof(double) * N, cudaMemcpyDeviceToDevice, st))) return e;
  k_scale_values<<<(unsigned)blocks, threads, 0, st>>>(a, D, Hv, Jv);
  return cudaGetLastError();
}

cudaError_t launch_scale_vec(int64_t n, int64_t m, const double* D, const double* xx, const double* xy, double* yx,
                             double* yy, cudaStream_t st) {
  const int threads = 256;
  int64_t blocks = (n + m + threads - 1) / threads;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (blocks < 1) blocks = 1;
  k_scale_vec<<<(unsigned)blocks, threads, 0, st>>>(n, m, D, xx, xy, yx, yy);
  return cudaGetLastError();
}

}  // namespace kkt
