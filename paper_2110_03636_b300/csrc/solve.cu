// Persistent, cooperative CG on the Schur complement (eqs. Schur1/Schur2 and
// Algorithm 1's solve steps):
//   r^_x = r_x + gamma J^T r_y;  w = H^-1 r^_x;  b_S = J w - r_y;
//   CG on (S + d2 I) dy = b_S with S = J H^-1 J^T, one product per iteration
//   = J^T p, forward and backward triangular solves with L, J (Sec. 4.1);
//   dx = H^-1 (r^_x - J^T dy).
// Everything runs inside one kernel launch: no host round trip inside CG.
// Grid-wide phases are separated by a software grid barrier; the triangular
// solves are dependency-driven sweeps over "pieces" (column ranges of at most
// solve_w columns of one supernode) and "chunks" (row ranges of a piece's
// off-diagonal block), handed out in a fixed topological order through an
// atomic ticket. Every wait is bounded (DevStatus::abort on timeout).
// The CG recurrences, dot products and scalars are FP64 in both precisions;
// T is the storage/arithmetic type of L and of the triangular-solve vector.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace kkt {

constexpr int kSolveThreads = 256;
constexpr int kSWMax = 256;

template <typename T>
struct SolveSmem {
  T vec[kSWMax];
  T aux[kSolveThreads];
  double dred[(kSolveThreads / 32) * 2];
  double bcast[2];
  int item;
  int flag;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ bool grid_barrier(const SolveArgs<T>& a, SolveSmem<T>& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const int gen = ld_acquire(&a.bar[1]);
    __threadfence();
    if (atomicAdd(&a.bar[0], 1) == (int)gridDim.x - 1) {
      atomicExch(&a.bar[0], 0);
      __threadfence();
      st_release(&a.bar[1], gen + 1);
    } else {
      ok = wait_geq(&a.bar[1], gen + 1, a.st, a.spin) ? 1 : 0;
    }
    if (ld_acquire(&a.st->abort)) ok = 0;
    sm.flag = ok;
  }
  __syncthreads();
  return sm.flag != 0;
}

// per-block partial sums of two values -> a.red[block*4 + {0,1}]
template <typename T>
__device__ void block_partial2(const SolveArgs<T>& a, SolveSmem<T>& sm, double v0, double v1) {
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sm.dred[warp * 2] = v0; sm.dred[warp * 2 + 1] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < kSolveThreads / 32; w++) { s0 += sm.dred[w * 2]; s1 += sm.dred[w * 2 + 1]; }
    a.red[blockIdx.x * 4] = s0;
    a.red[blockIdx.x * 4 + 1] = s1;
  }
}

// the same grid totals in every block (fixed summation order)
template <typename T>
__device__ void grid_total2(const SolveArgs<T>& a, SolveSmem<T>& sm, double& t0, double& t1) {
  if (threadIdx.x < 32) {
    double s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
      s0 += __ldcg(&a.red[b * 4]);
      s1 += __ldcg(&a.red[b * 4 + 1]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (threadIdx.x == 0) { sm.bcast[0] = s0; sm.bcast[1] = s1; }
  }
  __syncthreads();
  t0 = sm.bcast[0];
  t1 = sm.bcast[1];
  __syncthreads();
}

// --------------------------------------------------------------- forward
template <typename T>
__device__ bool fwd_head(const SolveArgs<T>& a, SolveSmem<T>& sm, int p, int e) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.flag = wait_geq(&a.fwd_arrive[p], e * a.pc_need[p], a.st, a.spin);
  __syncthreads();
  if (!sm.flag) return false;
  const int pw = a.pc_w[p], ld = a.pc_ld[p], f = a.pc_first[p];
  const T* Lp = a.L + a.pc_off[p];
  T* vec = sm.vec;
  for (int i = tid; i < pw; i += blockDim.x) vec[i] = ldcg(&a.v[f + i]);
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  for (int jb = 0; jb < pw; jb += 32) {
    const int bwb = min(32, pw - jb);
    if (warp == 0) {
      T Lr[32];
#pragma unroll
      for (int k = 0; k < 32; k++)
        Lr[k] = (lane < bwb && k <= lane) ? Lp[(int64_t)(jb + lane) + (int64_t)(jb + k) * ld] : T(0);
      T val = lane < bwb ? vec[jb + lane] : T(0);
#pragma unroll
      for (int j = 0; j < 32; j++) {
        if (j < bwb) {
          if (lane == j) val = val / Lr[j];
          const T yj = __shfl_sync(0xffffffffu, val, j);
          if (lane > j) val -= Lr[j] * yj;
        }
      }
      if (lane < bwb) vec[jb + lane] = val;
    }
    __syncthreads();
    for (int i = jb + bwb + tid; i < pw; i += blockDim.x) {
      T acc = T(0);
      for (int k = 0; k < bwb; k++) acc += Lp[(int64_t)i + (int64_t)(jb + k) * ld] * vec[jb + k];
      vec[i] -= acc;
    }
    __syncthreads();
  }
  for (int i = tid; i < pw; i += blockDim.x) a.v[f + i] = vec[i];
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(&a.fwd_done[p], e);
  return true;
}

template <typename T>
__device__ bool fwd_chunk(const SolveArgs<T>& a, SolveSmem<T>& sm, int c, int e) {
  const int tid = threadIdx.x;
  const int p = a.ch_piece[c];
  if (tid == 0) sm.flag = wait_geq(&a.fwd_done[p], e, a.st, a.spin);
  __syncthreads();
  if (!sm.flag) return false;
  const int pw = a.pc_w[p], ld = a.pc_ld[p], f = a.pc_first[p];
  const int r0 = a.ch_r0[c], nr = a.ch_nr[c];
  const T* Lp = a.L + a.pc_off[p];
  T* vec = sm.vec;
  for (int k = tid; k < pw; k += blockDim.x) vec[k] = ldcg(&a.v[f + k]);
  __syncthreads();
  const int nrr = (nr + 31) & ~31;
  const int G = max(1, (int)blockDim.x / nrr);
  const int i = tid % nrr, g = tid / nrr;
  T acc = T(0);
  if (g < G && i < nr)
    for (int k = g; k < pw; k += G) acc += Lp[(int64_t)(r0 + i) + (int64_t)k * ld] * vec[k];
  sm.aux[tid] = acc;
  __syncthreads();
  if (tid < nr) {
    T s = T(0);
    for (int gg = 0; gg < G; gg++) s += sm.aux[gg * nrr + tid];
    const int row = a.sn_rows[a.pc_row[p] + r0 + tid];
    atomicAdd(&a.v[row], -s);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0)
    for (int64_t t = a.ch_tptr[c]; t < a.ch_tptr[c + 1]; t++) atomicAdd(&a.fwd_arrive[a.ch_tgt[t]], 1);
  return true;
}

// --------------------------------------------------------------- backward
template <typename T>
__device__ bool bwd_chunk(const SolveArgs<T>& a, SolveSmem<T>& sm, int c, int e) {
  const int tid = threadIdx.x;
  const int p = a.ch_piece[c];
  if (tid == 0) {
    int ok = 1;
    for (int64_t t = a.ch_tptr[c]; t < a.ch_tptr[c + 1] && ok; t++) ok = wait_geq(&a.bwd_done[a.ch_tgt[t]], e, a.st, a.spin);
    sm.flag = ok;
  }
  __syncthreads();
  if (!sm.flag) return false;
  const int pw = a.pc_w[p], ld = a.pc_ld[p];
  const int r0 = a.ch_r0[c], nr = a.ch_nr[c];
  const T* Lp = a.L + a.pc_off[p];
  T* xs = sm.aux;
  for (int i = tid; i < nr; i += blockDim.x) xs[i] = ldcg(&a.v[a.sn_rows[a.pc_row[p] + r0 + i]]);
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  T* z = a.zpart + a.pc_zoff[p] + (int64_t)a.ch_k[c] * pw;
  for (int k = warp; k < pw; k += nw) {
    T s = T(0);
    for (int i = lane; i < nr; i += 32) s += Lp[(int64_t)(r0 + i) + (int64_t)k * ld] * xs[i];
    s = warp_sum(s);
    if (lane == 0) z[k] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) atomicAdd(&a.bwd_arrive[p], 1);
  return true;
}

template <typename T>
__device__ bool bwd_head(const SolveArgs<T>& a, SolveSmem<T>& sm, int p, int e) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.flag = wait_geq(&a.bwd_arrive[p], e * a.pc_nchunk[p], a.st, a.spin);
  __syncthreads();
  if (!sm.flag) return false;
  const int pw = a.pc_w[p], ld = a.pc_ld[p], f = a.pc_first[p], nch = a.pc_nchunk[p];
  const T* Lp = a.L + a.pc_off[p];
  const T* z = a.zpart + a.pc_zoff[p];
  T* vec = sm.vec;
  for (int i = tid; i < pw; i += blockDim.x) {
    T t = ldcg(&a.v[f + i]);
    for (int k = 0; k < nch; k++) t -= ldcg(&z[(int64_t)k * pw + i]);
    vec[i] = t;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nblk = (pw + 31) / 32;
  for (int b = nblk - 1; b >= 0; b--) {
    const int jb = b * 32, bwb = min(32, pw - jb);
    if (jb + bwb < pw) {
      for (int jj = warp; jj < bwb; jj += nw) {
        const int j = jb + jj;
        T s = T(0);
        for (int i = jb + bwb + lane; i < pw; i += 32) s += Lp[(int64_t)i + (int64_t)j * ld] * vec[i];
        s = warp_sum(s);
        if (lane == 0) vec[j] -= s;
      }
      __syncthreads();
    }
    if (warp == 0) {
      T Lc[32];
#pragma unroll
      for (int j = 0; j < 32; j++)
        Lc[j] = (lane < bwb && j < bwb && j >= lane) ? Lp[(int64_t)(jb + j) + (int64_t)(jb + lane) * ld] : T(0);
      T t = lane < bwb ? vec[jb + lane] : T(0);
#pragma unroll
      for (int j = 31; j >= 0; j--) {
        if (j < bwb) {
          if (lane == j) t = t / Lc[j];
          const T xj = __shfl_sync(0xffffffffu, t, j);
          if (lane < j) t -= Lc[j] * xj;
        }
      }
      if (lane < bwb) vec[jb + lane] = t;
    }
    __syncthreads();
  }
  for (int i = tid; i < pw; i += blockDim.x) a.v[f + i] = vec[i];
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(&a.bwd_done[p], e);
  return true;
}

template <typename T, bool FWD>
__device__ bool sweep(const SolveArgs<T>& a, SolveSmem<T>& sm, int seq, int e) {
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&a.disp[(seq + 1) % 3], 0);
  const int32_t* items = FWD ? a.fwd_items : a.bwd_items;
  for (;;) {
    if (threadIdx.x == 0) sm.item = atomicAdd(&a.disp[seq % 3], 1);
    __syncthreads();
    const int it = sm.item;
    __syncthreads();
    if (it >= a.nitems) return true;
    const int code = items[it];
    bool ok;
    if (FWD) ok = code < 0 ? fwd_head(a, sm, -1 - code, e) : fwd_chunk(a, sm, code, e);
    else ok = code < 0 ? bwd_head(a, sm, -1 - code, e) : bwd_chunk(a, sm, code, e);
    if (!ok) return false;
  }
}

// one H^-1 application on a.v (forward then backward sweep)
template <typename T>
__device__ bool hsolve(const SolveArgs<T>& a, SolveSmem<T>& sm, int& seq, int& e) {
  e++;
  if (!sweep<T, true>(a, sm, seq++, e)) return false;
  if (!grid_barrier(a, sm)) return false;
  if (!sweep<T, false>(a, sm, seq++, e)) return false;
  return grid_barrier(a, sm);
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) k_cg(SolveArgs<T> a) {
  __shared__ SolveSmem<T> sm;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = a.n, m = a.m;
  int seq = 0, e = 0;
  // phase 0: r^_x = r_x + gamma J^T r_y in permuted labels; v = r^_x
  for (int64_t k = gt; k < n; k += gs) {
    const int32_t o = a.perm[k];
    double s = 0.0;
    if (a.mode == 0)
      for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * a.by[a.JT_row[q]];
    const double rh = a.bx[o] + a.gamma * s;
    a.rhx[k] = rh;
    a.v[k] = (T)rh;
  }
  if (!grid_barrier(a, sm)) return;
  if (!hsolve(a, sm, seq, e)) return;
  if (a.mode == 1) {
    for (int64_t k = gt; k < n; k += gs) {
      const double val = (double)ldcg(&a.v[k]);
      const int32_t o = a.perm[k];
      a.ox[o] = a.accumulate ? a.ox[o] + val : val;
    }
    return;
  }
  // b_S = J w - r_y
  double part = 0.0;
  for (int64_t i = gt; i < m; i += gs) {
    double s = 0.0;
    for (int64_t q = a.J_rowptr[i]; q < a.J_rowptr[i + 1]; q++) s += a.Jv[q] * (double)ldcg(&a.v[a.Jcol_perm[q]]);
    const double b = s - a.by[i];
    a.bS[i] = b; a.r[i] = b; a.p[i] = b; a.y[i] = 0.0;
    part += b * b;
  }
  block_partial2(a, sm, part, 0.0);
  if (!grid_barrier(a, sm)) return;
  double bn2, dummy;
  grid_total2(a, sm, bn2, dummy);
  double rho = bn2, rqmax = 0.0, d2 = 0.0;
  int it = 0, status = 4, brk = 0;
  const double stop = a.rtol * sqrt(bn2);
  for (;;) {
    if (sqrt(rho) <= stop) { status = 0; break; }
    if (it >= a.maxit) { status = 4; break; }
    for (int64_t k = gt; k < n; k += gs) {
      double s = 0.0;
      for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * __ldcg(&a.p[a.JT_row[q]]);
      a.v[k] = (T)s;
    }
    if (!grid_barrier(a, sm)) return;
    if (!hsolve(a, sm, seq, e)) return;
    double pq = 0.0, pp = 0.0;
    for (int64_t i = gt; i < m; i += gs) {
      double s = 0.0;
      for (int64_t q = a.J_rowptr[i]; q < a.J_rowptr[i + 1]; q++) s += a.Jv[q] * (double)ldcg(&a.v[a.Jcol_perm[q]]);
      const double pi = __ldcg(&a.p[i]);
      const double qi = s + d2 * pi;
      a.q[i] = qi;
      pq += pi * qi;
      pp += pi * pi;
    }
    block_partial2(a, sm, pq, pp);
    if (!grid_barrier(a, sm)) return;
    double PQ, PP;
    grid_total2(a, sm, PQ, PP);
    it++;
    const double rq = PQ / PP;
    if (rq > rqmax) rqmax = rq;
    if (!(PQ > 0.0) || rq <= 1e-12 * rqmax) {
      if (d2 == 0.0 && a.delta2 > 0.0) {        // restart once on S + delta_2 I
        brk = 1;
        d2 = a.delta2;
        rqmax = 0.0;
        rho = bn2;
        for (int64_t i = gt; i < m; i += gs) {
          const double b = __ldcg(&a.bS[i]);
          a.y[i] = 0.0; a.r[i] = b; a.p[i] = b;
        }
        if (!grid_barrier(a, sm)) return;
        continue;
      }
      status = 3;
      break;
    }
    const double alpha = rho / PQ;
    double rr = 0.0;
    for (int64_t i = gt; i < m; i += gs) {
      const double pi = __ldcg(&a.p[i]), qi = __ldcg(&a.q[i]);
      a.y[i] += alpha * pi;
      const double ri = __ldcg(&a.r[i]) - alpha * qi;
      a.r[i] = ri;
      rr += ri * ri;
    }
    block_partial2(a, sm, rr, 0.0);
    if (!grid_barrier(a, sm)) return;
    double rho2;
    grid_total2(a, sm, rho2, dummy);
    const double beta = rho2 / rho;
    rho = rho2;
    for (int64_t i = gt; i < m; i += gs) a.p[i] = __ldcg(&a.r[i]) + beta * __ldcg(&a.p[i]);
    if (!grid_barrier(a, sm)) return;
  }
  // dx = H^-1 (r^_x - J^T dy)
  for (int64_t k = gt; k < n; k += gs) {
    double s = 0.0;
    for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * __ldcg(&a.y[a.JT_row[q]]);
    a.v[k] = (T)(__ldcg(&a.rhx[k]) - s);
  }
  if (!grid_barrier(a, sm)) return;
  if (!hsolve(a, sm, seq, e)) return;
  for (int64_t k = gt; k < n; k += gs) {
    const double val = (double)ldcg(&a.v[k]);
    const int32_t o = a.perm[k];
    a.ox[o] = a.accumulate ? a.ox[o] + val : val;
  }
  for (int64_t i = gt; i < m; i += gs) {
    const double yi = __ldcg(&a.y[i]);
    a.oy[i] = a.accumulate ? a.oy[i] + yi : yi;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->cg_iters = it;
    a.st->cg_status = status;
    a.st->breakdown = brk;
  }
}

template <typename T>
int solve_grid_size(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg<T>, kSolveThreads, 0);
  if (per < 1) per = 1;
  return sms * per;
}

template <typename T>
cudaError_t launch_solve(const SolveArgs<T>& a, int grid, cudaStream_t st) {
  SolveArgs<T> args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)k_cg<T>, dim3(grid), dim3(kSolveThreads), params, 0, st);
}

template int solve_grid_size<double>(int);
template int solve_grid_size<float>(int);
template cudaError_t launch_solve<double>(const SolveArgs<double>&, int, cudaStream_t);
template cudaError_t launch_solve<float>(const SolveArgs<float>&, int, cudaStream_t);

// --------------------------------------------------------------- residual
__global__ void __launch_bounds__(256) k_residual(ResArgs a) {
  __shared__ double sred[8][4];
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  double r2 = 0, b2 = 0, x2 = 0, kmax = 0;
  for (int64_t i = gt; i < a.n; i += gs) {
    const double xi = a.x[i];
    double s = a.bx[i] - a.delta * xi;
    double ra = fabs(a.delta);
    for (int64_t q = a.Hs_ptr[i]; q < a.Hs_ptr[i + 1]; q++) {
      const double h = a.Hv[a.Hs_vidx[q]];
      s -= h * a.x[a.Hs_col[q]];
      ra += fabs(h);
    }
    for (int64_t q = a.JT_ptr[i]; q < a.JT_ptr[i + 1]; q++) {
      const double jv = a.Jv[a.JT_vidx[q]];
      s -= jv * a.y[a.JT_row[q]];
      ra += fabs(jv);
    }
    a.res_x[i] = s;
    r2 += s * s;
    b2 += a.bx[i] * a.bx[i];
    x2 += xi * xi;
    kmax = fmax(kmax, ra);
  }
  for (int64_t i = gt; i < a.m; i += gs) {
    double s = a.by[i], ra = 0.0;
    for (int64_t q = a.J_rowptr[i]; q < a.J_rowptr[i + 1]; q++) {
      s -= a.Jv[q] * a.x[a.J_colidx[q]];
      ra += fabs(a.Jv[q]);
    }
    a.res_y[i] = s;
    r2 += s * s;
    b2 += a.by[i] * a.by[i];
    x2 += a.y[i] * a.y[i];
    kmax = fmax(kmax, ra);
  }
  r2 = warp_sum(r2); b2 = warp_sum(b2); x2 = warp_sum(x2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = fmax(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sred[warp][0] = r2; sred[warp][1] = b2; sred[warp][2] = x2; sred[warp][3] = kmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int w = 0; w < 8; w++) { t[0] += sred[w][0]; t[1] += sred[w][1]; t[2] += sred[w][2]; t[3] = fmax(t[3], sred[w][3]); }
    for (int j = 0; j < 4; j++) a.red[blockIdx.x * 4 + j] = t[j];
  }
}

__global__ void k_residual_final(ResArgs a, int nblocks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[4] = {0, 0, 0, 0};
  for (int b = 0; b < nblocks; b++) {
    t[0] += a.red[b * 4]; t[1] += a.red[b * 4 + 1]; t[2] += a.red[b * 4 + 2];
    t[3] = fmax(t[3], a.red[b * 4 + 3]);
  }
  const double res = sqrt(t[0]), bn = sqrt(t[1]), xn = sqrt(t[2]);
  a.st->res_norm = res;
  a.st->b_norm = bn;
  a.st->x_norm = xn;
  a.st->k_norm_inf = t[3];
  a.st->rr = bn > 0 ? res / bn : res;
  a.st->be = res / (t[3] * xn + bn);
}

cudaError_t launch_residual(const ResArgs& a, cudaStream_t st) {
  const int blocks = 296;
  k_residual<<<blocks, 256, 0, st>>>(a);
  k_residual_final<<<1, 32, 0, st>>>(a, blocks);
  return cudaGetLastError();
}

}  // namespace kkt
