// Numeric supernodal (multifrontal) Cholesky of
//   A = P (H~ + delta I + gamma J^T J) P^T = L L^T
// (Sec. 4, eq. gamma; Sec. 4.1 H_delta; Algorithm 1: "Try L L^T = chol(H_delta)").
//
// Layout: supernode s owns a column-major panel of snr[s] x sw[s] entries
// (its rows = its columns followed by the rows below, ld = snr[s]) and an
// update matrix U_s of rb x rb (rb = snr[s] - sw[s], ld = rb) holding
//   U_s = - L21 L21^T + (children's updates)
// (the SYRK stores it, then the children's update-matrix entries are added),
// which is extend-added into the parent's front. Fronts of one tree level are
// processed together; siblings add into the same parent entries with device
// atomics, so the summation order of those contributions is not fixed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.hpp"

namespace kkt {

// ------------------------------------------------------------------ assembly
// Panel slot t <- sum of its sources: H~ entries, delta on the diagonal and
// gamma * J_ra * J_rb for each pair of entries of each row r of J.
template <typename T>
__global__ void k_assemble(int64_t nslot, const int64_t* __restrict__ slot_pos,
                           const int64_t* __restrict__ src_ptr, const int32_t* __restrict__ srcA,
                           const int32_t* __restrict__ srcB, const double* __restrict__ Hv,
                           const double* __restrict__ Jv, const double* __restrict__ dg, T* __restrict__ L,
                           int64_t bsH, int64_t bsJ, int64_t bsL) {
  const double delta = dg[0], gamma = dg[1];   // device scalars: a captured graph replays with new values
  Hv += blockIdx.y * bsH;                       // system blockIdx.y of a batched launch
  Jv += blockIdx.y * bsJ;
  L += blockIdx.y * bsL;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nslot; t += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t q = src_ptr[t]; q < src_ptr[t + 1]; q++) {
      const int32_t a = srcA[q], b = srcB[q];
      v += (b == -1) ? Hv[a] : (b == -2 ? delta : gamma * Jv[a] * Jv[b]);
    }
    L[slot_pos[t]] = (T)v;
  }
}

// ------------------------------------------------------------------- POTRF
// Column block kb (kPB columns) of each listed front: Cholesky of the
// kPB x kPB diagonal tile in shared memory, written back to the panel. A
// pivot <= 0 or non-finite records the column in DevStatus::fail_col.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf(const int4* __restrict__ items, int kb, FacArgs<T> a) {
  batch_view(a);
  __shared__ T D[kPB][kPB + 1];
  const int s = items[blockIdx.x].x;
  const int w = a.sw[s], nr = a.snr[s], ld = a.sld[s];
  const int c0 = kb * kPB;
  const int bw = min(kPB, w - c0);
  T* P = a.L + a.poff[s];
  const int tid = threadIdx.x;
  for (int e = tid; e < kPB * kPB; e += blockDim.x) {
    const int i = e % kPB, j = e / kPB;
    D[i][j] = (i < bw && j <= i) ? P[(int64_t)(c0 + i) + (int64_t)(c0 + j) * ld] : T(0);
  }
  __syncthreads();
  for (int j = 0; j < bw; j++) {
    if (tid == 0) {
      T d = D[j][j];
      if (!(d > T(0)) || !isfinite((double)d)) {
        atomicMin(&a.st->fail_col, a.sfirst[s] + c0 + j);
        d = T(1);
      }
      D[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < bw; i += blockDim.x) D[i][j] /= D[j][j];
    __syncthreads();
    const int rem = bw - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e % rem, k = j + 1 + e / rem;
      if (k <= i) D[i][k] -= D[i][j] * D[k][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < kPB * kPB; e += blockDim.x) {
    const int i = e % kPB, j = e / kPB;
    if (i < bw && j <= i) P[(int64_t)(c0 + i) + (int64_t)(c0 + j) * ld] = D[i][j];
  }
}

// -------------------------------------------------------------------- TRSM
// Rows below the diagonal tile of column block kb: X = A D^-T with D the
// factored tile (read from the panel); items (s, row tile of kTR rows).
template <typename T>
__global__ void __launch_bounds__(kTR) k_trsm(const int4* __restrict__ items, int kb, FacArgs<T> a) {
  batch_view(a);
  __shared__ T D[kPB][kPB + 1];
  const int4 it = items[blockIdx.x];
  const int s = it.x, t = it.y;
  const int w = a.sw[s], nr = a.snr[s], ld = a.sld[s];
  const int c0 = kb * kPB;
  const int bw = min(kPB, w - c0);
  T* P = a.L + a.poff[s];
  const int tid = threadIdx.x;
  for (int e = tid; e < kPB * kPB; e += blockDim.x) {
    const int i = e % kPB, j = e / kPB;
    D[i][j] = (i < bw && j <= i) ? P[(int64_t)(c0 + i) + (int64_t)(c0 + j) * ld] : T(i == j ? 1 : 0);
  }
  __syncthreads();
  const int r = c0 + bw + t * kTR + tid;
  if (r < nr) {
    T x[kPB];
#pragma unroll
    for (int k = 0; k < kPB; k++) x[k] = (k < bw) ? P[(int64_t)r + (int64_t)(c0 + k) * ld] : T(0);
#pragma unroll
    for (int j = 0; j < kPB; j++) {
      if (j < bw) {
        T sacc = x[j];
#pragma unroll
        for (int k = 0; k < j; k++) sacc -= x[k] * D[j][k];
        x[j] = sacc / D[j][j];
      }
    }
#pragma unroll
    for (int k = 0; k < kPB; k++)
      if (k < bw) P[(int64_t)r + (int64_t)(c0 + k) * ld] = x[k];
  }
}

// ------------------------------------------------- fused block step
// Right-looking step for column block kb of each listed front, one CTA per
// (front, tile of kTR rows below the block), after the in-panel updates of
// the earlier blocks:
//   D = chol(A[blk, blk]),   L[r, blk] = A[r, blk] D^-T   for the tile's rows r.
// Every CTA of a front factors the same D (same inputs, same operation
// order, so the same bits); tile 0 keeps it in the level's scratch slot
// (k_dstore moves it into the panel after the level's last step, so no
// CTA reads a half-written diagonal tile). Replaces the separate POTRF and
// TRSM launches.
template <typename T>
__device__ __forceinline__ void warp_potrf32(T (&D)[kPB][kPB + 1], T* dinv, int bw, int fail_base, DevStatus* st) {
  // lane i holds row i of the tile
  const int lane = threadIdx.x & 31;
  T d[kPB];
#pragma unroll
  for (int k = 0; k < kPB; k++) d[k] = (lane < bw && k <= lane) ? D[lane][k] : T(lane == k ? 1 : 0);
#pragma unroll
  for (int j = 0; j < kPB; j++) {
    if (j < bw) {
      T djj = __shfl_sync(0xffffffffu, d[j], j);
      if (!(djj > T(0)) || !isfinite(djj)) {
        if (lane == 0) atomicMin(&st->fail_col, fail_base + j);
        djj = T(1);
      }
      // one reciprocal square root and multiplies: the IEEE square root and
      // a division per column made up most of this warp's time (each
      // column waits on the previous one)
      const T rs = rsqrt(djj);
      if (lane == j) {
        d[j] = djj * rs;
        dinv[j] = rs;
      }
      if (lane > j) d[j] = d[j] * rs;
#pragma unroll
      for (int k = j + 1; k < kPB; k++) {
        const T lkj = __shfl_sync(0xffffffffu, d[j], k);
        if (lane >= k) d[k] -= d[j] * lkj;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kPB; k++)
    if (lane < bw && k <= lane) D[lane][k] = d[k];
}

static_assert(kFItem == 3 * 4, "block-step and update items are three int4");

template <typename T>
__global__ void __launch_bounds__(kTR) k_block(const int4* __restrict__ items, int kb, FacArgs<T> a) {
  batch_view(a);
  __shared__ T D[kPB][kPB + 1];
  __shared__ T Dinv[kPB];   // reciprocals of the factored tile's diagonal
  const int4 it = items[3 * blockIdx.x], fm = items[3 * blockIdx.x + 1], fo = items[3 * blockIdx.x + 2];
  const int t = it.y;
  const int w = fm.x, nr = fm.y, ld = fm.z, sfirst = fm.w;
  const int c0 = kb * kPB;
  const int bw = min(kPB, w - c0);
  T* P = a.L + (int64_t)(((uint64_t)(uint32_t)fo.y << 32) | (uint32_t)fo.x);
  const int tid = threadIdx.x;
  const int r = c0 + bw + t * kTR + tid;
  const bool row = r < nr;
  T x[kPB];
#pragma unroll
  for (int j = 0; j < kPB; j++) x[j] = (row && j < bw) ? P[(int64_t)r + (int64_t)(c0 + j) * ld] : T(0);
  for (int e = tid; e < kPB * kPB; e += kTR) {
    const int i = e % kPB, j = e / kPB;
    D[i][j] = (i < bw && j <= i) ? P[(int64_t)(c0 + i) + (int64_t)(c0 + j) * ld] : T(0);
  }
  __syncthreads();
  if (tid < 32) warp_potrf32(D, Dinv, bw, sfirst + c0, a.st);
  __syncthreads();
  if (t == 0) {
    T* dst = a.Dsc + (int64_t)it.z * (kPB * kPB);
    for (int e = tid; e < kPB * kPB; e += kTR) dst[e] = D[e % kPB][e / kPB];
  }
  if (row) {
#pragma unroll
    for (int j = 0; j < kPB; j++) {
      if (j < bw) {
        // two partial sums halve the dependent FMA chain
        T s0 = x[j], s1 = T(0);
#pragma unroll
        for (int k = 0; k + 1 < j; k += 2) {
          s0 -= x[k] * D[j][k];
          s1 -= x[k + 1] * D[j][k + 1];
        }
        if (j & 1) s0 -= x[j - 1] * D[j][j - 1];
        x[j] = (s0 + s1) * Dinv[j];
      }
    }
#pragma unroll
    for (int j = 0; j < kPB; j++)
      if (j < bw) P[(int64_t)r + (int64_t)(c0 + j) * ld] = x[j];
  }
}

// The level's factored diagonal tiles from the scratch into the panels.
template <typename T>
__global__ void __launch_bounds__(256) k_dstore(const int4* __restrict__ items, FacArgs<T> a) {
  batch_view(a);
  const int4 it = items[blockIdx.x];
  const int s = it.x, c0 = it.y * kPB;
  const int w = a.sw[s], ld = a.sld[s];
  const int bw = min(kPB, w - c0);
  T* P = a.L + a.poff[s];
  const T* src = a.Dsc + (int64_t)it.z * (kPB * kPB);
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e % kPB, j = e / kPB;
    if (i < bw && j <= i) P[(int64_t)(c0 + i) + (int64_t)(c0 + j) * ld] = src[e];
  }
}

// ------------------------------------------------------- in-panel update
// Right-looking update of the panel columns after block kb:
//   P[i, j] -= sum_k P[i, c0+k] P[j, c0+k],  j >= c0+bw, i >= j.
// items (s, row tile of kUR rows, column tile of kPB columns).
template <typename T>
__global__ void __launch_bounds__(256) k_panel_update(const int4* __restrict__ items, int kb, FacArgs<T> a) {
  batch_view(a);
  __shared__ T As[kUR][kPB + 1];
  __shared__ T Bs[kPB][kPB + 1];
  const int4 it = items[3 * blockIdx.x], fm = items[3 * blockIdx.x + 1], fo = items[3 * blockIdx.x + 2];
  const int rt = it.y, ct = it.z;
  const int w = fm.x, nr = fm.y, ld = fm.z;
  const int c0 = kb * kPB;
  const int bw = min(kPB, w - c0);
  const int cstart = c0 + bw + ct * kPB;
  const int cw = min(kPB, w - cstart);
  const int rstart = cstart + rt * kUR;
  const int rn = min(kUR, nr - rstart);
  T* P = a.L + (int64_t)(((uint64_t)(uint32_t)fo.y << 32) | (uint32_t)fo.x);
  const int tid = threadIdx.x;
  for (int e = tid; e < kUR * kPB; e += blockDim.x) {
    const int i = e % kUR, k = e / kUR;
    As[i][k] = (i < rn && k < bw) ? P[(int64_t)(rstart + i) + (int64_t)(c0 + k) * ld] : T(0);
  }
  for (int e = tid; e < kPB * kPB; e += blockDim.x) {
    const int j = e % kPB, k = e / kPB;
    Bs[j][k] = (j < cw && k < bw) ? P[(int64_t)(cstart + j) + (int64_t)(c0 + k) * ld] : T(0);
  }
  __syncthreads();
  const int i = tid % kUR;            // consecutive threads -> consecutive rows
  const int jg = tid / kUR;           // 4 groups of 8 columns
  T acc[8];
#pragma unroll
  for (int q = 0; q < 8; q++) acc[q] = T(0);
  for (int k = 0; k < bw; k++) {
    const T av = As[i][k];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] += av * Bs[jg * 8 + q][k];
  }
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int j = jg * 8 + q;
    if (i < rn && j < cw && rstart + i >= cstart + j)
      P[(int64_t)(rstart + i) + (int64_t)(cstart + j) * ld] -= acc[q];
  }
}

// ---------------------------------------------------------------- SYRK
// U_s = -L21 L21^T on 64 x 64 tiles (ti >= tj), k = panel width.
template <typename T>
__global__ void __launch_bounds__(256) k_syrk(const int4* __restrict__ items, FacArgs<T> a) {
  batch_view(a);
  constexpr int KC = 16;
  __shared__ T As[KC][kST + 1];
  __shared__ T Bs[KC][kST + 1];
  const int4 it = items[blockIdx.x];
  const int s = it.x, ti = it.y, tj = it.z;
  const int w = a.sw[s], nr = a.snr[s], ld = a.sld[s];
  const int rb = nr - w;
  const T* P = a.L + a.poff[s];
  T* U = a.U + a.uoff[s];
  const int i0 = ti * kST, j0 = tj * kST;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) acc[x][y] = T(0);
  for (int k0 = 0; k0 < w; k0 += KC) {
    for (int e = tid; e < KC * kST; e += blockDim.x) {
      const int r = e % kST, k = e / kST;
      const bool kin = k0 + k < w;
      As[k][r] = (kin && i0 + r < rb) ? P[(int64_t)(w + i0 + r) + (int64_t)(k0 + k) * ld] : T(0);
      Bs[k][r] = (kin && j0 + r < rb) ? P[(int64_t)(w + j0 + r) + (int64_t)(k0 + k) * ld] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; k++) {
      T av[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; x++) av[x] = As[k][tx + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; y++) bv[y] = Bs[k][ty + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; y++)
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int gi = i0 + tx + 16 * x, gj = j0 + ty + 16 * y;
      if (gi < rb && gj < rb && gi >= gj) U[(int64_t)gi + (int64_t)gj * rb] = -acc[x][y];
    }
}

// ----------------------------------------------------- SYRK, 128 x 128 tiles
// FP32 fronts with rb >= kBigRows: U_s = -L21 L21^T on 128 x 128 tiles
// (ti >= tj), 256 threads with 8 x 8 register tiles (rows tx*4 + {0..3, 64..67},
// columns ty*4 + {0..3, 64..67}, tx = tid % 16, ty = tid / 16), K staged 16
// columns at a time through two shared-memory buffers.
__global__ void __launch_bounds__(256) k_syrk128(const int4* __restrict__ items, FacArgs<float> a) {
  batch_view(a);
  constexpr int KC = 16, TS = 128;
  __shared__ __align__(16) float As[2][KC][TS];
  __shared__ __align__(16) float Bs[2][KC][TS];
  const int4 it = items[blockIdx.x];
  const int s = it.x, ti = it.y, tj = it.z;
  const int w = a.sw[s], nr = a.snr[s], ld = a.sld[s];
  const int rb = nr - w;
  const float* P = a.L + a.poff[s];
  float* U = a.U + a.uoff[s];
  const int i0 = ti * TS, j0 = tj * TS;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[8][8];
#pragma unroll
  for (int x = 0; x < 8; x++)
#pragma unroll
    for (int y = 0; y < 8; y++) acc[x][y] = 0.f;
  // each thread stages 8 entries of A and 8 of B per chunk: row tid % 128,
  // columns (tid / 128) * 8 + {0..7}
  const int lr = tid % TS, lk = (tid / TS) * 8;
  const bool ra = i0 + lr < rb, rbv = j0 + lr < rb;
  const float* pa = P + (w + i0 + lr);
  const float* pb = P + (w + j0 + lr);
  float va[8], vb[8];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int k = k0 + lk + q;
      va[q] = (ra && k < w) ? pa[(int64_t)k * ld] : 0.f;
      vb[q] = (rbv && k < w) ? pb[(int64_t)k * ld] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      As[buf][lk + q][lr] = va[q];
      Bs[buf][lk + q][lr] = vb[q];
    }
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < w; k0 += KC) {
    const bool more = k0 + KC < w;
    if (more) load(k0 + KC);
#pragma unroll
    for (int k = 0; k < KC; k++) {
      const float4 a0 = *(const float4*)&As[buf][k][tx * 4];
      const float4 a1 = *(const float4*)&As[buf][k][tx * 4 + 64];
      const float4 b0 = *(const float4*)&Bs[buf][k][ty * 4];
      const float4 b1 = *(const float4*)&Bs[buf][k][ty * 4 + 64];
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int x = 0; x < 8; x++)
#pragma unroll
        for (int y = 0; y < 8; y++) acc[x][y] += av[x] * bv[y];
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int y = 0; y < 8; y++) {
    const int gj = j0 + ty * 4 + (y & 3) + (y >> 2) * 64;
#pragma unroll
    for (int x = 0; x < 8; x++) {
      const int gi = i0 + tx * 4 + (x & 3) + (x >> 2) * 64;
      if (gi < rb && gj < rb && gi >= gj) U[(int64_t)gi + (int64_t)gj * rb] = -acc[x][y];
    }
  }
}

// --------------------------------------------------------------- extend-add
// Adds U_s into the parent's front: entry (i, j) of U_s goes to position
// (rel[i], rel[j]) of the parent's rows, i.e. the parent's panel when rel[j]
// is one of its columns, else its update matrix.
template <typename T>
__global__ void __launch_bounds__(256) k_extend_add(const int4* __restrict__ items, FacArgs<T> a) {
  batch_view(a);
  const int4 it = items[blockIdx.x];
  const int s = it.x, j0 = it.y, j1 = it.z;   // child columns [j0, min(j0 + kEC, j1))
  const int p = a.sparent[s];
  const int w = a.sw[s], rb = a.snr[s] - w;
  const int wp = a.sw[p], nrp = a.snr[p], rbp = nrp - wp, ldp = a.sld[p];
  const int32_t* __restrict__ rel = a.rel + a.srow[s] + w;
  const T* __restrict__ Us = a.U + a.uoff[s];   // column j at Us + j * rb, rows j..rb-1 used
  // an item's columns all land in the parent's panel or all in its update
  // matrix (the plan splits the children's columns there)
  const bool panel = rel[j0] < wp;
  T* __restrict__ dst = panel ? a.L + a.poff[p] : a.U + a.uoff[p] - wp;   // + row + col * ld
  const int64_t ldd = panel ? ldp : rbp;
  const int cofs = panel ? 0 : wp;
  const int bd = blockDim.x;
  // four columns x four rows per thread at a time: every index and value
  // load is issued before the adds, so a thread waits one memory round trip
  // per sixteen entries
  for (int jj = 0; jj < kEC; jj += 4) {
    const int jb = j0 + jj;
    if (jb >= j1) break;
    T* __restrict__ col[4];
    int jc[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      jc[c] = jb + c < min(j1, j0 + kEC) ? jb + c : rb;   // rb: no rows
      col[c] = jc[c] < rb ? dst + (int64_t)(rel[jc[c]] - cofs) * ldd : dst;
    }
    for (int ib = threadIdx.x; jb + ib < rb; ib += 4 * bd) {
      int ai[4][4];
      T v[4][4];
#pragma unroll
      for (int c = 0; c < 4; c++)
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = jc[c] + ib + u * bd;
          ai[c][u] = i < rb ? __ldg(&rel[i]) : -1;
          v[c][u] = i < rb ? Us[i + (int64_t)jc[c] * rb] : T(0);
        }
#pragma unroll
      for (int c = 0; c < 4; c++)
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (ai[c][u] >= 0) atomicAdd(&col[c][ai[c][u]], v[c][u]);
    }
  }
}


static cudaError_t launch_syrk128(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb) {
  k_syrk128<<<dim3((unsigned)cnt, (unsigned)nb), 256, 0, st>>>(items, a);
  return cudaGetLastError();
}
template <typename T>
static cudaError_t launch_syrk128(const int4*, int64_t, const FacArgs<T>&, cudaStream_t, int) {
  return cudaErrorNotSupported;   // FP64 fronts keep the 64 x 64 tiles
}

static cudaError_t launch_split_tc(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb) {
  return launch_tc_split(items, cnt, a, st, nb);
}
template <typename T>
static cudaError_t launch_split_tc(const int4*, int64_t, const FacArgs<T>&, cudaStream_t, int) {
  return cudaErrorNotSupported;   // the FP64 factor has no tensor-core path
}
static cudaError_t launch_syrk_tc(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb) {
  return launch_tc_update(items, cnt, a, st, nb);
}
template <typename T>
static cudaError_t launch_syrk_tc(const int4*, int64_t, const FacArgs<T>&, cudaStream_t, int) {
  return cudaErrorNotSupported;   // the tensor-core updates are the FP32 factor's
}

// ---------------------------------------------------------- triangle inverses
// For every triangular-solve piece: X = T^-1 of its pw x pw diagonal
// triangle T (lower), stored packed by columns (column k holds rows k..pw-1,
// padded to a multiple of 4), so that the solve applies T^-1 as a dense
// mat-vec. Thread k computes column k by forward substitution; T is staged
// in shared memory.
template <typename T>
__global__ void __launch_bounds__(128) k_tri_inv(InvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ts = (T*)smem_raw;
  a.L += blockIdx.y * a.bsL;
  a.Linv += blockIdx.y * a.bsI;
  const int p = blockIdx.x;
  const int pw = a.pc_w[p], ld = a.pc_ld[p], c = a.pc_c[p];
  const T* L = a.L + a.pc_colbase[p] + c;      // (row c, col c) of the supernode panel
  for (int e = threadIdx.x; e < pw * pw; e += blockDim.x) {
    const int i = e % pw, j = e / pw;
    Ts[i + j * pw] = (i >= j) ? L[(int64_t)i + (int64_t)j * ld] : T(0);
  }
  __syncthreads();
  T* X = a.Linv + a.pc_inv[p];
  for (int k = threadIdx.x; k < pw; k += blockDim.x) {
    int64_t off = 0;                              // packed column offset
    for (int j = 0; j < k; j++) off += (pw - j + 3) & ~3;
    T* xk = X + off - k;                          // xk[i] = X(i, k), i >= k
    xk[k] = T(1) / Ts[k + k * pw];
    for (int i = k + 1; i < pw; i++) {
      T s = T(0);
      for (int j = k; j < i; j++) s += Ts[i + j * pw] * xk[j];
      xk[i] = -s / Ts[i + i * pw];
    }
    for (int i = pw; i < k + ((pw - k + 3) & ~3); i++) xk[i] = T(0);   // padding
  }
}

template <typename T>
cudaError_t launch_tri_inv(const InvArgs<T>& a, int64_t npieces, int max_pw, cudaStream_t st, int nb) {
  const size_t smem = sizeof(T) * (size_t)max_pw * max_pw;
  cudaError_t e = raise_smem_limit(k_tri_inv<T>, smem);
  if (e) return e;
  if (npieces <= 0) return cudaSuccess;
  k_tri_inv<T><<<dim3((unsigned)npieces, (unsigned)nb), 128, smem, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_tri_inv<double>(const InvArgs<double>&, int64_t, int, cudaStream_t, int);
template cudaError_t launch_tri_inv<float>(const InvArgs<float>&, int64_t, int, cudaStream_t, int);

cudaError_t prof_begin(Prof* pr, cudaStream_t st) {
  if (!pr) return cudaSuccess;
  return cudaEventRecord(pr->a, st);
}

cudaError_t prof_end(Prof* pr, int kind, cudaStream_t st) {
  if (!pr) return cudaSuccess;
  cudaError_t e = cudaEventRecord(pr->b, st);
  if (e) return e;
  if ((e = cudaEventSynchronize(pr->b))) return e;
  float ms = 0.f;
  if ((e = cudaEventElapsedTime(&ms, pr->a, pr->b))) return e;
  pr->ms[kind] += ms;
  pr->n[kind] += 1;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_factor(const FacArgs<T>& a, const FacLists& fl, const double* dg, cudaStream_t st,
                          Prof* prof, int nb) {
  cudaError_t e;
  // nb systems: the panels of system b start at a.L + b * a.bsL (contiguous
  // when bsL = panel_total, as the batched form lays them out)
  if ((e = cudaMemsetAsync(a.L, 0, sizeof(T) * (size_t)fl.panel_total * nb, st))) return e;
  const unsigned y = (unsigned)nb;
  {
    const int threads = 256;
    int64_t blocks = (fl.nslot + threads - 1) / threads;
    if (blocks > 148 * 64) blocks = 148 * 64;
    if (blocks < 1) blocks = 1;
    if ((e = prof_begin(prof, st))) return e;
    k_assemble<T><<<dim3((unsigned)blocks, y), threads, 0, st>>>(fl.nslot, fl.slot_pos, fl.src_ptr, fl.srcA, fl.srcB,
                                                                  a.Hv, a.Jv, dg, a.L, a.bsH, a.bsJ, a.bsL);
    if ((e = prof_end(prof, 0, st))) return e;
  }
  for (const Launch& L : *fl.launches) {
    if (L.cnt <= 0) continue;
    if ((e = prof_begin(prof, st))) return e;
    const dim3 g((unsigned)L.cnt, y);
    switch (L.kind) {
      case 0: k_potrf<T><<<g, 256, 0, st>>>(fl.it_potrf + L.off, L.kb, a); break;
      case 1: k_trsm<T><<<g, kTR, 0, st>>>(fl.it_trsm + L.off, L.kb, a); break;
      case 2: k_panel_update<T><<<g, 256, 0, st>>>(fl.it_pupd + 3 * L.off, L.kb, a); break;
      case 3: k_syrk<T><<<g, 256, 0, st>>>(fl.it_syrk + L.off, a); break;
      case 4: k_extend_add<T><<<g, 256, 0, st>>>(fl.it_eadd + L.off, a); break;
      case 6:
        if ((e = launch_syrk_tc(fl.it_syrk_tc + (kTcItem / 4) * L.off, L.cnt, a, st, nb))) return e;
        break;
      case 7: k_block<T><<<g, kTR, 0, st>>>(fl.it_block + 3 * L.off, L.kb, a); break;
      case 8:
        if ((e = launch_syrk128(fl.it_syrk128 + L.off, L.cnt, a, st, nb))) return e;
        break;
      case 9: k_dstore<T><<<g, 256, 0, st>>>(fl.it_dstore + L.off, a); break;
      case 10:
        if ((e = launch_split_tc(fl.it_tc_split + (kTcItem / 4) * L.off, L.cnt, a, st, nb))) return e;
        break;
    }
    // kinds 0..4 -> profile slots 1..5; 8 (128-tile SYRK) shares the SYRK
    // slot, 7 and 9 the block slot; 10 (operand split) has slot 6
    const int slot = L.kind == 6    ? KKT_K_SYRK_TC_PROF
                     : L.kind == 10 ? KKT_K_TC_SPLIT_PROF
                                    : ((L.kind == 7 || L.kind == 9) ? KKT_K_BLOCK_PROF : (L.kind == 8 ? 4 : 1 + L.kind));
    if ((e = prof_end(prof, slot, st))) return e;
  }
  return cudaGetLastError();
}

template cudaError_t launch_factor<double>(const FacArgs<double>&, const FacLists&, const double*, cudaStream_t,
                                           Prof*, int);
template cudaError_t launch_factor<float>(const FacArgs<float>&, const FacLists&, const double*, cudaStream_t,
                                          Prof*, int);

}  // namespace kkt
