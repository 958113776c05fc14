// Persistent, cooperative CG on the Schur complement (eqs. Schur1/Schur2 and
// Algorithm 1's solve steps):
//   r^_x = r_x + gamma J^T r_y;  w = H^-1 r^_x;  b_S = J w - r_y;
// With a.xacc set (the mixed-precision form), eq. Schur2's back-substitution
// dx = H^-1 (r^_x - J^T dy) is not a third solve: every CG product already
// forms t_i = H^-1 J^T p_i, and with dy = sum alpha_i p_i, dx = w - sum
// alpha_i t_i is accumulated (FP64) along the CG recurrence, saving one H^-1
// application per refinement pass. The sum cancels when H_delta is nearly
// singular along null(J), so the FP64 form keeps Algorithm 1's direct solve.
//   CG on (S + d2 I) dy = b_S with S = J H^-1 J^T, one product per iteration
//   = J^T p, forward and backward triangular solves with L, J (Sec. 4.1);
//   dx = H^-1 (r^_x - J^T dy).
// Everything runs inside one kernel launch: no host round trip inside CG.
// Grid-wide phases are separated by a software grid barrier; the triangular
// solves are dependency-driven sweeps over "pieces" (column ranges of at most
// solve_w columns of one supernode) and "chunks" (row ranges of a piece's
// off-diagonal block), handed out in a fixed topological order through an
// atomic ticket. Every wait is bounded (DevStatus::abort on timeout). In the
// forward sweep a chunk subtracts L21 y from the vector at its rows; in the
// backward sweep it subtracts L21^T x from the vector at its piece's columns
// (atomic adds in both, so the head of a piece finds its right-hand side
// complete once the arrival count says so).
// Signalling: a CTA barrier, then thread 0 alone publishes with a release
// store or a fence + atomic (the fence is cumulative over the writes the
// barrier ordered before it; measured cheaper than release reductions); a
// waiter polls with an acquire load, then barriers its CTA.
// The CG recurrences, dot products and scalars are FP64 in both precisions;
// T is the storage/arithmetic type of L and of the triangular-solve vector.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace kkt {

constexpr int kSolveThreads = 256;

// Static shared state; the tiles live in dynamic shared memory.
struct SolveSmemHdr {
  unsigned long long mbar;   // completion of the bulk copies of the current item
  unsigned phase;
  int item, code;   // the CTA's current ticket and its item code
  int flag;
  // cycle counters of thread 0 (kept when a.instr != nullptr): dispatch,
  // dependency waits, bulk-copy waits, whole items, grid barriers, items
  long long c_disp, c_dep, c_mbar, c_item, c_bar, n_items;
  long long c_kind[3], n_kind[3];   // whole-item cycles and counts: subtrees, heads, chunks
  long long c_lvl, n_lvl;           // subtree items: cycles in the level loops, levels
  long long c_ph[16], t_mark;       // phases of heads and forward chunks (thread 0)
  double dred[(kSolveThreads / 32) * 2];
  double bcast[2];
};

template <typename T>
struct Tiles {
  T* A;     // packed inverse of a piece triangle (heads, subtrees)
  T* B;     // chunk-0 tile of a head, a subtree's panels
  T* C;     // a chunk's tile
  T* vec;   // sw
  T* vec2;  // sw
  T* aux;   // max_rows + kSolveThreads
};

__host__ __device__ static size_t packed_inv(size_t pw) {
  size_t t = 0;
  for (size_t k = 0; k < pw; k++) t += (pw - k + 3) & ~(size_t)3;
  return t;
}
// Shared memory: region A holds a head's or a subtree's packed inverses,
// region B the row tile of a head's chunk 0 (ent0 entries) or a subtree's
// panels (esub), C a chunk's row tile (ent), each + 8 entries per column of
// start alignment. Without overlap (ov = 0) C is B. With it (ov = 1) C
// starts where A does: a chunk of one right-hand side never uses A, and the
// region is then max(C, A + B) instead of A + max(B, C) (three solve CTAs
// per SM fit where two did). Every region starts on 128 bytes (TMA boxes).
__host__ __device__ static size_t tileA(int sw, int /*ent*/) { return packed_inv((size_t)sw); }
__host__ __device__ static size_t round128(size_t elem, size_t x) {
  const size_t q = 128 / elem;
  return (x + q - 1) / q * q;
}
struct SolveLayout {
  size_t b_off, c_off, vec_off;   // element offsets from the aligned base (A at 0)
};
__host__ __device__ static SolveLayout solve_layout(size_t elem, int sw, int ent, int ent0, int esub, int ov) {
  SolveLayout l;
  const size_t a = round128(elem, tileA(sw, ent));
  const size_t b = (size_t)max(ent0, esub) + 8 * (size_t)sw;
  const size_t c = (size_t)ent + 8 * (size_t)sw;
  l.b_off = a;
  if (ov) {
    l.c_off = 0;
    l.vec_off = max(round128(elem, c), a + b);
  } else {
    l.c_off = a;
    l.vec_off = a + max(b, c);
  }
  return l;
}

size_t solve_smem_bytes(size_t elem, int sw, int ent, int ent0, int esub, int max_rows, int ov) {
  const SolveLayout l = solve_layout(elem, sw, ent, ent0, esub, ov);
  return elem * (l.vec_off + 2 * (size_t)sw + (size_t)max_rows + kSolveThreads) + 128;   // + base alignment
}

// Offset of column k in a packed pw-wide inverse: sum over j < k of
// round4(pw - j) = S(pw) - S(pw - k), S(x) = sum_{m=1..x} round4(m)
// = x(x+1)/2 + 6 floor(x/4) + {0,3,5,6}[x mod 4].
__device__ __forceinline__ int packed_S(int x) {
  const int tail = (x & 3) == 0 ? 0 : ((x & 3) == 1 ? 3 : ((x & 3) == 2 ? 5 : 6));
  return x * (x + 1) / 2 + 6 * (x >> 2) + tail;
}
__device__ __forceinline__ int packed_off(int pw, int k) { return packed_S(pw) - packed_S(pw - k); }


// out_i = sum_k tile[k*cs + d0 + i] * x[k] for i < nr, handed to
// emit(i, u, out_i) with u the thread's row slot (i = tid + u * blockDim for
// u < 4, u = -1 beyond); the k range is split among thread groups when the
// rows are few, and with more rows than threads every sum is formed before
// the first is handed over
template <typename T, typename F>
__device__ void rows_matvec(const T* tile, int cs, int d0, int nr, int pw, const T* x, T* part, F emit) {
  const int tid = threadIdx.x;
  if (nr <= (int)blockDim.x) {
    const int rr = (nr + 31) & ~31;
    const int G = max(1, (int)blockDim.x / rr);
    const int i = tid % rr, g = tid / rr;
    // four independent partial sums (the FMA chain, not the shared-memory
    // loads, would otherwise set the pace)
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    if (g < G && i < nr) {
      const T* tc = tile + d0 + i;
      int k = g;
      for (; k + 3 * G < pw; k += 4 * G) {
        a0 += tc[k * cs] * x[k];
        a1 += tc[(k + G) * cs] * x[k + G];
        a2 += tc[(k + 2 * G) * cs] * x[k + 2 * G];
        a3 += tc[(k + 3 * G) * cs] * x[k + 3 * G];
      }
      for (; k < pw; k += G) a0 += tc[k * cs] * x[k];
    }
    part[tid] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (tid < nr) {
      T o = T(0);
      for (int gg = 0; gg < G; gg++) o += part[gg * rr + tid];
      emit(tid, 0, o);
    }
  } else {
    T acc4[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int i = tid + u * (int)blockDim.x;
      T acc = T(0);
      if (i < nr)
        for (int k = 0; k < pw; k++) acc += tile[k * cs + d0 + i] * x[k];
      acc4[u] = acc;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int i = tid + u * (int)blockDim.x;
      if (i < nr) emit(i, u, acc4[u]);
    }
    for (int i = tid + 4 * (int)blockDim.x; i < nr; i += blockDim.x) {
      T acc = T(0);
      for (int k = 0; k < pw; k++) acc += tile[k * cs + d0 + i] * x[k];
      emit(i, -1, acc);
    }
  }
}

// rows_matvec for R right-hand sides at once: out_ij = sum_k tile[k*cs + d0 + i]
// * X[j*pw + k], handed to emit(i, j, out_ij); each tile entry is read once
// for all of them (part: R * blockDim entries)
template <typename T, typename F>
__device__ void rows_matvec_multi(const T* tile, int cs, int d0, int nr, int pw, const T* X, int R, T* part, F emit) {
  const int tid = threadIdx.x;
  T acc[kMaxRhs];
#pragma unroll
  for (int j = 0; j < kMaxRhs; j++) acc[j] = T(0);
  if (nr <= (int)blockDim.x) {
    const int rr = (nr + 31) & ~31;
    const int G = max(1, (int)blockDim.x / rr);
    const int i = tid % rr, g = tid / rr;
    if (g < G && i < nr)
      for (int k = g; k < pw; k += G) {
        const T tv = tile[k * cs + d0 + i];
#pragma unroll
        for (int j = 0; j < kMaxRhs; j++)
          if (j < R) acc[j] += tv * X[j * pw + k];
      }
#pragma unroll
    for (int j = 0; j < kMaxRhs; j++)
      if (j < R) part[j * blockDim.x + tid] = acc[j];
    __syncthreads();
    if (tid < nr)
      for (int j = 0; j < R; j++) {
        T o = T(0);
        for (int gg = 0; gg < G; gg++) o += part[j * blockDim.x + gg * rr + tid];
        emit(tid, j, o);
      }
  } else {
    for (int i = tid; i < nr; i += blockDim.x) {
#pragma unroll
      for (int j = 0; j < kMaxRhs; j++) acc[j] = T(0);
      for (int k = 0; k < pw; k++) {
        const T tv = tile[k * cs + d0 + i];
#pragma unroll
        for (int j = 0; j < kMaxRhs; j++)
          if (j < R) acc[j] += tv * X[j * pw + k];
      }
#pragma unroll
      for (int j = 0; j < kMaxRhs; j++)
        if (j < R) emit(i, j, acc[j]);
    }
  }
}

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

// Sums eight per-lane values over the warp at once: each halving step trades
// half of a lane's columns with the partner lane, so the eight totals take
// 4 + 2 + 1 + 1 + 1 shuffles instead of 8 x 5. On return lanes 4c..4c+3
// hold the total of column c in v[0].
template <typename T>
__device__ __forceinline__ T warp_sum8(T (&v)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const T send = b4 ? v[j] : v[j + 4];
    const T keep = b4 ? v[j + 4] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const T send = b3 ? v[j] : v[j + 2];
    const T keep = b3 ? v[j + 2] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const T send = b2 ? v[0] : v[1];
    const T keep = b2 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

// thread 0: charge the cycles since the last mark to phase i (profile runs)
template <typename T>
__device__ __forceinline__ void mark(const SolveArgs<T>& a, SolveSmemHdr& h, int i) {
  if (a.instr && threadIdx.x == 0) {
    const long long now = clock64();
    if (i >= 0) h.c_ph[i] += now - h.t_mark;
    h.t_mark = now;
  }
}

// ------------------------------------------------------- TMA bulk copies
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(m)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* m, unsigned phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(m))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 3-D tiled TMA load of the box at (x = row, y = column, z = system of a batch)
// of a tensor map held in global memory; x * element size is a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          saddr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(saddr(m))
      : "memory");
}

// All threads: wait for the current bulk copies (bounded). On timeout the
// abort word is set and the wait is retried once more, bounded, so that no
// copy is left in flight into this CTA's shared memory.
template <typename T>
__device__ bool mbar_wait(const SolveArgs<T>& a, SolveSmemHdr& h) {
  const long long tw = clock64();
  const unsigned ph = h.phase;
  bool ok = mbar_test(&h.mbar, ph);
  if (!ok) {
    long long t0 = clock64();
    while (!(ok = mbar_test(&h.mbar, ph))) {
      if (clock64() - t0 > a.spin) {
        atomicExch(&a.st->abort, 1);
        t0 = clock64();
        while (!mbar_test(&h.mbar, ph) && clock64() - t0 < a.spin) {}
        break;
      }
    }
  }
  ok = __syncthreads_and(ok);   // every thread takes the same exit
  if (threadIdx.x == 0) {
    h.phase ^= 1u;
    h.c_mbar += clock64() - tw;
  }
  __syncthreads();
  return ok;
}

// Warp 0 stages rows [r0, r0 + nrows) (piece-local) of the piece's pw
// columns into `tile` (column stride cs), starting at the supernode row
// rounded down to 4 so every copy starts on 16 bytes (offset returned):
// one 2-D TMA box through the piece's tensor map when tma is set (cs = the
// box rows; rows past the panel read as zeros), else one bulk copy per column.
template <typename T>
__device__ int stage_tile(const SolveArgs<T>& a, int p, int64_t colbase, int ld, int c, int pw, int r0, int nrows,
                          int cs, int tma, T* tile, uint32_t& bytes_out, unsigned long long* mbar, bool issue) {
  const int R0 = c + r0;
  const int A0 = R0 & ~3;
  if (tma) {
    bytes_out = (uint32_t)cs * (uint32_t)pw * (uint32_t)sizeof(T);
    if (issue && threadIdx.x == 0) tma_load_3d(tile, a.tmaps + (int64_t)p * 128, A0, 0, a.tz, mbar);
  } else {
    const int E = (R0 + nrows + 3) & ~3;
    const uint32_t bytes = (uint32_t)(E - A0) * (uint32_t)sizeof(T);
    bytes_out = bytes * (uint32_t)pw;
    if (issue) {
      const T* base = a.L + colbase + A0;
      for (int k = threadIdx.x; k < pw; k += 32) bulk_g2s(tile + (int64_t)k * cs, base + (int64_t)k * ld, bytes, mbar);
    }
  }
  return R0 - A0;
}

// Publish (the 32 lanes of one warp, after a CTA barrier that follows the
// CTA's writes): one arrival on counters[tg[q]] for every q in [q0, q1). Each
// lane fences before its increments, and the fence is cumulative over the
// writes the barrier ordered before it; the lanes spread the index loads and
// increments of a long target list.
__device__ __forceinline__ void signal_all(int* counters, const int32_t* tg, int64_t q0, int64_t q1) {
  __threadfence();
  for (int64_t q = q0 + (threadIdx.x & 31); q < q1; q += 32) atomicAdd(&counters[__ldg(&tg[q])], 1);
}

// out[i] = v[rows[i]] for i < nr <= 4 * blockDim: every row index is loaded
// before any value, so the block waits two memory round trips, not 2 per
// blockDim rows.
template <typename T>
__device__ __forceinline__ void gather_rows(const T* v, const int32_t* rows, int nr, T* out) {
  const int tid = threadIdx.x, bd = blockDim.x;
  int r[4];
#pragma unroll
  for (int u = 0; u < 4; u++) r[u] = tid + u * bd < nr ? __ldg(&rows[tid + u * bd]) : -1;
  T x[4];
#pragma unroll
  for (int u = 0; u < 4; u++) x[u] = r[u] >= 0 ? ldcg(&v[r[u]]) : T(0);
#pragma unroll
  for (int u = 0; u < 4; u++)
    if (r[u] >= 0) out[tid + u * bd] = x[u];
  for (int i = tid + 4 * bd; i < nr; i += bd) out[i] = ldcg(&v[rows[i]]);
}

// The sn_rows entries of rows tid + u * blockDim (u < 4) of an item, fetched
// before the item waits on its inputs (0 past nr).
__device__ __forceinline__ void prefetch_rows4(const int32_t* rows, int nr, int (&r)[4]) {
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int i = (int)threadIdx.x + u * (int)blockDim.x;
    r[u] = i < nr ? __ldg(&rows[i]) : 0;
  }
}

// The sn_rows entry of row i of an item (i < nr), fetched before the item
// waits on its inputs when the item has at most one row per thread.
__device__ __forceinline__ int prefetch_row(const int32_t* rows, int nr) {
  return (int)threadIdx.x < nr ? __ldg(&rows[threadIdx.x]) : 0;
}

// --------------------------------------------------------------- forward
template <typename T>
__device__ bool fwd_head(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int p, int e) {
  const int tid = threadIdx.x;
  mark(a, h, -1);
  const HeadDesc d = a.hdesc[p];
  const int pw = d.pw, f = d.f, rn = d.rn;
  const int32_t* rows = a.sn_rows + d.rowbase + pw;
  int myrows[4];
  prefetch_rows4(rows, rn, myrows);
  if (tid < 32) {
    uint32_t b1 = 0;
    if (tid == 0) fence_proxy_async();
    const uint32_t binv = (uint32_t)((d.inv1 - d.inv0) * sizeof(T));
    if (rn > 0) stage_tile(a, p, d.colbase, d.ld, d.c, pw, pw, rn, d.cs, d.tma, t.B, b1, &h.mbar, false);
    if (tid == 0) mbar_expect_tx(&h.mbar, binv + b1);
    __syncwarp();
    if (tid == 0) bulk_g2s(t.A, a.Linv + d.inv0, binv, &h.mbar);
    if (rn > 0) stage_tile(a, p, d.colbase, d.ld, d.c, pw, pw, rn, d.cs, d.tma, t.B, b1, &h.mbar, true);
    mark(a, h, 0);
    if (tid == 0) {
      const long long t0 = clock64();
      h.flag = wait_geq(&a.fwd_arrive[p], e * d.need, a.st, a.spin);
      h.c_dep += clock64() - t0;
    }
    mark(a, h, 1);
  }
  __syncthreads();
  const bool dep = h.flag != 0;
  if (dep)
    for (int i = tid; i < pw; i += blockDim.x) t.vec[i] = ldcg(&a.v[f + i]);
  if (!mbar_wait(a, h) || !dep) return false;
  mark(a, h, 2);
  // y = T^-1 b with the packed inverse (column k holds rows k..pw-1); the
  // k range of each row is split into G contiguous parts, one per thread
  // group, walked with a running column offset and two partial sums
  const int pr = (pw + 31) & ~31;
  const int G = max(1, (int)blockDim.x / pr);
  const int gi = tid % pr, gg0 = tid / pr;
  const int kspan = (pw + G - 1) / G;
  const int kb = gg0 * kspan, ke = min(gi + 1, kb + kspan);
  const int off0 = gg0 < G && kb < pw ? packed_off(pw, kb) : 0;
  for (int j = 0; j < a.nrhs; j++) {
    T* vj = a.v + (int64_t)j * a.n;
    if (j > 0) {
      for (int i = tid; i < pw; i += blockDim.x) t.vec[i] = ldcg(&vj[f + i]);
      __syncthreads();
    }
    T acc = T(0), acc2 = T(0);
    if (gg0 < G && gi < pw) {
      int off = off0, k = kb;
      for (; k + 1 < ke; k += 2) {
        acc += t.A[off + gi - k] * t.vec[k];
        off += (pw - k + 3) & ~3;
        acc2 += t.A[off + gi - k - 1] * t.vec[k + 1];
        off += (pw - k + 2) & ~3;
      }
      if (k < ke) acc += t.A[off + gi - k] * t.vec[k];
    }
    t.aux[tid] = acc + acc2;
    __syncthreads();
    if (tid < pw) {
      T y = T(0);
      for (int g = 0; g < G; g++) y += t.aux[g * pr + tid];
      t.vec2[tid] = y;
      vj[f + tid] = y;
    }
    __syncthreads();
  }
  mark(a, h, 14);
  // the piece's done flag (its chunks wait on it) goes out after chunk 0, so
  // the fence of chunk 0's arrivals serves both and the next piece's head,
  // usually on the critical path, does not wait for a second one
  if (rn == 0 && tid == 0) st_release(&a.fwd_done[p], e);
  if (rn > 0) {
    // chunk 0: b[rows] -= L21(0:rn) y
    const int d0 = (d.c + pw) & 3;
    for (int j = 0; j < a.nrhs; j++) {
      T* vj = a.v + (int64_t)j * a.n;
      if (a.nrhs > 1) {
        for (int i = tid; i < pw; i += blockDim.x) t.vec2[i] = ldcg(&vj[f + i]);
        __syncthreads();
      }
      rows_matvec(t.B, d.cs, d0, rn, pw, t.vec2, t.aux, [&](int i, int u, T o) {
        atomicAdd(&vj[u >= 0 ? myrows[u] : rows[i]], -o);
      });
      __syncthreads();
    }
    if (tid < 32) {
      signal_all(a.fwd_arrive, a.hd_tgt, d.tp0, d.tp1);
      if (tid == 0) st_relaxed(&a.fwd_done[p], e);   // ordered by signal_all's fence
    }
  }
  mark(a, h, 15);
  return true;
}

template <typename T>
__device__ bool fwd_chunk(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int c, int e) {
  const int tid = threadIdx.x;
  mark(a, h, -1);
  const ChunkDesc d = a.cdesc[c];
  const int p = d.p, pw = d.pw, f = d.f, nr = d.nr;
  const int32_t* rows = a.sn_rows + d.rowbase;
  int myrows[4];
  prefetch_rows4(rows, nr, myrows);
  const int myrow = myrows[0];
  if (tid < 32) {
    uint32_t b = 0;
    if (tid == 0) fence_proxy_async();
    stage_tile(a, p, d.colbase, d.ld, d.c, pw, d.r0, nr, d.cs, d.tma, t.C, b, &h.mbar, false);
    if (tid == 0) mbar_expect_tx(&h.mbar, b);
    __syncwarp();
    stage_tile(a, p, d.colbase, d.ld, d.c, pw, d.r0, nr, d.cs, d.tma, t.C, b, &h.mbar, true);
    mark(a, h, 3);
    if (tid == 0) {
      const long long t0 = clock64();
      h.flag = wait_geq(&a.fwd_done[p], e, a.st, a.spin);
      h.c_dep += clock64() - t0;
    }
    mark(a, h, 4);
  }
  __syncthreads();
  const bool dep = h.flag != 0;
  const int R = a.nrhs;
  if (R > 1 && !a.ov && R * pw <= a.max_rows + kSolveThreads && (size_t)R * blockDim.x <= packed_inv((size_t)a.sw)) {
    // all right-hand sides' piece vectors at once (into the gathered-vector
    // region; chunks leave the inverse region free for the partial sums)
    T* X = t.aux;
    if (dep)
      for (int idx = tid; idx < R * pw; idx += blockDim.x)
        X[idx] = ldcg(&a.v[(int64_t)(idx / pw) * a.n + f + idx % pw]);
    if (!mbar_wait(a, h) || !dep) return false;
    const int d0 = (d.c + d.r0) & 3;
    rows_matvec_multi(t.C, d.cs, d0, nr, pw, X, R, t.A, [&](int i, int j, T o) {
      atomicAdd(&a.v[(int64_t)j * a.n + (nr <= (int)blockDim.x ? myrow : rows[i])], -o);
    });
    __syncthreads();
    if (tid < 32) signal_all(a.fwd_arrive, a.ch_tgt, d.tp0, d.tp1);
    return true;
  }
  if (dep)
    for (int k = tid; k < pw; k += blockDim.x) t.vec[k] = ldcg(&a.v[f + k]);
  if (!mbar_wait(a, h) || !dep) return false;
  mark(a, h, 5);
  const int d0 = (d.c + d.r0) & 3;
  for (int j = 0; j < a.nrhs; j++) {
    T* vj = a.v + (int64_t)j * a.n;
    if (j > 0) {
      for (int k = tid; k < pw; k += blockDim.x) t.vec[k] = ldcg(&vj[f + k]);
      __syncthreads();
    }
    rows_matvec(t.C, d.cs, d0, nr, pw, t.vec, t.aux, [&](int i, int u, T o) {
      atomicAdd(&vj[u >= 0 ? myrows[u] : rows[i]], -o);
    });
    __syncthreads();
  }
  mark(a, h, 6);
  if (tid < 32) signal_all(a.fwd_arrive, a.ch_tgt, d.tp0, d.tp1);
  mark(a, h, 7);
  return true;
}

// --------------------------------------------------------------- backward
template <typename T>
__device__ bool bwd_chunk(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int c, int e) {
  const int tid = threadIdx.x;
  const ChunkDesc d = a.cdesc[c];
  const int p = d.p, pw = d.pw, nr = d.nr;
  const int32_t* rows = a.sn_rows + d.rowbase;
  const int myrow = prefetch_row(rows, nr);
  if (tid < 32) {
    uint32_t b = 0;
    if (tid == 0) fence_proxy_async();
    stage_tile(a, p, d.colbase, d.ld, d.c, pw, d.r0, nr, d.cs, d.tma, t.C, b, &h.mbar, false);
    if (tid == 0) mbar_expect_tx(&h.mbar, b);
    __syncwarp();
    stage_tile(a, p, d.colbase, d.ld, d.c, pw, d.r0, nr, d.cs, d.tma, t.C, b, &h.mbar, true);
    const long long t0 = clock64();
    const bool ok = warp_wait_all(a.bwd_done, a.ch_tgt, d.tp0, d.tp1, e, a.st, a.spin);
    if (tid == 0) {
      h.flag = ok ? 1 : 0;
      h.c_dep += clock64() - t0;
    }
  }
  __syncthreads();
  const bool dep = h.flag != 0;
  auto gather = [&](const T* vj) {
    if (nr <= (int)blockDim.x) {
      if (tid < nr) t.aux[tid] = ldcg(&vj[myrow]);
    } else {
      gather_rows(vj, rows, nr, t.aux);
    }
  };
  const int R = a.nrhs;
  const int d0 = (d.c + d.r0) & 3;
  const int cs = d.cs;
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (R > 1 && !a.ov && (size_t)R * nr <= packed_inv((size_t)a.sw)) {
    // every right-hand side's values at the chunk rows at once (inverse region)
    T* Gx = t.A;
    if (dep)
      for (int idx = tid; idx < R * nr; idx += blockDim.x) {
        const int j = idx / nr, i = idx % nr;
        Gx[idx] = ldcg(&a.v[(int64_t)j * a.n + (i == tid && nr <= (int)blockDim.x ? myrow : rows[i])]);
      }
    if (!mbar_wait(a, h) || !dep) return false;
    for (int k = warp; k < pw; k += nw) {
      T acc[kMaxRhs];
#pragma unroll
      for (int j = 0; j < kMaxRhs; j++) acc[j] = T(0);
      for (int i = lane; i < nr; i += 32) {
        const T tv = t.C[k * cs + d0 + i];
#pragma unroll
        for (int j = 0; j < kMaxRhs; j++)
          if (j < R) acc[j] += tv * Gx[j * nr + i];
      }
#pragma unroll
      for (int j = 0; j < kMaxRhs; j++)
        if (j < R) {
          const T sj = warp_sum(acc[j]);
          if (lane == 0) atomicAdd(&a.v[(int64_t)j * a.n + d.f + k], -sj);
        }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(&a.bwd_arrive[p], 1);
    }
    return true;
  }
  if (dep) gather(a.v);
  if (!mbar_wait(a, h) || !dep) return false;
  for (int j = 0; j < a.nrhs; j++) {
    if (j > 0) {
      gather(a.v + (int64_t)j * a.n);
      __syncthreads();
    }
    T* vj = a.v + (int64_t)j * a.n + d.f;
    for (int k0 = 8 * warp; k0 < pw; k0 += 8 * nw) {
      T acc[8];
#pragma unroll
      for (int q = 0; q < 8; q++) acc[q] = T(0);
      for (int i = lane; i < nr; i += 32) {
        const T xv = t.aux[i];
#pragma unroll
        for (int q = 0; q < 8; q++)
          if (k0 + q < pw) acc[q] += t.C[(k0 + q) * cs + d0 + i] * xv;
      }
      const T sum = warp_sum8(acc);
      const int k = k0 + (lane >> 2);
      if ((lane & 3) == 0 && k < pw) atomicAdd(&vj[k], -sum);
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    atomicAdd(&a.bwd_arrive[p], 1);
  }
  return true;
}

template <typename T>
__device__ bool bwd_head(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int p, int e) {
  const int tid = threadIdx.x;
  mark(a, h, -1);
  const HeadDesc d = a.hdesc[p];
  const int pw = d.pw, f = d.f, rn = d.rn, nch = d.nch;
  const int32_t* rows = a.sn_rows + d.rowbase + pw;
  const int myrow = prefetch_row(rows, rn);
  if (tid < 32) {
    uint32_t b1 = 0;
    if (tid == 0) fence_proxy_async();
    const uint32_t binv = (uint32_t)((d.inv1 - d.inv0) * sizeof(T));
    if (rn > 0) stage_tile(a, p, d.colbase, d.ld, d.c, pw, pw, rn, d.cs, d.tma, t.B, b1, &h.mbar, false);
    if (tid == 0) mbar_expect_tx(&h.mbar, binv + b1);
    __syncwarp();
    if (tid == 0) bulk_g2s(t.A, a.Linv + d.inv0, binv, &h.mbar);
    if (rn > 0) stage_tile(a, p, d.colbase, d.ld, d.c, pw, pw, rn, d.cs, d.tma, t.B, b1, &h.mbar, true);
    mark(a, h, 8);
    const long long t0 = clock64();
    bool ok = warp_wait_all(a.bwd_done, a.hd_tgt, d.tp0, d.tp1, e, a.st, a.spin);
    if (tid == 0) {
      ok = ok && wait_geq(&a.bwd_arrive[p], e * nch, a.st, a.spin);
      h.flag = ok ? 1 : 0;
      h.c_dep += clock64() - t0;
    }
    mark(a, h, 9);
  }
  __syncthreads();
  const bool dep = h.flag != 0;
  // t = v[cols] (the piece's chunks have already subtracted their products
  // from it) and v at the chunk-0 rows
  auto gather = [&](int j) {
    const T* vj = a.v + (int64_t)j * a.n;
    if (rn <= (int)blockDim.x) {
      if (tid < rn) t.aux[tid] = ldcg(&vj[myrow]);
    } else {
      gather_rows(vj, rows, rn, t.aux);
    }
    for (int i = tid; i < pw; i += blockDim.x) t.vec[i] = ldcg(&vj[f + i]);
  };
  if (dep) gather(0);
  if (!mbar_wait(a, h) || !dep) return false;
  mark(a, h, 10);
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < a.nrhs; j++) {
    if (j > 0) {
      gather(j);
      __syncthreads();
    }
    // each warp takes eight columns at a time and sums them together
    if (rn > 0) {
      const int d0 = (d.c + pw) & 3;
      const int cs = d.cs;
      for (int k0 = 8 * warp; k0 < pw; k0 += 8 * nw) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; q++) acc[q] = T(0);
        for (int i = lane; i < rn; i += 32) {
          const T xv = t.aux[i];
#pragma unroll
          for (int q = 0; q < 8; q++)
            if (k0 + q < pw) acc[q] += t.B[(k0 + q) * cs + d0 + i] * xv;
        }
        const T sum = warp_sum8(acc);
        const int k = k0 + (lane >> 2);
        if ((lane & 3) == 0 && k < pw) t.vec[k] -= sum;
      }
      __syncthreads();
    }
    mark(a, h, 11);
    // x = T^-T t: x_k = sum_{i >= k} Tinv[i, k] t_i (packed columns)
    for (int k0 = 8 * warp; k0 < pw; k0 += 8 * nw) {
      T acc[8];
      int off[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        acc[q] = T(0);
        off[q] = packed_off(pw, min(k0 + q, pw - 1)) - (k0 + q);
      }
      for (int i = k0 + lane; i < pw; i += 32) {
        const T tv = t.vec[i];
#pragma unroll
        for (int q = 0; q < 8; q++)
          if (i >= k0 + q) acc[q] += t.A[off[q] + i] * tv;
      }
      const T sum = warp_sum8(acc);
      const int k = k0 + (lane >> 2);
      if ((lane & 3) == 0 && k < pw) t.vec2[k] = sum;
    }
    __syncthreads();
    mark(a, h, 12);
    T* vj = a.v + (int64_t)j * a.n;
    for (int i = tid; i < pw; i += blockDim.x) vj[f + i] = t.vec2[i];
    __syncthreads();
  }
  if (tid == 0) st_release(&a.bwd_done[p], e);
  mark(a, h, 13);
  return true;
}


// ------------------------------------------------------------ small subtrees
// A subtree whose columns [clo, chi) fit in shared memory is solved by one
// CTA: its descendants are all inside it, so in the forward sweep it depends
// on nothing and in the backward sweep only on the pieces owning its rows
// outside [clo, chi). Its supernodes are consecutive, so their panels and
// the inverses of their triangles are two contiguous ranges, each staged
// into shared memory with one bulk copy (the plan keeps both within the
// tile regions).
template <typename T>
__device__ void stage_subtree(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int st, int64_t& pbase,
                              int64_t& ibase) {
  const int s0 = a.st_first[st], s1 = a.st_last[st];
  pbase = a.poff[s0];
  ibase = a.pc_inv[a.sn_piece[s0]];
  if (threadIdx.x == 0) {
    const uint32_t bp = (uint32_t)((a.poff[s1] + (int64_t)a.sld[s1] * a.sw_[s1] - pbase) * sizeof(T));
    const uint32_t bi = (uint32_t)((a.pc_inv[a.sn_piece[s1] + 1] - ibase) * sizeof(T));
    fence_proxy_async();
    mbar_expect_tx(&h.mbar, bp + bi);
    bulk_g2s(t.B, a.L + pbase, bp, &h.mbar);
    bulk_g2s(t.A, a.Linv + ibase, bi, &h.mbar);
  }
}

// Forward step of one subtree supernode by one warp: y = T^-1 x on its
// columns (packed inverse), then x[row] -= L21 y for its rows below, into
// shared memory inside the subtree's column range and into v outside it.
template <typename T>
__device__ void warp_fwd_supernode(const SolveArgs<T>& a, const Tiles<T>& t, int s, int clo, int chi,
                                   int64_t pbase, int64_t ibase, T* xs, T* vj) {
  const int lane = threadIdx.x & 31;
  const int w = __ldg(&a.sw_[s]), nr = __ldg(&a.snr[s]), ld = __ldg(&a.sld[s]), f = __ldg(&a.sfirst[s]) - clo;
  const T* P = t.B + (__ldg(&a.poff[s]) - pbase);
  const T* Inv = t.A + (__ldg(&a.pc_inv[__ldg(&a.sn_piece[s])]) - ibase);
  const int32_t* rows = a.sn_rows + __ldg(&a.srow[s]);
  // lane owns rows lane + 32c; the k loop runs once for all four of them
  T y[4] = {T(0), T(0), T(0), T(0)};
  {
    int off = 0;
    for (int k = 0; k < w; k++) {
      const T xk = xs[f + k];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const int i = lane + 32 * c;
        if (i >= k && i < w) y[c] += Inv[off + i - k] * xk;
      }
      off += (w - k + 3) & ~3;
    }
  }
  __syncwarp();
#pragma unroll
  for (int c = 0; c < 4; c++)
    if (lane + 32 * c < w) xs[f + lane + 32 * c] = y[c];
  __syncwarp();
  for (int r = w + lane; r < nr; r += 128) {
    int rr[4];
    T o[4];
#pragma unroll
    for (int u = 0; u < 4; u++) rr[u] = r + 32 * u < nr ? __ldg(&rows[r + 32 * u]) : -1;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      o[u] = T(0);
      if (rr[u] >= 0)
        for (int k = 0; k < w; k++) o[u] += P[r + 32 * u + k * ld] * xs[f + k];
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (rr[u] < 0) continue;
      if (rr[u] < chi) atomicAdd(&xs[rr[u] - clo], -o[u]);
      else atomicAdd(&vj[rr[u]], -o[u]);
    }
  }
}

// Backward step of one subtree supernode by one warp: t = x - L21^T x[rows]
// on its columns, then x = T^-T t. Scratch of this warp (kSubScratch
// entries): t (w <= 128 entries), then x at the first rows below.
constexpr int kSubScratch = 160;
template <typename T>
__device__ void warp_bwd_supernode(const SolveArgs<T>& a, const Tiles<T>& t, int s, int clo, int chi,
                                   int64_t pbase, int64_t ibase, T* xs, T* scratch, const T* vj) {
  const int lane = threadIdx.x & 31;
  const int w = __ldg(&a.sw_[s]), nr = __ldg(&a.snr[s]), ld = __ldg(&a.sld[s]), f = __ldg(&a.sfirst[s]) - clo;
  const T* P = t.B + (__ldg(&a.poff[s]) - pbase);
  const T* Inv = t.A + (__ldg(&a.pc_inv[__ldg(&a.sn_piece[s])]) - ibase);
  const int32_t* rows = a.sn_rows + __ldg(&a.srow[s]);
  // gather x at the rows below into the scratch after t (w entries) once;
  // rows beyond the scratch are read where they are
  T* xr = scratch + w;
  const int cache = kSubScratch - w;
  const int nb = nr - w;
  for (int r = lane; r < nb && r < cache; r += 32) {
    const int row = __ldg(&rows[w + r]);
    xr[r] = row < chi ? xs[row - clo] : ldcg(&vj[row]);
  }
  __syncwarp();
  // eight columns at a time: a row past the cache is fetched once per eight
  for (int k0 = 0; k0 < w; k0 += 8) {
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = T(0);
    for (int r = lane; r < nb; r += 32) {
      T x;
      if (r < cache) {
        x = xr[r];
      } else {
        const int row = __ldg(&rows[w + r]);
        x = row < chi ? xs[row - clo] : ldcg(&vj[row]);
      }
#pragma unroll
      for (int q = 0; q < 8; q++)
        if (k0 + q < w) acc[q] += P[w + r + (k0 + q) * ld] * x;
    }
    const T sum = warp_sum8(acc);
    const int k = k0 + (lane >> 2);
    if ((lane & 3) == 0 && k < w) scratch[k] = xs[f + k] - sum;
  }
  __syncwarp();
  // x = T^-T t (packed columns: column k holds rows k..w-1)
  for (int k0 = 0; k0 < w; k0 += 8) {
    T acc[8];
    int off[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      acc[q] = T(0);
      off[q] = packed_off(w, min(k0 + q, w - 1)) - (k0 + q);
    }
    for (int i = k0 + lane; i < w; i += 32) {
      const T tv = scratch[i];
#pragma unroll
      for (int q = 0; q < 8; q++)
        if (i >= k0 + q) acc[q] += Inv[off[q] + i] * tv;
    }
    const T sum = warp_sum8(acc);
    const int k = k0 + (lane >> 2);
    if ((lane & 3) == 0 && k < w) xs[f + k] = sum;
  }
  __syncwarp();
}

// Small subtrees: the supernodes of one item are processed level by level
// (height above the item's leaves), one warp per supernode; supernodes of
// one level are independent, so one CTA barrier per level suffices.
template <typename T>
__device__ bool fwd_subtree(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int st) {
  const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;
  const int clo = a.st_clo[st], chi = a.st_chi[st];
  mark(a, h, -1);
  int64_t pbase, ibase;
  stage_subtree(a, h, t, st, pbase, ibase);
  T* xs = t.vec2;
  for (int i = tid; i < chi - clo; i += blockDim.x) xs[i] = ldcg(&a.v[clo + i]);
  if (!mbar_wait(a, h)) return false;
  const long long tl0 = clock64();
  for (int j = 0; j < a.nrhs; j++) {
    T* vj = a.v + (int64_t)j * a.n;
    if (j > 0) {
      for (int i = tid; i < chi - clo; i += blockDim.x) xs[i] = ldcg(&vj[clo + i]);
      __syncthreads();
    }
    for (int L = a.st_lptr[st]; L + 1 < a.st_lptr[st + 1]; L++) {
      for (int q = a.st_lev[L] + warp; q < a.st_lev[L + 1]; q += nw)
        warp_fwd_supernode(a, t, a.st_sn[q], clo, chi, pbase, ibase, xs, vj);
      __syncthreads();
    }
    for (int i = tid; i < chi - clo; i += blockDim.x) vj[clo + i] = xs[i];
    __syncthreads();
  }
  if (tid == 0) {
    h.c_lvl += clock64() - tl0;
    h.n_lvl += a.st_lptr[st + 1] - a.st_lptr[st] - 1;
  }
  if (tid < 32) signal_all(a.fwd_arrive, a.st_tgt, a.st_tptr[st], a.st_tptr[st + 1]);
  return true;
}

template <typename T>
__device__ bool bwd_subtree(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int st, int e) {
  const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;
  const int clo = a.st_clo[st], chi = a.st_chi[st];
  int64_t pbase, ibase;
  stage_subtree(a, h, t, st, pbase, ibase);
  if (tid < 32) {
    const long long t0 = clock64();
    const bool ok = warp_wait_all(a.bwd_done, a.st_tgt, a.st_tptr[st], a.st_tptr[st + 1], e, a.st, a.spin);
    if (tid == 0) {
      h.flag = ok ? 1 : 0;
      h.c_dep += clock64() - t0;
    }
  }
  __syncthreads();
  const bool dep = h.flag != 0;
  T* xs = t.vec2;
  if (dep)
    for (int i = tid; i < chi - clo; i += blockDim.x) xs[i] = ldcg(&a.v[clo + i]);
  if (!mbar_wait(a, h) || !dep) return false;
  T* scratch = t.aux + kSubScratch * warp;   // 8 warps x 160 <= max_rows + kSolveThreads
  const long long tl0 = clock64();
  for (int j = 0; j < a.nrhs; j++) {
    T* vj = a.v + (int64_t)j * a.n;
    if (j > 0) {
      for (int i = tid; i < chi - clo; i += blockDim.x) xs[i] = ldcg(&vj[clo + i]);
      __syncthreads();
    }
    for (int L = a.st_lptr[st + 1] - 2; L >= a.st_lptr[st]; L--) {
      for (int q = a.st_lev[L] + warp; q < a.st_lev[L + 1]; q += nw)
        warp_bwd_supernode(a, t, a.st_sn[q], clo, chi, pbase, ibase, xs, scratch, vj);
      __syncthreads();
    }
    for (int i = tid; i < chi - clo; i += blockDim.x) vj[clo + i] = xs[i];
    __syncthreads();   // the results are read after the next grid barrier
  }
  if (tid == 0) {
    h.c_lvl += clock64() - tl0;
    h.n_lvl += a.st_lptr[st + 1] - a.st_lptr[st] - 1;
  }
  return true;
}

template <typename T>
__device__ bool grid_barrier(const SolveArgs<T>& a, SolveSmemHdr& h) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long tb = clock64();
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
    h.flag = ok;
    h.c_bar += clock64() - tb;
  }
  __syncthreads();
  return h.flag != 0;
}

// per-block partial sums of two values -> a.red[block * kRedStride + 2 slot + {0,1}]
template <typename T>
__device__ void block_partial2(const SolveArgs<T>& a, SolveSmemHdr& h, double v0, double v1, int slot = 0) {
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();   // the previous call's reader of dred is done
  if (lane == 0) { h.dred[warp * 2] = v0; h.dred[warp * 2 + 1] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < kSolveThreads / 32; w++) { s0 += h.dred[w * 2]; s1 += h.dred[w * 2 + 1]; }
    a.red[blockIdx.x * kRedStride + 2 * slot] = s0;
    a.red[blockIdx.x * kRedStride + 2 * slot + 1] = s1;
  }
}

// the same grid totals in every block (fixed summation order)
template <typename T>
__device__ void grid_total2(const SolveArgs<T>& a, SolveSmemHdr& h, double& t0, double& t1, int slot = 0) {
  if (threadIdx.x < 32) {
    double s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
      s0 += __ldcg(&a.red[b * kRedStride + 2 * slot]);
      s1 += __ldcg(&a.red[b * kRedStride + 2 * slot + 1]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (threadIdx.x == 0) { h.bcast[0] = s0; h.bcast[1] = s1; }
  }
  __syncthreads();
  t0 = h.bcast[0];
  t1 = h.bcast[1];
  __syncthreads();
}

template <typename T, bool FWD>
__device__ bool sweep(const SolveArgs<T>& a, SolveSmemHdr& h, const Tiles<T>& t, int seq, int e) {
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&a.disp[(seq + 1) % 3], 0);
  const int32_t* items = FWD ? a.fwd_items : a.bwd_items;
  for (;;) {
    // warp 1 takes the next ticket and reads its item code while warp 0 may
    // still be publishing the previous item (a fence and the arrival
    // atomics): the two round trips overlap instead of adding up
    long long td = 0;
    if (threadIdx.x == 0) td = clock64();
    if (threadIdx.x == 32) {
      const int t = atomicAdd(&a.disp[seq % 3], 1);
      h.item = t;
      h.code = t < a.nitems ? items[t] : 0;
    }
    __syncthreads();
    const int it = h.item;
    const int code = h.code;
    __syncthreads();
    unsigned long long tg0 = 0;
    if (threadIdx.x == 0) {
      const long long now = clock64();
      h.c_disp += now - td;
      td = now;
      if (a.trace) tg0 = globaltimer();
    }
    if (it >= a.nitems) return true;
    const int kind = code < -(int)a.npieces ? 0 : (code < 0 ? 1 : 2);
    bool ok;
    if (code < -(int)a.npieces) {
      const int st = -1 - (int)a.npieces - code;
      ok = FWD ? fwd_subtree(a, h, t, st) : bwd_subtree(a, h, t, st, e);
    } else if (FWD) {
      ok = code < 0 ? fwd_head(a, h, t, -1 - code, e) : fwd_chunk(a, h, t, code, e);
    } else {
      ok = code < 0 ? bwd_head(a, h, t, -1 - code, e) : bwd_chunk(a, h, t, code, e);
    }
    if (threadIdx.x == 0) {
      if (a.trace && seq < 2) {
        unsigned long long* q = a.trace + 3 * ((int64_t)seq * a.nitems + it);
        q[0] = tg0;
        q[1] = globaltimer();
        q[2] = blockIdx.x;
      }
      const long long dt = clock64() - td;
      h.c_item += dt;
      h.n_items++;
      h.c_kind[kind] += dt;
      h.n_kind[kind]++;
    }
    if (!ok) return false;
  }
}

// one H^-1 application on a.v (forward then backward sweep)
template <typename T>
__device__ void flush_counters(const SolveArgs<T>& a, SolveSmemHdr& h) {
  if (a.instr && threadIdx.x == 0) {
    atomicAdd(&a.instr[0], (unsigned long long)h.c_disp);
    atomicAdd(&a.instr[1], (unsigned long long)h.c_dep);
    atomicAdd(&a.instr[2], (unsigned long long)h.c_mbar);
    atomicAdd(&a.instr[3], (unsigned long long)h.c_item);
    atomicAdd(&a.instr[4], (unsigned long long)h.c_bar);
    atomicAdd(&a.instr[5], (unsigned long long)h.n_items);
    atomicAdd(&a.instr[6], 1ull);
    for (int k = 0; k < 3; k++) {
      atomicAdd(&a.instr[7 + 2 * k], (unsigned long long)h.c_kind[k]);
      atomicAdd(&a.instr[8 + 2 * k], (unsigned long long)h.n_kind[k]);
    }
    atomicAdd(&a.instr[13], (unsigned long long)h.c_lvl);
    atomicAdd(&a.instr[14], (unsigned long long)h.n_lvl);
    for (int k = 0; k < 16; k++) atomicAdd(&a.instr[16 + k], (unsigned long long)h.c_ph[k]);
  }
}

template <typename T>
__device__ bool hsolve(const SolveArgs<T>& a, SolveSmemHdr& sm, const Tiles<T>& t, int& seq, int& e) {
  e++;
  if (!sweep<T, true>(a, sm, t, seq++, e)) return false;
  if (!grid_barrier(a, sm)) return false;
  if (!sweep<T, false>(a, sm, t, seq++, e)) return false;
  return grid_barrier(a, sm);
}

// MB = resident CTAs per SM the register allocation is bounded for
template <typename T, int MB>
__global__ void __launch_bounds__(kSolveThreads, MB) k_cg(SolveArgs<T> a) {
  __shared__ SolveSmemHdr sm;
  extern __shared__ __align__(16) unsigned char dsm[];
  Tiles<T> tl;
  {
    // every region at a 128-byte aligned shared address (TMA boxes)
    const uint32_t sa = saddr(dsm);
    T* base = (T*)(dsm + ((128u - (sa & 127u)) & 127u));
    const SolveLayout l = solve_layout(sizeof(T), a.sw, a.ent, a.ent0, a.esub, a.ov);
    tl.A = base;
    tl.B = base + l.b_off;
    tl.C = base + l.c_off;
    tl.vec = base + l.vec_off;
  }
  tl.vec2 = tl.vec + a.sw;
  tl.aux = tl.vec2 + a.sw;
  if (threadIdx.x == 0) {
    mbar_init(&sm.mbar);
    sm.phase = 0;
    sm.c_disp = sm.c_dep = sm.c_mbar = sm.c_item = sm.c_bar = sm.n_items = 0;
    for (int k = 0; k < 3; k++) sm.c_kind[k] = sm.n_kind[k] = 0;
    sm.c_lvl = sm.n_lvl = 0;
    for (int k = 0; k < 16; k++) sm.c_ph[k] = 0;
    sm.t_mark = 0;
  }
  __syncthreads();
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = a.n, m = a.m;
  int seq = 0, e = 0;
  const int R = a.nrhs;
  // phase 0: r^_x = r_x + gamma J^T r_y in permuted labels; v = r^_x
  for (int j = 0; j < R; j++) {
    const double* bx = a.bx + (int64_t)j * n;
    const double* by = a.by + (int64_t)j * m;
    double* rhx = a.rhx + (int64_t)j * n;
    T* v = a.v + (int64_t)j * n;
    for (int64_t k = gt; k < n; k += gs) {
      const int32_t o = a.perm[k];
      double s = 0.0;
      if (a.mode == 0)
        for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * by[a.JT_row[q]];
      const double rh = bx[o] + a.gamma * s;
      rhx[k] = rh;
      v[k] = (T)rh;
    }
  }
  if (!grid_barrier(a, sm)) return;
  if (!hsolve(a, sm, tl, seq, e)) return;
  if (a.mode == 1) {
    for (int j = 0; j < R; j++) {
      const T* v = a.v + (int64_t)j * n;
      double* ox = a.ox + (int64_t)j * n;
      for (int64_t k = gt; k < n; k += gs) {
        const double val = (double)ldcg(&v[k]);
        const int32_t o = a.perm[k];
        ox[o] = a.accumulate ? ox[o] + val : val;
      }
    }
    flush_counters(a, sm);
    return;
  }
  // per-right-hand-side CG state: identical in every CTA (grid totals are
  // summed in a fixed order), kept in shared memory
  __shared__ double s_rho[kMaxRhs], s_rqmax[kMaxRhs], s_d2[kMaxRhs], s_bn2[kMaxRhs], s_alpha[kMaxRhs];
  __shared__ int s_it[kMaxRhs], s_status[kMaxRhs], s_brk[kMaxRhs], s_step[kMaxRhs];
  // keep w = H^-1 r^_x (FP64) and start dx = w
  for (int j = 0; j < R && a.xacc; j++) {
    const T* v = a.v + (int64_t)j * n;
    double* wv = a.wv + (int64_t)j * n;
    double* xa = a.xa + (int64_t)j * n;
    for (int64_t k = gt; k < n; k += gs) {
      const double wk = (double)ldcg(&v[k]);
      wv[k] = wk;
      xa[k] = wk;
    }
  }
  // b_S = J w - r_y
  for (int j = 0; j < R; j++) {
    const T* v = a.v + (int64_t)j * n;
    const double* by = a.by + (int64_t)j * m;
    double *bS = a.bS + j * m, *r = a.r + j * m, *p = a.p + j * m, *y = a.y + j * m;
    double part = 0.0;
    for (int64_t i = gt; i < m; i += gs) {
      double s = 0.0;
      for (int64_t q = a.J_rowptr[i]; q < a.J_rowptr[i + 1]; q++) s += a.Jv[q] * (double)ldcg(&v[a.Jcol_perm[q]]);
      const double b = s - by[i];
      bS[i] = b; r[i] = b; p[i] = b; y[i] = 0.0;
      part += b * b;
    }
    block_partial2(a, sm, part, 0.0, j);
  }
  if (!grid_barrier(a, sm)) return;
  for (int j = 0; j < R; j++) {
    double bn2, dummy;
    grid_total2(a, sm, bn2, dummy, j);
    if (threadIdx.x == 0) {
      s_bn2[j] = bn2; s_rho[j] = bn2; s_rqmax[j] = 0.0; s_d2[j] = 0.0;
      s_it[j] = 0; s_status[j] = -1; s_brk[j] = 0;
    }
  }
  __syncthreads();
  for (;;) {
    // status -1 = running; 0 converged, 3 breakdown, 4 iteration limit
    if (threadIdx.x == 0)
      for (int j = 0; j < R; j++) {
        if (s_status[j] != -1) continue;
        if (sqrt(s_rho[j]) <= a.rtol * sqrt(s_bn2[j])) s_status[j] = 0;
        else if (s_it[j] >= a.maxit) s_status[j] = 4;
      }
    __syncthreads();
    bool any = false;
    for (int j = 0; j < R; j++) any |= s_status[j] == -1;
    if (!any) break;
    // v = J^T p (finished right-hand sides ride along unchanged)
    for (int j = 0; j < R; j++) {
      const double* p = a.p + j * m;
      T* v = a.v + (int64_t)j * n;
      for (int64_t k = gt; k < n; k += gs) {
        double s = 0.0;
        for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * __ldcg(&p[a.JT_row[q]]);
        v[k] = (T)s;
      }
    }
    if (!grid_barrier(a, sm)) return;
    if (!hsolve(a, sm, tl, seq, e)) return;
    for (int j = 0; j < R; j++) {
      if (s_status[j] != -1) continue;
      const T* v = a.v + (int64_t)j * n;
      const double* p = a.p + j * m;
      double* q_ = a.q + j * m;
      const double d2 = s_d2[j];
      double pq = 0.0, pp = 0.0;
      for (int64_t i = gt; i < m; i += gs) {
        double s = 0.0;
        for (int64_t q = a.J_rowptr[i]; q < a.J_rowptr[i + 1]; q++) s += a.Jv[q] * (double)ldcg(&v[a.Jcol_perm[q]]);
        const double pi = __ldcg(&p[i]);
        const double qi = s + d2 * pi;
        q_[i] = qi;
        pq += pi * qi;
        pp += pi * pi;
      }
      block_partial2(a, sm, pq, pp, j);
    }
    if (!grid_barrier(a, sm)) return;
    // step kind per right-hand side: 1 = CG step, 2 = delta_2 restart
    for (int j = 0; j < R; j++) {
      if (s_status[j] != -1) continue;
      double PQ, PP;
      grid_total2(a, sm, PQ, PP, j);
      if (threadIdx.x == 0) {
        s_it[j]++;
        const double rq = PQ / PP;
        if (rq > s_rqmax[j]) s_rqmax[j] = rq;
        if (!(PQ > 0.0) || rq <= 1e-12 * s_rqmax[j]) {
          if (s_d2[j] == 0.0 && a.delta2 > 0.0) {   // restart once on S + delta_2 I
            s_brk[j] = 1; s_d2[j] = a.delta2; s_rqmax[j] = 0.0; s_rho[j] = s_bn2[j];
            s_step[j] = 2;
          } else {
            s_status[j] = 3;
            s_step[j] = 0;
          }
        } else {
          s_alpha[j] = s_rho[j] / PQ;
          s_step[j] = 1;
        }
      }
    }
    __syncthreads();
    for (int j = 0; j < R; j++) {
      if (s_status[j] != -1) continue;
      double *p = a.p + j * m, *r = a.r + j * m, *y = a.y + j * m;
      const double* q_ = a.q + j * m;
      if (s_step[j] == 2) {
        const double* bS = a.bS + j * m;
        for (int64_t i = gt; i < m; i += gs) {
          const double b = __ldcg(&bS[i]);
          y[i] = 0.0; r[i] = b; p[i] = b;
        }
        if (a.xacc) {
          const double* wv = a.wv + (int64_t)j * n;
          double* xa = a.xa + (int64_t)j * n;
          for (int64_t k = gt; k < n; k += gs) xa[k] = __ldcg(&wv[k]);
        }
        continue;
      }
      const double alpha = s_alpha[j];
      if (a.xacc) {
        // dx -= alpha t, t = H^-1 J^T p of this product (still in v)
        const T* v = a.v + (int64_t)j * n;
        double* xa = a.xa + (int64_t)j * n;
        for (int64_t k = gt; k < n; k += gs) xa[k] -= alpha * (double)ldcg(&v[k]);
      }
      double rr = 0.0;
      for (int64_t i = gt; i < m; i += gs) {
        const double pi = __ldcg(&p[i]), qi = __ldcg(&q_[i]);
        y[i] += alpha * pi;
        const double ri = __ldcg(&r[i]) - alpha * qi;
        r[i] = ri;
        rr += ri * ri;
      }
      block_partial2(a, sm, rr, 0.0, j);
    }
    if (!grid_barrier(a, sm)) return;
    for (int j = 0; j < R; j++) {
      if (s_status[j] != -1 || s_step[j] != 1) continue;
      double rho2, dummy;
      grid_total2(a, sm, rho2, dummy, j);
      const double beta = rho2 / s_rho[j];
      double* p = a.p + j * m;
      const double* r = a.r + j * m;
      for (int64_t i = gt; i < m; i += gs) p[i] = __ldcg(&r[i]) + beta * __ldcg(&p[i]);
      __syncthreads();
      if (threadIdx.x == 0) s_rho[j] = rho2;
    }
    if (!grid_barrier(a, sm)) return;
  }
  // dx = H^-1 (r^_x - J^T dy) (eq. Schur2): accumulated, or a direct solve
  if (!a.xacc) {
    for (int j = 0; j < R; j++) {
      const double* y = a.y + j * m;
      const double* rhx = a.rhx + (int64_t)j * n;
      T* v = a.v + (int64_t)j * n;
      for (int64_t k = gt; k < n; k += gs) {
        double s = 0.0;
        for (int64_t q = a.JT_ptr[k]; q < a.JT_ptr[k + 1]; q++) s += a.Jv[a.JT_vidx[q]] * __ldcg(&y[a.JT_row[q]]);
        v[k] = (T)(__ldcg(&rhx[k]) - s);
      }
    }
    if (!grid_barrier(a, sm)) return;
    if (!hsolve(a, sm, tl, seq, e)) return;
  }
  for (int j = 0; j < R; j++) {
    const double* xa = a.xa + (int64_t)j * n;
    const T* v = a.v + (int64_t)j * n;
    const double* y = a.y + j * m;
    double* ox = a.ox + (int64_t)j * n;
    double* oy = a.oy + j * m;
    for (int64_t k = gt; k < n; k += gs) {
      const double val = a.xacc ? __ldcg(&xa[k]) : (double)ldcg(&v[k]);
      const int32_t o = a.perm[k];
      ox[o] = a.accumulate ? ox[o] + val : val;
    }
    for (int64_t i = gt; i < m; i += gs) {
      const double yi = __ldcg(&y[i]);
      oy[i] = a.accumulate ? oy[i] + yi : yi;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int it = 0, status = 0, brk = 0;
    for (int j = 0; j < R; j++) {
      a.rhs_stat[3 * j] = s_it[j];
      a.rhs_stat[3 * j + 1] = s_status[j];
      a.rhs_stat[3 * j + 2] = s_brk[j];
      it = max(it, s_it[j]);
      status = max(status, s_status[j]);
      brk |= s_brk[j];
    }
    a.st->cg_iters = it;
    a.st->cg_status = status;
    a.st->breakdown = brk;
  }
  flush_counters(a, sm);
}

template <typename T>
using CgKernel = void (*)(SolveArgs<T>);

template <typename T>
static CgKernel<T> cg_kernel(int ctas) {
  return ctas >= 4 ? k_cg<T, 4> : (ctas == 3 ? k_cg<T, 3> : k_cg<T, 2>);
}

template <typename T>
int solve_grid_size(int device, int sw, int ent, int ent0, int esub, int max_rows, int ov, int ctas) {
  int sms = 0, per = 0, maxsm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  const size_t smem = solve_smem_bytes(sizeof(T), sw, ent, ent0, esub, max_rows, ov);
  if (smem > (size_t)maxsm) return 0;
  auto k = cg_kernel<T>(ctas);
  if (raise_smem_limit(k, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kSolveThreads, smem);
  if (per < 1) return 0;
  return sms * std::min(per, std::max(ctas, 2));
}

template <typename T>
cudaError_t launch_solve(const SolveArgs<T>& a, int grid, int ctas, cudaStream_t st) {
  SolveArgs<T> args = a;
  void* params[] = {&args};
  const size_t smem = solve_smem_bytes(sizeof(T), a.sw, a.ent, a.ent0, a.esub, a.max_rows, a.ov);
  return cudaLaunchCooperativeKernel((const void*)cg_kernel<T>(ctas), dim3(grid), dim3(kSolveThreads), params, smem,
                                     st);
}

template int solve_grid_size<double>(int, int, int, int, int, int, int, int);
template int solve_grid_size<float>(int, int, int, int, int, int, int, int);
template cudaError_t launch_solve<double>(const SolveArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_solve<float>(const SolveArgs<float>&, int, int, cudaStream_t);

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
