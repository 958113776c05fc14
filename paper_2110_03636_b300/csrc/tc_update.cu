// Dense supernode updates on the 5th-generation tensor cores (tcgen05) for
// the FP32 factor (Sec. 4, eq. gamma: the multifrontal Cholesky of H_gamma;
// Algorithm 1's "chol(H_delta)").
//
// One tile computes C = A B^T over a K range of one front's panel, where A
// and B are 128-row blocks of the panel (column-major, ld = sld[s]):
//   mode 0 (update matrix):  U_s[gi, gj] = -C   (the SYRK U_s = -L21 L21^T)
//   mode 1 (in-panel):       P[row, col] -= C   (right-looking panel update)
//
// Precision. Each FP32 operand x is split into TF32 parts hi = rna(x),
// lo = rna(x - hi) (22 significant bits together) and the product is taken
// as hi*hi + hi*lo + lo*hi, the split-precision scheme of Ootomo & Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing
// the FP32 theoretical peak performance" (2022). The tensor core accumulates
// in FP32 without rounding to nearest, so its accumulator in tensor memory
// only ever holds kGroup K chunks: the epilogue warps drain it after each
// group and sum the groups with round-to-nearest FP32 adds, so the
// accumulation error grows with the number of groups the way an FMA loop's
// does, not with K.
//
// Two launches per tensor-core step:
//   k_tc_split   splits the step's operands once: each 128-row block x 16-K
//                chunk of a front's rows becomes one operand tile (hi then lo,
//                8 KB each) in the K-major core-matrix layout the MMA reads
//                (8 rows x 16 bytes per core matrix, no swizzle), in a global
//                workspace. HBM-bound: 4 bytes read, 8 written per value.
//   k_tc_update  one CTA per SM, persistent over the step's tiles, each 128
//                rows x 256 columns (A one row block, B two):
//     warp 8     copies A's operand tile and B's two into a ring of kOp
//                shared-memory stages (cp.async.bulk, mbarrier transaction
//                counts), B's two hi parts adjacent (256 rows) and then its
//                two lo parts;
//     warp 9     MMA issuer (one thread) and tensor-memory owner: 3 MMAs
//                (M = 128, N = 256, K = 8) per 8-wide K step into one of two
//                256-column FP32 accumulators;
//     warps 0-7  drain + epilogue: warp w reads lanes 32 (w % 4) .. + 31
//                (tile rows) and columns 128 (w / 4) .. + 127 with
//                tcgen05.ld, adds them into the tile's running sums in its
//                registers with round-to-nearest, and stores the finished
//                tile.
// Splitting in the tile kernel itself would read every raw value from and
// write its two parts to shared memory once per tile that uses it, and
// shared-memory bandwidth (the bulk copies' writes and the MMAs' operand
// reads) is what bounds the tile kernel; split once, an operand is only
// copied in and read by the MMAs, and N = 256 reads A once per 256 output
// columns instead of 128.
// Every wait is bounded; a wait that runs out sets DevStatus::abort, every
// role leaves its loop, copies and MMAs in flight are waited for (bounded)
// and the tensor memory is released before the CTA exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.hpp"

namespace kkt {
namespace tcu {

constexpr int KC = 16;                        // K per chunk (one operand tile)
constexpr uint32_t OPT = 128 * KC * 4;        // bytes of one split part (hi or lo) of an operand tile (8 KB)
constexpr uint32_t TILE = 2 * OPT;            // bytes of an operand tile: hi, then lo
static_assert(TILE == kTcTileFloats * 4, "operand tile size");
// A stage holds one K chunk of a 128 x 256 output tile: A's operand tile,
// then B's hi parts of its two 128-row blocks (256 rows, contiguous in the
// core-matrix layout), then their lo parts.
constexpr uint32_t STAGE = TILE + 2 * TILE;   // 48 KB
constexpr int kOp = 4;                        // ring depth
constexpr int kGroup = 4;                     // K chunks accumulated in tensor memory per drain (64 K)
constexpr uint32_t LBO = 128;                 // bytes between core matrices along K
constexpr uint32_t SBO = (KC / 4) * 128;      // bytes between 8-row groups
constexpr int kThreads = 320;
constexpr uint32_t kSmem = kOp * STAGE + 1024;   // + barriers, slack

// barrier indices
constexpr int B_OP_FULL = 0, B_OP_EMPTY = kOp, B_ACC_FULL = 2 * kOp, B_ACC_EMPTY = B_ACC_FULL + 2,
              B_DONE = B_ACC_EMPTY + 2, kBars = B_DONE + 1;
static_assert(kBars * 8 <= 1024, "barriers fit the reserved shared memory");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool bar_test(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity. Gives up when the CTA's
// abort flag is set or after kSpinCycles (then it raises the flag and the
// device status's abort word).
__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t parity, volatile int* abrt, DevStatus* st) {
  if (bar_test(b, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (bar_test(b, parity)) return true;
    if (*abrt) return false;
    if (clock64() - t0 > kSpinCycles) {
      *abrt = 1;
      atomicExch(&st->abort, 1);
      return false;
    }
  }
}
// Bounded wait that ignores the abort flag (used after an abort, to let
// copies and MMAs already issued land before the CTA releases its memory).
__device__ __forceinline__ void bar_drain(unsigned long long* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!bar_test(b, parity) && clock64() - t0 < kSpinCycles) {
  }
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One panel row's KC values of a K chunk (column-major panel: consecutive
// lanes read consecutive rows, so each of the KC loads is one coalesced
// 128-byte line per warp); the nv valid columns, zeros beyond.
__device__ __forceinline__ void ld_row(float (&v)[KC], const float* p, int64_t ld, int nv) {
#pragma unroll
  for (int k = 0; k < KC; k++) v[k] = k < nv ? __ldg(p + k * ld) : 0.f;
}

__device__ __forceinline__ int64_t i64_of(int lo, int hi) { return (int64_t)(uint32_t)lo | ((int64_t)hi << 32); }

// bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completion counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(b))
               : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

// split one row's KC values into TF32 hi/lo parts and store them at row i of
// the hi and lo operand tiles (K-major core-matrix layout)
__device__ __forceinline__ void split_store(const float (&xv)[KC], unsigned char* hi, unsigned char* lo, int i);

// shared-memory matrix descriptor: K-major, no swizzle, core matrices of 8
// rows x 16 bytes, LBO between core matrices along K, SBO between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;                     // descriptor version of this architecture
  return d;
}
__device__ __forceinline__ uint32_t koff(int i, int k) {
  return (uint32_t)((i >> 3) * SBO + (k >> 2) * LBO + (i & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ void split_store(const float (&xv)[KC], unsigned char* hi, unsigned char* lo, int i) {
#pragma unroll
  for (int q = 0; q < KC / 4; q++) {
    float4 h, l;
    float* hp = &h.x;
    float* lp = &l.x;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const float x = xv[4 * q + r];
      const float xh = tf32_rna(x);
      hp[r] = xh;
      lp[r] = tf32_rna(x - xh);
    }
    const uint32_t off = koff(i, 4 * q);
    *(float4*)(hi + off) = h;
    *(float4*)(lo + off) = l;
  }
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// 32 consecutive tensor-memory columns of this warp's 32 lanes (one
// register per column per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t (&r)[32], uint32_t ta) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
}
__device__ __forceinline__ void mma_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
               : "memory");
}

}  // namespace tcu

// Split item (kTcItem ints = four int4): (ld, rows of the front, first row
// of the row block, K begin), (K end, first chunk, end chunk, 0), (panel
// offset lo, hi, first operand tile lo, hi). One CTA of 128 threads per item;
// thread i splits row i of the block, chunk by chunk, into operand tiles
// first tile + 0, 1, ... (rows past the front and columns past K end are
// zeros).
__global__ void __launch_bounds__(128) k_tc_split(const int4* __restrict__ items, FacArgs<float> a) {
  using namespace tcu;
  batch_view(a);
  const int4* q = items + (kTcItem / 4) * (int64_t)blockIdx.x;
  const int4 q0 = q[0], q1 = q[1], q2 = q[2];
  const int i = threadIdx.x;
  const int64_t ld = q0.x;
  const int nr = q0.y, row = q0.z + i, klo = q0.w, khi = q1.x, c0 = q1.y, c1 = q1.z;
  const float* P = a.L + i64_of(q2.x, q2.y) + row;
  unsigned char* dst = (unsigned char*)(a.W + i64_of(q2.z, q2.w) * kTcTileFloats);
  for (int c = c0; c < c1; c++) {
    const int k0 = klo + c * KC;
    const int nv = row < nr ? min(KC, khi - k0) : 0;
    float v[KC];
    ld_row(v, nv > 0 ? P + (int64_t)k0 * ld : P, ld, nv);
    unsigned char* o = dst + (size_t)(c - c0) * TILE;
    split_store(v, o, o + OPT, i);
  }
}

// Tile item (kTcItem ints): (A operand tile lo, hi, B operand tile lo, hi),
// (chunks, mode, panel row of A, panel row of B), (ld, rows, width, B has a
// second row block), (output offset lo, hi, 0, 0). The tile is 128 rows
// (A's block) x 256 columns (B's block and the next one, whose operand tiles
// follow B's after `chunks` tiles); chunk c of A is operand tile A + c. The
// output is U_s (mode 0, offset uoff[s]) or the panel (mode 1, poff[s]);
// columns past the front (a missing second block) are computed from whatever
// the stage holds there and never stored.
__global__ void __launch_bounds__(tcu::kThreads, 1)
    k_tc_update(const int4* __restrict__ items, int64_t nitems, FacArgs<float> a) {
  using namespace tcu;
  batch_view(a);                                         // system blockIdx.y of a batched launch
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* opb = sm;                               // [kOp][STAGE]
  unsigned long long* bar = (unsigned long long*)(opb + kOp * STAGE);
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abrt = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < kOp; q++) {
      bar_init(&bar[B_OP_FULL + q], 1);
      bar_init(&bar[B_OP_EMPTY + q], 1);
    }
    for (int q = 0; q < 2; q++) {
      bar_init(&bar[B_ACC_FULL + q], 1);
      bar_init(&bar[B_ACC_EMPTY + q], 8);
    }
    bar_init(&bar[B_DONE], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    // two 256-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == 8) {
    // ------------------------------------------------ operand copies
    if (lane == 0) {
      uint32_t rc = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const int4* q = items + (kTcItem / 4) * t;
        const int4 q0 = q[0], q1 = q[1], q2 = q[2];
        const int64_t ta = i64_of(q0.x, q0.y), tb = i64_of(q0.z, q0.w);
        const int nk = q1.x;
        const bool two = q2.w != 0;
        for (int c = 0; c < nk; c++) {
          const uint32_t slot = rc % kOp, round = rc / kOp;
          if (!(ok = bar_wait(&bar[B_OP_EMPTY + slot], (round & 1) ^ 1, abrt, a.st))) break;
          unsigned char* dst = opb + slot * STAGE;
          const float* pa = a.W + (ta + c) * kTcTileFloats;
          const float* pb = a.W + (tb + c) * kTcTileFloats;
          const float* pb2 = a.W + (tb + nk + c) * kTcTileFloats;
          bar_expect_tx(&bar[B_OP_FULL + slot], two ? STAGE : STAGE - TILE);
          bulk_load(dst, pa, TILE, &bar[B_OP_FULL + slot]);                       // A hi, lo
          bulk_load(dst + TILE, pb, OPT, &bar[B_OP_FULL + slot]);                 // B rows 0..127 hi
          bulk_load(dst + 2 * TILE, pb + OPT / 4, OPT, &bar[B_OP_FULL + slot]);   // B rows 0..127 lo
          if (two) {
            bulk_load(dst + TILE + OPT, pb2, OPT, &bar[B_OP_FULL + slot]);        // B rows 128..255 hi
            bulk_load(dst + 2 * TILE + OPT, pb2 + OPT / 4, OPT, &bar[B_OP_FULL + slot]);   // lo
          }
          rc++;
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits
        for (uint32_t q = rc > (uint32_t)kOp ? rc - kOp : 0; q < rc; q++)
          bar_drain(&bar[B_OP_FULL + q % kOp], (q / kOp) & 1);
      }
    }
  } else if (warp == 9) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      // D = F32, A = B = TF32, both K-major, N = 256, M = 128
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (32u << 17) | (8u << 24);
      uint32_t oc = 0, gc = 0;
      bool ok = true, issued = false;
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const int nk = items[(kTcItem / 4) * t + 1].x;
        for (int g0 = 0; g0 < nk && ok; g0 += kGroup) {
          const uint32_t b = gc & 1;
          if (!(ok = bar_wait(&bar[B_ACC_EMPTY + b], ((gc >> 1) & 1) ^ 1, abrt, a.st))) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + b * 256;
          const int g1 = min(nk, g0 + kGroup);
          for (int c = g0; c < g1; c++) {
            const uint32_t os = oc % kOp, orr = oc / kOp;
            if (!(ok = bar_wait(&bar[B_OP_FULL + os], orr & 1, abrt, a.st))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = saddr(opb + os * STAGE);
            const uint32_t ah = base, al = base + OPT, bh = base + TILE, bl = base + 2 * TILE;
#pragma unroll
            for (int kk = 0; kk < KC / 8; kk++) {
              const uint32_t ko = kk * 2 * LBO;
              mma_tf32(d, sdesc(ah + ko), sdesc(bh + ko), idesc, (c > g0 || kk > 0) ? 1u : 0u);
              mma_tf32(d, sdesc(ah + ko), sdesc(bl + ko), idesc, 1u);
              mma_tf32(d, sdesc(al + ko), sdesc(bh + ko), idesc, 1u);
            }
            issued = true;
            mma_commit(&bar[B_OP_EMPTY + os]);
            oc++;
          }
          if (!ok) break;
          mma_commit(&bar[B_ACC_FULL + b]);
          gc++;
        }
      }
      if (issued) {
        // every MMA issued has completed before the tensor memory is released
        mma_commit(&bar[B_DONE]);
        bar_drain(&bar[B_DONE], 0);
      }
    }
  } else {
    // ------------------------------------------------ drain + epilogue (warps 0-7)
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile rows) and
    // columns 128 (w / 4) .. + 127 of the 256; the tile's running sums stay
    // in its registers, one per column, added with round-to-nearest
    const int quad = warp & 3, half = warp >> 2;
    const int i = 32 * quad + lane;          // tile row = tensor-memory lane
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    uint32_t gc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
      const int4* q = items + (kTcItem / 4) * t;
      const int4 q1 = q[1], q2 = q[2], q3 = q[3];
      const int nk = q1.x, mode = q1.y, ra = q1.z, cb = q1.w + 128 * half;
      const int ld = q2.x, nr = q2.y, w = q2.z;
      const int64_t out = i64_of(q3.x, q3.y);
      if (mode != 0) {
        // in-panel tile: pull this row's 128 outputs into L2 while the MMAs
        // run, so the read-modify-write below waits on L2, not on HBM
        const int row = ra + i;
        const float* P = a.L + out + row;
        if (row < nr)
          for (int j = 0; j < 128 && cb + j < w; j++)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(P + (int64_t)(cb + j) * ld));
      }
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; j++) acc[j] = 0.f;
      for (int g0 = 0; g0 < nk; g0 += kGroup) {
        const uint32_t b = gc & 1;
        bool got = true;
        if (lane == 0) got = bar_wait(&bar[B_ACC_FULL + b], (gc >> 1) & 1, abrt, a.st);
        if (!(ok = __shfl_sync(0xffffffffu, got, 0))) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ta = tmem + lane_off + b * 256 + half * 128;
#pragma unroll
        for (int c4 = 0; c4 < 4; c4++) {
          uint32_t r[32];
          tmem_ld32(r, ta + (uint32_t)(c4 * 32));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 32; j++) acc[c4 * 32 + j] += __uint_as_float(r[j]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) bar_arrive(&bar[B_ACC_EMPTY + b]);
        gc++;
      }
      if (!ok) break;
      // store the finished tile
      if (mode == 0) {
        const int rbk = nr - w;
        const int gi = ra - w + i, gj0 = cb - w;
        float* U = a.U + out;
        if (gi < rbk) {
#pragma unroll
          for (int j = 0; j < 128; j++) {
            const int gj = gj0 + j;
            if (gj < rbk && gi >= gj) U[(int64_t)gi + (int64_t)gj * rbk] = -acc[j];
          }
        }
      } else {
        // read-modify-write in batches of 32 independent loads
        const int row = ra + i;
        float* __restrict__ P = a.L + out + row;
        if (row < nr) {
#pragma unroll
          for (int c4 = 0; c4 < 4; c4++) {
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const int col = cb + c4 * 32 + j;
              v[j] = (col < w && row >= col) ? P[(int64_t)col * ld] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const int col = cb + c4 * 32 + j;
              if (col < w && row >= col) P[(int64_t)col * ld] = v[j] - acc[c4 * 32 + j];
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 9) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

cudaError_t launch_tc_split(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb) {
  if (cnt <= 0) return cudaSuccess;
  k_tc_split<<<dim3((unsigned)cnt, (unsigned)nb), 128, 0, st>>>(items, a);
  return cudaGetLastError();
}

cudaError_t launch_tc_update(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcu::kSmem);
    if (e) return e;
    attr = true;
  }
  // one CTA per SM in all: nb systems share the SMs (each system's tiles go
  // round-robin over its gridDim.x CTAs)
  const int64_t per = std::max<int64_t>(1, kTcGrid / nb);
  const int64_t grid = cnt < per ? cnt : per;
  k_tc_update<<<dim3((unsigned)grid, (unsigned)nb), tcu::kThreads, tcu::kSmem, st>>>(items, cnt, a);
  return cudaGetLastError();
}

}  // namespace kkt
