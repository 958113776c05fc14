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
// only ever holds kGroup K chunks: the epilogue warps drain it into FP32
// registers after each group and sum the groups with round-to-nearest adds,
// so the accumulation error grows with the number of groups the way an FMA
// loop's does, not with K.
//
// Pipeline (one CTA per SM, persistent over the launch's tiles):
//   warp 8      TMA producer: 2-D boxes of 132 rows x 32 columns of the
//               panel (the row start rounded down to a multiple of 4, as the
//               16-byte rule for the innermost TMA coordinate requires) into
//               a ring of kRaw stages;
//   warps 4-7   converters: raw FP32 -> hi/lo TF32 tiles in the K-major
//               core-matrix layout the MMA reads (8 rows x 16 bytes per core
//               matrix, no swizzle), ring of kOp stages;
//   warp 9      MMA issuer (one thread) and tensor-memory owner: 3 MMAs per
//               8-wide K step into one of two 128 x 128 FP32 accumulators;
//   warps 0-3   drain + epilogue: tcgen05.ld of the accumulator (warp w
//               reads lanes 32w..32w+31 = tile rows), FP32 sums in
//               registers, stores of the finished tile.
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

constexpr int KC = 32;                        // K per chunk (one TMA box)
constexpr int BOXR = kTcBoxRows;              // rows per TMA box: 128 + up to 3 of start alignment
constexpr uint32_t RAW = BOXR * KC * 4;       // bytes of one raw box (16896)
constexpr uint32_t OPT = 128 * KC * 4;        // bytes of one split operand tile (16384)
constexpr int kRaw = 2, kOp = 2;              // ring depths
constexpr int kGroup = 2;                     // K chunks accumulated in tensor memory per drain
constexpr uint32_t LBO = 128;                 // bytes between core matrices along K
constexpr uint32_t SBO = (KC / 4) * 128;      // bytes between 8-row groups
constexpr int kThreads = 320;
constexpr uint32_t kSmem = kRaw * 2 * RAW + kOp * 4 * OPT + 1024;   // + barriers, slack

// barrier indices
constexpr int B_RAW_FULL = 0, B_RAW_EMPTY = kRaw, B_OP_FULL = 2 * kRaw, B_OP_EMPTY = 2 * kRaw + kOp,
              B_ACC_FULL = 2 * kRaw + 2 * kOp, B_ACC_EMPTY = B_ACC_FULL + 2, B_DONE = B_ACC_EMPTY + 2,
              kBars = B_DONE + 1;
static_assert(kBars * 8 <= 1024, "barriers fit the reserved shared memory");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
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

// 3-D tiled TMA load: (x = panel row, y = panel column, z = system of a batch)
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          saddr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(saddr(b))
      : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

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
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
               : "memory");
}

}  // namespace tcu

// Item of a tensor-core update launch (two int4): (s, row of A, row of B,
// tensor map), (first K column, end K column, mode, 0). Rows are panel rows
// of front s; A = B for a diagonal tile.
__global__ void __launch_bounds__(tcu::kThreads, 1)
    k_tc_update(const int4* __restrict__ items, int64_t nitems, const uint8_t* __restrict__ maps, FacArgs<float> a) {
  using namespace tcu;
  batch_view(a);                                         // system blockIdx.y of a batched launch
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* raw = sm;                               // [kRaw][A, B][RAW]
  unsigned char* opb = sm + kRaw * 2 * RAW;              // [kOp][A hi, A lo, B hi, B lo][OPT]
  unsigned long long* bar = (unsigned long long*)(opb + kOp * 4 * OPT);
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abrt = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < kRaw; q++) {
      bar_init(&bar[B_RAW_FULL + q], 1);
      bar_init(&bar[B_RAW_EMPTY + q], 4);
    }
    for (int q = 0; q < kOp; q++) {
      bar_init(&bar[B_OP_FULL + q], 4);
      bar_init(&bar[B_OP_EMPTY + q], 1);
    }
    for (int q = 0; q < 2; q++) {
      bar_init(&bar[B_ACC_FULL + q], 1);
      bar_init(&bar[B_ACC_EMPTY + q], 4);
    }
    bar_init(&bar[B_DONE], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    // two 128-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == 8) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t rc = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const int4 i0 = items[2 * t], i1 = items[2 * t + 1];
        const void* mp = maps + (size_t)i0.w * 128;
        const bool diag = i0.y == i0.z;
        const int xa = i0.y & ~3, xb = i0.z & ~3;
        const int nk = (i1.y - i1.x + KC - 1) / KC;
        for (int c = 0; c < nk; c++) {
          const uint32_t slot = rc % kRaw, round = rc / kRaw;
          if (!(ok = bar_wait(&bar[B_RAW_EMPTY + slot], (round & 1) ^ 1, abrt, a.st))) break;
          unsigned char* dst = raw + slot * 2 * RAW;
          bar_expect_tx(&bar[B_RAW_FULL + slot], diag ? RAW : 2 * RAW);
          tma_load_3d(dst, mp, xa, i1.x + c * KC, (int)blockIdx.y, &bar[B_RAW_FULL + slot]);
          if (!diag) tma_load_3d(dst + RAW, mp, xb, i1.x + c * KC, (int)blockIdx.y, &bar[B_RAW_FULL + slot]);
          rc++;
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits
        for (uint32_t q = rc > (uint32_t)kRaw ? rc - kRaw : 0; q < rc; q++)
          bar_drain(&bar[B_RAW_FULL + q % kRaw], (q / kRaw) & 1);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------ converters
    const int i = tid - 128;                 // tile row
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
      const int4 i0 = items[2 * t], i1 = items[2 * t + 1];
      const bool diag = i0.y == i0.z;
      const int sa = i0.y & 3, sb = i0.z & 3;
      const int nk = (i1.y - i1.x + KC - 1) / KC;
      for (int c = 0; c < nk; c++) {
        const uint32_t rs = rc % kRaw, rr = rc / kRaw, os = rc % kOp, orr = rc / kOp;
        bool w = true;
        if (lane == 0)
          w = bar_wait(&bar[B_RAW_FULL + rs], rr & 1, abrt, a.st) &&
              bar_wait(&bar[B_OP_EMPTY + os], (orr & 1) ^ 1, abrt, a.st);
        if (!(ok = __shfl_sync(0xffffffffu, w, 0))) break;
        const float* ra = (const float*)(raw + rs * 2 * RAW);
        unsigned char* o = opb + os * 4 * OPT;
#pragma unroll
        for (int half = 0; half < 2; half++) {
          if (half == 1 && diag) break;
          const float* src = ra + (half ? BOXR * KC : 0) + (half ? sb : sa) + i;
          unsigned char* hi = o + (half ? 2 : 0) * OPT;
          unsigned char* lo = hi + OPT;
          // all 32 loads of the row first: the stores below go to other
          // shared-memory tiles, but the compiler cannot tell, so loads
          // interleaved with them would each wait out their latency
          float xv[KC];
#pragma unroll
          for (int k = 0; k < KC; k++) xv[k] = src[k * BOXR];
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
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          bar_arrive(&bar[B_RAW_EMPTY + rs]);
          bar_arrive(&bar[B_OP_FULL + os]);
        }
        rc++;
      }
    }
  } else if (warp == 9) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      // D = F32, A = B = TF32, both K-major, N = 128, M = 128
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (16u << 17) | (8u << 24);
      uint32_t oc = 0, gc = 0;
      bool ok = true, issued = false;
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const int4 i0 = items[2 * t], i1 = items[2 * t + 1];
        const bool diag = i0.y == i0.z;
        const int nk = (i1.y - i1.x + KC - 1) / KC;
        for (int g0 = 0; g0 < nk && ok; g0 += kGroup) {
          const uint32_t b = gc & 1;
          if (!(ok = bar_wait(&bar[B_ACC_EMPTY + b], ((gc >> 1) & 1) ^ 1, abrt, a.st))) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + b * 128;
          const int g1 = min(nk, g0 + kGroup);
          for (int c = g0; c < g1; c++) {
            const uint32_t os = oc % kOp, orr = oc / kOp;
            if (!(ok = bar_wait(&bar[B_OP_FULL + os], orr & 1, abrt, a.st))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = saddr(opb + os * 4 * OPT);
            const uint32_t ah = base, al = base + OPT, bh = diag ? ah : base + 2 * OPT, bl = diag ? al : base + 3 * OPT;
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
    // ------------------------------------------------ drain + epilogue (warps 0-3)
    const int i = 32 * warp + lane;          // tile row = tensor-memory lane
    uint32_t gc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
      const int4 i0 = items[2 * t], i1 = items[2 * t + 1];
      const int nk = (i1.y - i1.x + KC - 1) / KC;
      if (i1.z != 0) {
        // in-panel tile: pull this row's 128 outputs into L2 while the MMAs
        // run, so the read-modify-write below waits on L2, not on HBM
        const int s = i0.x;
        const int ld = a.sld[s], nr = a.snr[s], w = a.sw[s];
        const int row = i0.y + i;
        const float* P = a.L + a.poff[s] + row;
        if (row < nr)
          for (int j = 0; j < 128 && i0.z + j < w; j++)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(P + (int64_t)(i0.z + j) * ld));
      }
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; j++) acc[j] = 0.f;
      for (int g0 = 0; g0 < nk; g0 += kGroup) {
        const uint32_t b = gc & 1;
        bool w = true;
        if (lane == 0) w = bar_wait(&bar[B_ACC_FULL + b], (gc >> 1) & 1, abrt, a.st);
        if (!(ok = __shfl_sync(0xffffffffu, w, 0))) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + b * 128;
#pragma unroll
        for (int c4 = 0; c4 < 4; c4++) {
          uint32_t r[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
              : "r"(ta + (uint32_t)(c4 * 32)));
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
      const int s = i0.x;
      const int w = a.sw[s], nr = a.snr[s];
      if (i1.z == 0) {
        const int rb = nr - w;
        const int gi = i0.y - w + i, gj0 = i0.z - w;
        float* U = a.U + a.uoff[s];
        if (gi < rb) {
#pragma unroll
          for (int j = 0; j < 128; j++) {
            const int gj = gj0 + j;
            if (gj < rb && gi >= gj) U[(int64_t)gi + (int64_t)gj * rb] = -acc[j];
          }
        }
      } else {
        // read-modify-write in batches of 32 independent loads
        const int ld = a.sld[s];
        const int row = i0.y + i, col0 = i0.z;
        float* __restrict__ P = a.L + a.poff[s] + row;
        if (row < nr) {
#pragma unroll
          for (int c4 = 0; c4 < 4; c4++) {
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const int col = col0 + c4 * 32 + j;
              v[j] = (col < w && row >= col) ? P[(int64_t)col * ld] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const int col = col0 + c4 * 32 + j;
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
  if (warp == 9) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

cudaError_t launch_tc_update(const int4* items, int64_t cnt, const uint8_t* maps, const FacArgs<float>& a,
                             cudaStream_t st, int nb) {
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
  k_tc_update<<<dim3((unsigned)grid, (unsigned)nb), tcu::kThreads, tcu::kSmem, st>>>(items, cnt, maps, a);
  return cudaGetLastError();
}

}  // namespace kkt
