// Shared device helpers for the KKT kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace kkt {

// Device status block written by kernels, read by the host after a call.
struct DevStatus {
  int32_t fail_col;        // first column with a pivot <= 0 or non-finite (INT32_MAX = none)
  int32_t abort;           // a bounded wait gave up (1) or a bounds check failed (2)
  int32_t cg_iters;        // products with S in the last solve pass
  int32_t cg_status;       // 0 converged, 3 breakdown after restart, 4 max iterations
  int32_t breakdown;       // a small quadratic form was met (delta_2 restart used)
  int32_t pad[3];
  double rr, be, res_norm, b_norm, x_norm, k_norm_inf;
};

// Spin limit for every wait on another CTA's flag: ~4e9 cycles (about two
// seconds at 2 GHz). A wait that runs out sets DevStatus::abort and returns.
constexpr long long kSpinCycles = 4000000000LL;

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait (thread 0 of the CTA) until *flag >= target or the abort word is set.
// Returns false when the wait gave up.
__device__ __forceinline__ bool wait_geq(const int* flag, int target, DevStatus* st,
                                         long long limit = kSpinCycles) {
  if (ld_acquire(flag) >= target) return true;
  const long long t0 = clock64();
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_acquire(&st->abort)) return false;
    if (clock64() - t0 > limit) {
      atomicExch(&st->abort, 1);
      return false;
    }
    __nanosleep(64);
  }
}

// Wait (all 32 lanes of one warp) until flags[tg[q]] >= target for every q
// in [q0, q1): the lanes poll different flags at once, so a list of k
// satisfied flags costs one round trip per 32 instead of k. Flags only grow
// within a sweep, so a lane moves on as soon as its current flag is met.
// Returns false (in every lane) when the wait gave up or the abort word is set.
__device__ __forceinline__ bool warp_wait_all(const int* flags, const int32_t* tg, int64_t q0, int64_t q1,
                                              int target, DevStatus* st, long long limit = kSpinCycles) {
  bool ok = true;
  const long long t0 = clock64();
  int spins = 0;
  for (int64_t q = q0 + (threadIdx.x & 31); q < q1;) {
    if (ld_acquire(&flags[__ldg(&tg[q])]) >= target) {
      q += 32;
      continue;
    }
    if ((++spins & 15) == 0) {
      if (ld_acquire(&st->abort)) { ok = false; break; }
      if (clock64() - t0 > limit) {
        atomicExch(&st->abort, 1);
        ok = false;
        break;
      }
    }
  }
  return __all_sync(0xffffffffu, ok);
}

// Raises kernel k's dynamic shared-memory limit to at least `bytes` and never
// lowers it: handles with different plans launch the same kernels with
// different sizes (also from several threads, and from graphs captured
// earlier), and every launch needs the limit at or above its own size.
template <typename K>
inline cudaError_t raise_smem_limit(K k, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)k);
  if (e) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace kkt
