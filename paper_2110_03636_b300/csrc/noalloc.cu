// Residual of the 2x2 KKT system for callers that cannot allocate device
// memory (see kkt_residual_noalloc in kkt.h).
//
// Some callers cannot call cudaMalloc: code running inside a process whose
// device memory is owned by another allocator (a framework's caching pool,
// an embedding application with a fixed budget), code called from a region
// where allocation is forbidden, or code that must not synchronize the
// device (cudaMalloc/cudaFree can). This entry point needs no allocation:
// its scratch is the fixed array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "kkt.h"

namespace {

constexpr int64_t kNoAllocMaxRows = KKT_NOALLOC_MAX_ROWS;  // n + m limit
constexpr int kNaBlocks = 296;                              // 2 x 148 SMs
constexpr int kNaThreads = 256;

// [0, n+m): absolute row sums of K_delta (cleared by every call);
// [kNoAllocMaxRows, + 4 * kNaBlocks): per-block partial norms.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxRows + 4 * kNaBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device. The
// host-side name is only a stand-in for the symbol, so the address is
// looked up with cudaGetSymbolAddress: on the first call on each device,
// and again on every call whose stream is not capturing (a device reset
// between calls reloads the module, possibly at another address). A call
// made during stream capture uses the address cached by an earlier call.
cudaError_t scratch_on_current_device(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void k_na_init(int64_t n, int64_t m, double delta, const double* rx, const double* ry, const double* dx,
                          double* res_x, double* res_y, double* rowsum) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      res_x[i] = rx[i] - delta * dx[i];
      rowsum[i] = fabs(delta);
    } else {
      res_y[i - n] = ry[i - n];
      rowsum[i] = 0.0;
    }
  }
}

// H~ given by its lower triangle: entry (i, j), i >= j, acts on rows i and j.
__global__ void k_na_h(int64_t n, const int64_t* Hp, const int32_t* Hi, const double* Hv, const double* dx,
                       double* res_x, double* rowsum) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double own = 0.0, own_abs = 0.0;
    const double xj = dx[j];
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
      const int32_t i = Hi[q];
      const double h = Hv[q];
      if (i == j) {
        own += h * xj;
        own_abs += fabs(h);
      } else {
        atomicAdd(&res_x[i], -h * xj);
        atomicAdd(&rowsum[i], fabs(h));
        own += h * dx[i];
        own_abs += fabs(h);
      }
    }
    atomicAdd(&res_x[j], -own);
    atomicAdd(&rowsum[j], own_abs);
  }
}

// J rows: res_y = r_y - J dx, res_x -= J^T dy
__global__ void k_na_j(int64_t n, int64_t m, const int64_t* Jp, const int32_t* Ji, const double* Jv, const double* dx,
                       const double* dy, double* res_x, double* res_y, double* rowsum) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, a = 0.0;
    const double yr = dy[r];
    for (int64_t q = Jp[r]; q < Jp[r + 1]; q++) {
      const int32_t c = Ji[q];
      const double v = Jv[q];
      s += v * dx[c];
      a += fabs(v);
      atomicAdd(&res_x[c], -v * yr);
      atomicAdd(&rowsum[c], fabs(v));
    }
    res_y[r] -= s;
    rowsum[n + r] = a;
  }
}

__global__ void __launch_bounds__(kNaThreads) k_na_norms(int64_t n, int64_t m, const double* rx, const double* ry,
                                                         const double* dx, const double* dy, const double* res_x,
                                                         const double* res_y, const double* rowsum, double* part) {
  __shared__ double sh[kNaThreads / 32][4];
  double r2 = 0, b2 = 0, x2 = 0, km = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = i < n ? res_x[i] : res_y[i - n];
    const double b = i < n ? rx[i] : ry[i - n];
    const double x = i < n ? dx[i] : dy[i - n];
    r2 += r * r;
    b2 += b * b;
    x2 += x * x;
    km = fmax(km, rowsum[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    km = fmax(km, __shfl_xor_sync(0xffffffffu, km, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sh[w][0] = r2; sh[w][1] = b2; sh[w][2] = x2; sh[w][3] = km; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int k = 0; k < kNaThreads / 32; k++) {
      t[0] += sh[k][0]; t[1] += sh[k][1]; t[2] += sh[k][2]; t[3] = fmax(t[3], sh[k][3]);
    }
    for (int k = 0; k < 4; k++) part[blockIdx.x * 4 + k] = t[k];
  }
}

__global__ void k_na_final(const double* part, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[4] = {0, 0, 0, 0};
  for (int b = 0; b < kNaBlocks; b++) {
    t[0] += part[b * 4]; t[1] += part[b * 4 + 1]; t[2] += part[b * 4 + 2];
    t[3] = fmax(t[3], part[b * 4 + 3]);
  }
  const double res = sqrt(t[0]), bn = sqrt(t[1]), xn = sqrt(t[2]);
  out[0] = bn > 0 ? res / bn : res;
  out[1] = res / (t[3] * xn + bn);
  out[2] = res;
  out[3] = t[3];
}

}  // namespace

extern "C" kkt_status kkt_residual_noalloc(int64_t n, int64_t m, const int64_t* H_colptr, const int32_t* H_rowidx,
                                           const double* H_vals, const int64_t* J_rowptr, const int32_t* J_colidx,
                                           const double* J_vals, double delta, const double* r_x, const double* r_y,
                                           const double* dx, const double* dy, double* res_x, double* res_y,
                                           double* norms, void* stream) {
  if (n < 1 || m < 0 || !H_colptr || !H_rowidx || !H_vals || !r_x || !dx || !res_x || !norms) return KKT_ERR_INVALID;
  if (m > 0 && (!J_rowptr || !J_colidx || !J_vals || !r_y || !dy || !res_y)) return KKT_ERR_INVALID;
  if (n + m > kNoAllocMaxRows) return KKT_ERR_TOO_LARGE;
  if (!std::isfinite(delta)) return KKT_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(st, &scratch);
  if (e != cudaSuccess) { cudaGetLastError(); return KKT_ERR_CUDA; }
  double* rowsum = scratch;
  double* part = scratch + kNoAllocMaxRows;
  k_na_init<<<kNaBlocks, kNaThreads, 0, st>>>(n, m, delta, r_x, r_y, dx, res_x, res_y, rowsum);
  k_na_h<<<kNaBlocks, kNaThreads, 0, st>>>(n, H_colptr, H_rowidx, H_vals, dx, res_x, rowsum);
  if (m > 0) k_na_j<<<kNaBlocks, kNaThreads, 0, st>>>(n, m, J_rowptr, J_colidx, J_vals, dx, dy, res_x, res_y, rowsum);
  k_na_norms<<<kNaBlocks, kNaThreads, 0, st>>>(n, m, r_x, r_y, dx, dy, res_x, res_y, rowsum, part);
  k_na_final<<<1, 32, 0, st>>>(part, norms);
  e = cudaGetLastError();
  return e == cudaSuccess ? KKT_OK : KKT_ERR_CUDA;
}
