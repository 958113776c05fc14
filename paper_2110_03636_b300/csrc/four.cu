// The 4x4 form of the KKT system (Sec. 3, eq. linsys4x4) on top of the 2x2
// solver: H~ = H + D_x + J_d^T D_s J_d is formed on the device for every
// factorization, the right-hand side r_x = r~_x + J_d^T (D_s r_yd + r_s)
// for every solve, and ds = J_d dx - r_yd, dy_d = D_s ds - r_s are
// recovered after it (eq. linsys2x2 and the elimination that precedes it).
// The wrapper uses the 2x2 solver only through its C entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "kkt.h"

namespace {

struct Arena {
  std::vector<void*> ptrs;
  bool failed = false;
  template <typename X>
  X* alloc(size_t count) {
    if (failed) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(X) * (count ? count : 1)) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return (X*)p;
  }
  template <typename X>
  X* upload(const std::vector<X>& v) {
    X* d = alloc<X>(v.size());
    if (d && !v.empty() && cudaMemcpy(d, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
    }
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// Every stored entry (i >= j) of H~ sums: H's entry (if present), D_x[j] on
// the diagonal, and D_s[r] J_d[r,i] J_d[r,j] over the rows r of J_d that hold
// both columns, in ascending r.
__global__ void k_form_htilde(int64_t nnz, const int64_t* __restrict__ hpos, const int32_t* __restrict__ dcol,
                              const int64_t* __restrict__ pr_ptr, const int32_t* __restrict__ pr_row,
                              const int64_t* __restrict__ pr_a, const int64_t* __restrict__ pr_b,
                              const double* __restrict__ H, const double* __restrict__ Dx,
                              const double* __restrict__ Jd, const double* __restrict__ Ds, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    double v = hpos[k] >= 0 ? H[hpos[k]] : 0.0;
    if (dcol[k] >= 0) v += Dx[dcol[k]];
    for (int64_t q = pr_ptr[k]; q < pr_ptr[k + 1]; q++) v += Ds[pr_row[q]] * (Jd[pr_a[q]] * Jd[pr_b[q]]);
    out[k] = v;
  }
}

// r_x[i] = r~_x[i] + sum_r J_d[r,i] (D_s[r] r_yd[r] + r_s[r]), by column of J_d
__global__ void k_rhs_4x4(int64_t n, const int64_t* __restrict__ jt_ptr, const int32_t* __restrict__ jt_row,
                          const int64_t* __restrict__ jt_pos, const double* __restrict__ Jd,
                          const double* __restrict__ Ds, const double* __restrict__ rxt,
                          const double* __restrict__ rs, const double* __restrict__ ryd, double* __restrict__ rx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = rxt[i];
    for (int64_t q = jt_ptr[i]; q < jt_ptr[i + 1]; q++) {
      const int r = jt_row[q];
      v += Jd[jt_pos[q]] * (Ds[r] * ryd[r] + rs[r]);
    }
    rx[i] = v;
  }
}

// ds = J_d dx - r_yd, then dy_d = D_s ds - r_s, by row of J_d
__global__ void k_recover_4x4(int64_t md, const int64_t* __restrict__ jp, const int32_t* __restrict__ jc,
                              const double* __restrict__ Jd, const double* __restrict__ Ds,
                              const double* __restrict__ dx, const double* __restrict__ ryd,
                              const double* __restrict__ rs, double* __restrict__ ds, double* __restrict__ dyd) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < md; r += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t q = jp[r]; q < jp[r + 1]; q++) v += Jd[q] * dx[jc[q]];
    v -= ryd[r];
    ds[r] = v;
    dyd[r] = Ds[r] * v - rs[r];
  }
}

unsigned grid_for(int64_t count) {
  const int64_t b = (count + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 16));
}

}  // namespace

struct kkt_handle4_s {
  kkt_handle inner = nullptr;
  int64_t n = 0, m = 0, md = 0, nnzHt = 0, nnzJd = 0;
  int device = 0;
  bool on_device = false;
  // host pattern of H~ (kept for kkt_get_4x4_pattern)
  std::vector<int64_t> ht_ptr;
  std::vector<int32_t> ht_row;
  Arena mem;
  int64_t *hpos = nullptr, *pr_ptr = nullptr, *pr_a = nullptr, *pr_b = nullptr;
  int32_t *dcol = nullptr, *pr_row = nullptr;
  int64_t *jt_ptr = nullptr, *jt_pos = nullptr, *jd_ptr = nullptr;
  int32_t *jt_row = nullptr, *jd_col = nullptr;
  double *ht_vals = nullptr, *Jdv = nullptr, *Ds = nullptr, *rx = nullptr;
};

namespace {

// Host half of kkt_analyse_4x4: validates J_d, forms the lower pattern of
// H~ = pat(H) U pat(J_d^T J_d) U diag and the source lists of its entries.
struct Form4 {
  std::vector<int64_t> ht_ptr, hpos, pr_ptr, pr_a, pr_b, jt_ptr, jt_pos;
  std::vector<int32_t> ht_row, dcol, pr_row, jt_row;
};

int form_pattern(int64_t n, int64_t md, const int64_t* Hp, const int32_t* Hi, const int64_t* Jdp,
                 const int32_t* Jdi, Form4& F) {
  if (Hp[0] != 0) return 1;
  for (int64_t j = 0; j < n; j++) {
    if (Hp[j + 1] < Hp[j]) return 1;
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
      if (Hi[q] < j || Hi[q] >= n || (q > Hp[j] && Hi[q] <= Hi[q - 1])) return 1;
    }
  }
  if (md > 0) {
    if (Jdp[0] != 0) return 1;
    for (int64_t r = 0; r < md; r++) {
      if (Jdp[r + 1] < Jdp[r]) return 1;
      for (int64_t q = Jdp[r]; q < Jdp[r + 1]; q++)
        if (Jdi[q] < 0 || Jdi[q] >= n || (q > Jdp[r] && Jdi[q] <= Jdi[q - 1])) return 1;
    }
  }
  // column lists of H~: H's rows, the diagonal, the J_d pairs
  std::vector<std::vector<int32_t>> col(n);
  for (int64_t j = 0; j < n; j++) {
    col[j].assign(Hi + Hp[j], Hi + Hp[j + 1]);
    col[j].push_back((int32_t)j);
  }
  for (int64_t r = 0; r < md; r++)
    for (int64_t a = Jdp[r]; a < Jdp[r + 1]; a++)
      for (int64_t b = a; b < Jdp[r + 1]; b++) col[Jdi[a]].push_back(Jdi[b]);
  F.ht_ptr.assign(n + 1, 0);
  for (int64_t j = 0; j < n; j++) {
    std::sort(col[j].begin(), col[j].end());
    col[j].erase(std::unique(col[j].begin(), col[j].end()), col[j].end());
    F.ht_ptr[j + 1] = F.ht_ptr[j] + (int64_t)col[j].size();
  }
  const int64_t nnz = F.ht_ptr[n];
  F.ht_row.resize(nnz);
  F.hpos.assign(nnz, -1);
  F.dcol.assign(nnz, -1);
  for (int64_t j = 0; j < n; j++) {
    std::copy(col[j].begin(), col[j].end(), F.ht_row.begin() + F.ht_ptr[j]);
    std::vector<int32_t>().swap(col[j]);
  }
  auto find = [&](int64_t j, int32_t i) {
    const auto b = F.ht_row.begin() + F.ht_ptr[j], e = F.ht_row.begin() + F.ht_ptr[j + 1];
    return (int64_t)(std::lower_bound(b, e, i) - F.ht_row.begin());
  };
  for (int64_t j = 0; j < n; j++) {
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) F.hpos[find(j, Hi[q])] = q;
    F.dcol[find(j, (int32_t)j)] = (int32_t)j;
  }
  // pair sources, grouped by target entry, ascending row r inside a group
  std::vector<int64_t> cnt(nnz + 1, 0), tgt;
  for (int64_t r = 0; r < md; r++)
    for (int64_t a = Jdp[r]; a < Jdp[r + 1]; a++)
      for (int64_t b = a; b < Jdp[r + 1]; b++) {
        const int64_t k = find(Jdi[a], Jdi[b]);
        tgt.push_back(k);
        cnt[k + 1]++;
      }
  for (int64_t k = 0; k < nnz; k++) cnt[k + 1] += cnt[k];
  F.pr_ptr = cnt;
  const int64_t np = cnt[nnz];
  F.pr_row.resize(np);
  F.pr_a.resize(np);
  F.pr_b.resize(np);
  int64_t t = 0;
  for (int64_t r = 0; r < md; r++)
    for (int64_t a = Jdp[r]; a < Jdp[r + 1]; a++)
      for (int64_t b = a; b < Jdp[r + 1]; b++) {
        const int64_t s = cnt[tgt[t++]]++;
        F.pr_row[s] = (int32_t)r;
        F.pr_a[s] = a;
        F.pr_b[s] = b;
      }
  // J_d^T by column, rows ascending
  F.jt_ptr.assign(n + 1, 0);
  const int64_t nnzJd = md > 0 ? Jdp[md] : 0;
  for (int64_t q = 0; q < nnzJd; q++) F.jt_ptr[Jdi[q] + 1]++;
  for (int64_t i = 0; i < n; i++) F.jt_ptr[i + 1] += F.jt_ptr[i];
  std::vector<int64_t> fill(F.jt_ptr.begin(), F.jt_ptr.end() - 1);
  F.jt_row.resize(nnzJd);
  F.jt_pos.resize(nnzJd);
  for (int64_t r = 0; r < md; r++)
    for (int64_t q = Jdp[r]; q < Jdp[r + 1]; q++) {
      const int64_t s = fill[Jdi[q]]++;
      F.jt_row[s] = (int32_t)r;
      F.jt_pos[s] = q;
    }
  return 0;
}

kkt_status cuda_status4(cudaError_t e) {
  if (e == cudaSuccess) return KKT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
}

kkt_status analyse4(int64_t n, int64_t m, int64_t md, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                    const int32_t* Ji, const int64_t* Jdp, const int32_t* Jdi, const kkt_options* opt, bool device,
                    kkt_handle4* out) {
  if (!out) return KKT_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || m < 0 || md < 0 || !Hp || !Hi || (md > 0 && (!Jdp || !Jdi))) return KKT_ERR_INVALID;
  Form4 F;
  if (form_pattern(n, md, Hp, Hi, Jdp, Jdi, F) != 0) return KKT_ERR_INVALID;
  kkt_handle4 h = new (std::nothrow) kkt_handle4_s();
  if (!h) return KKT_ERR_OOM;
  h->n = n; h->m = m; h->md = md;
  h->device = opt ? opt->device : 0;
  h->nnzHt = F.ht_ptr[n];
  h->nnzJd = md > 0 ? Jdp[md] : 0;
  kkt_status s = device ? kkt_analyse(n, m, F.ht_ptr.data(), F.ht_row.data(), Jp, Ji, opt, &h->inner)
                        : kkt_analyse_host(n, m, F.ht_ptr.data(), F.ht_row.data(), Jp, Ji, opt, &h->inner);
  if (s) { delete h; return s; }
  h->ht_ptr = std::move(F.ht_ptr);
  h->ht_row = std::move(F.ht_row);
  if (device) {
    Arena& A = h->mem;
    h->hpos = A.upload(F.hpos); h->dcol = A.upload(F.dcol);
    h->pr_ptr = A.upload(F.pr_ptr); h->pr_row = A.upload(F.pr_row);
    h->pr_a = A.upload(F.pr_a); h->pr_b = A.upload(F.pr_b);
    h->jt_ptr = A.upload(F.jt_ptr); h->jt_row = A.upload(F.jt_row); h->jt_pos = A.upload(F.jt_pos);
    h->jd_ptr = A.upload(md > 0 ? std::vector<int64_t>(Jdp, Jdp + md + 1) : std::vector<int64_t>(1, 0));
    h->jd_col = A.upload(md > 0 ? std::vector<int32_t>(Jdi, Jdi + h->nnzJd) : std::vector<int32_t>());
    h->ht_vals = A.alloc<double>(h->nnzHt);
    h->Jdv = A.alloc<double>(h->nnzJd);
    h->Ds = A.alloc<double>(md);
    h->rx = A.alloc<double>(n);
    if (A.failed) { kkt_destroy_4x4(h); return KKT_ERR_OOM; }
    h->on_device = true;
  }
  *out = h;
  return KKT_OK;
}

}  // namespace

extern "C" {

kkt_status kkt_analyse_4x4(int64_t n_x, int64_t m_c, int64_t m_d, const int64_t* H_colptr,
                           const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                           const int64_t* Jd_rowptr, const int32_t* Jd_colidx, const kkt_options* opt,
                           kkt_handle4* out) {
  if (opt && opt->ruiz_iters != 0) return KKT_ERR_INVALID;   // the 4x4 form does not scale
  return analyse4(n_x, m_c, m_d, H_colptr, H_rowidx, J_rowptr, J_colidx, Jd_rowptr, Jd_colidx, opt, true, out);
}

kkt_status kkt_analyse_4x4_host(int64_t n_x, int64_t m_c, int64_t m_d, const int64_t* H_colptr,
                                const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                                const int64_t* Jd_rowptr, const int32_t* Jd_colidx, const kkt_options* opt,
                                kkt_handle4* out) {
  return analyse4(n_x, m_c, m_d, H_colptr, H_rowidx, J_rowptr, J_colidx, Jd_rowptr, Jd_colidx, opt, false, out);
}

kkt_handle kkt_4x4_inner(kkt_handle4 h) { return h ? h->inner : nullptr; }

kkt_status kkt_get_4x4_pattern(kkt_handle4 h, int64_t* nnz, int64_t* colptr, int32_t* rowidx) {
  if (!h) return KKT_ERR_INVALID;
  if (nnz) *nnz = h->nnzHt;
  if (colptr) std::memcpy(colptr, h->ht_ptr.data(), sizeof(int64_t) * h->ht_ptr.size());
  if (rowidx && h->nnzHt) std::memcpy(rowidx, h->ht_row.data(), sizeof(int32_t) * h->ht_row.size());
  return KKT_OK;
}

kkt_status kkt_factor_4x4(kkt_handle4 h, const double* H_vals, const double* D_x, const double* Jd_vals,
                          const double* D_s, const double* J_vals, double delta, double gamma, void* stream) {
  if (!h || !H_vals || !D_x || (h->md > 0 && (!Jd_vals || !D_s))) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  kkt_status s;
  if ((s = cuda_status4(cudaSetDevice(h->device)))) return s;
  // the solve needs J_d and D_s after this call returns
  if (h->nnzJd && (s = cuda_status4(cudaMemcpyAsync(h->Jdv, Jd_vals, sizeof(double) * h->nnzJd,
                                                    cudaMemcpyDeviceToDevice, st))))
    return s;
  if (h->md && (s = cuda_status4(cudaMemcpyAsync(h->Ds, D_s, sizeof(double) * h->md, cudaMemcpyDeviceToDevice, st))))
    return s;
  k_form_htilde<<<grid_for(h->nnzHt), 256, 0, st>>>(h->nnzHt, h->hpos, h->dcol, h->pr_ptr, h->pr_row, h->pr_a,
                                                    h->pr_b, H_vals, D_x, h->Jdv, h->Ds, h->ht_vals);
  if ((s = cuda_status4(cudaGetLastError()))) return s;
  return kkt_factor(h->inner, h->ht_vals, J_vals, delta, gamma, stream);
}

kkt_status kkt_solve_4x4(kkt_handle4 h, const double* r_xt, const double* r_s, const double* r_y,
                         const double* r_yd, double* dx, double* ds, double* dy, double* dyd, void* stream) {
  if (!h || !r_xt || !dx || (h->m > 0 && (!r_y || !dy)) || (h->md > 0 && (!r_s || !r_yd || !ds || !dyd)))
    return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  kkt_status s;
  if ((s = cuda_status4(cudaSetDevice(h->device)))) return s;
  k_rhs_4x4<<<grid_for(h->n), 256, 0, st>>>(h->n, h->jt_ptr, h->jt_row, h->jt_pos, h->Jdv, h->Ds, r_xt, r_s, r_yd,
                                            h->rx);
  if ((s = cuda_status4(cudaGetLastError()))) return s;
  const kkt_status solved = kkt_solve(h->inner, h->rx, r_y, dx, dy, stream);
  if (solved != KKT_OK && solved != KKT_ERR_CG_MAXIT && solved != KKT_ERR_CG_BREAKDOWN) return solved;
  if (h->md) {
    k_recover_4x4<<<grid_for(h->md), 256, 0, st>>>(h->md, h->jd_ptr, h->jd_col, h->Jdv, h->Ds, dx, r_yd, r_s, ds,
                                                   dyd);
    if ((s = cuda_status4(cudaGetLastError()))) return s;
    if ((s = cuda_status4(cudaStreamSynchronize(st)))) return s;
  }
  return solved;
}

kkt_status kkt_destroy_4x4(kkt_handle4 h) {
  if (!h) return KKT_ERR_INVALID;
  if (h->inner) kkt_destroy(h->inner);
  if (!h->mem.ptrs.empty()) {
    cudaSetDevice(h->device);
    h->mem.release();
  }
  delete h;
  return KKT_OK;
}

}  // extern "C"
