// C ABI of the KKT solver: handle management, device memory, and the
// factor / solve / refinement drivers around the CUDA kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <climits>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "kkt.h"
#include "plan.hpp"
#include "symbolic.hpp"

using namespace kkt;

namespace {

struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool failed = false;
  template <typename X>
  X* alloc(size_t count) {
    if (failed) return nullptr;
    void* p = nullptr;
    const size_t b = sizeof(X) * (count ? count : 1);
    if (cudaMalloc(&p, b) != cudaSuccess) { cudaGetLastError(); failed = true; return nullptr; }
    ptrs.push_back(p);
    bytes += b;
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

}  // namespace

// concurrent solver handles of the batched form (kkt_solve_batch)
constexpr int kBatchSolvers = 4;

struct kkt_handle_s {
  kkt_options opt;
  Symbolic S;
  Plan P;
  std::vector<int64_t> hHp, hJp;   // host copies of the pattern (H~ lower CSC, J CSR)
  std::vector<int32_t> hHi, hJi;
  int device = 0;
  int grid = 0;
  int ctas = 2;   // solve-kernel CTAs per SM
  int grid2 = 0;  // the solve grid without the overlapped layout (several right-hand sides)
  int64_t nnzH = 0, nnzJ = 0;
  DevArena mem;
  // pattern / plan on the device
  int32_t *sfirst, *sw, *snr, *sld, *sparent, *rel, *sn_rows, *perm;
  int64_t *srow, *poff, *uoff;
  int4 *it_potrf, *it_trsm, *it_pupd, *it_syrk, *it_eadd, *it_syrk_tc, *it_block, *it_syrk128, *it_dstore,
      *it_tc_split;
  void* Dsc;
  float* Wtc = nullptr;         // split operand tiles of one tensor-core launch (FP32 factor)
  int64_t *slot_pos, *src_ptr;
  int32_t *srcA, *srcB;
  int32_t *Jcol_perm, *JT_row, *JT_vidx, *Hs_col, *Hs_vidx, *JTo_row, *JTo_vidx, *J_colidx;
  int64_t *JT_ptr, *Hs_ptr, *JTo_ptr, *J_rowptr;
  int32_t *pc_w, *pc_ld, *pc_c, *hd_tgt, *ch_tgt;
  int32_t *fwd_items, *bwd_items;
  int64_t *pc_colbase, *pc_inv;
  int32_t *st_first, *st_last, *st_clo, *st_chi, *st_tgt, *sn_piece;
  int64_t* st_tptr;
  int32_t *st_lptr, *st_lev, *st_sn;
  ChunkDesc* cdesc;
  HeadDesc* hdesc;
  uint8_t* tmaps;
  // values and workspace
  double *Hv, *Jv;
  void *L, *U, *v, *Linv;
  double *rhx, *p, *r, *y, *q, *bS, *red, *res_x, *res_y, *wv, *xa;
  double *stage_rx, *stage_ry, *stage_dx, *stage_dy;
  int* counters;   // fwd_arrive, fwd_done, bwd_arrive, bwd_done (npieces each), disp[3], bar[2]
  DevStatus* dst;
  DevStatus* hst = nullptr;  // pinned
  int32_t* rhs_stat = nullptr;   // per right-hand side: CG products, status, delta_2 restart
  // workspace of the multiple-right-hand-side solve (kMaxRhs vectors each),
  // allocated by the first kkt_solve_multi
  // saved factors of a batch of systems on this pattern (kkt_factor_batch):
  // slot b holds system b's panels, triangle inverses and values
  int64_t batch_cap = 0;
  void *bL = nullptr, *bLinv = nullptr;
  double *bHv = nullptr, *bJv = nullptr;
  std::vector<int32_t> bstatus;
  // FGMRES refinement workspace (first use): basis V (N x (kRestart + 1)),
  // preconditioned directions Z (N x kRestart), N = n + m
  double *fV = nullptr, *fZ = nullptr, *fw = nullptr, *fr = nullptr, *fzero = nullptr, *fpart = nullptr,
         *fdots = nullptr, *fcoef = nullptr, *fgs = nullptr;
  double* hflag = nullptr;   // pinned: the FGMRES stop flag and the step's residual contraction
  bool multi = false;
  void *mv;
  double *mrhx, *mp, *mr, *my, *mq, *mbS, *mres_x, *mres_y, *mwv, *mxa;
  double* d_dg = nullptr;    // device [delta, gamma, delta_min, delta_max, delta_prev, 0]: the
                             // assembly reads the first two, the delta_1 loop the rest
  unsigned long long* d_instr = nullptr;   // solve-kernel cycle counters (profile mode)
  unsigned long long* d_trace = nullptr;   // solve-kernel item timeline (profile mode)
  double* h_dg = nullptr;    // pinned staging for it
  cudaStream_t cap_stream = nullptr;   // private stream used to capture the factor graph
  cudaGraphExec_t fac_graph = nullptr; // the whole factorization as one CUDA graph
  cudaGraphExec_t reg_graph = nullptr; // Algorithm 1's delta_1 loop around it (conditional node)
  // what the solve reads: the single factor, or one system of the batch
  struct SolveView {
    void *L = nullptr, *Linv = nullptr;
    double *Hv = nullptr, *Jv = nullptr;
    uint8_t* tmaps = nullptr;
    int32_t tz = 0;   // the system's coordinate in the tensor maps' third dimension
  } sv;
  // batched form: nsys slots of panels, inverses, update matrices, diagonal
  // tile scratch, values and status; 3-D tensor maps over them; one graph
  void *bU = nullptr, *bDsc = nullptr;
  float* bWtc = nullptr;
  DevStatus* bst = nullptr;
  DevStatus* hbst = nullptr;   // pinned
  uint8_t* bs_maps = nullptr;
  cudaGraphExec_t bgraph = nullptr;
  int32_t bgraph_nb = 0;
  double bdelta = 0, bgamma = 0;   // the shift and gamma the batch was factored with
  // concurrent solves of a batch: helper handles made from this analysis
  // (own workspace and stream, a share of the SMs for the solve kernel) that
  // read each system's factor from the batch slots
  std::vector<kkt_handle> helpers;
  std::vector<cudaStream_t> hstreams;
  double delta_prev = 0;     // delta_1 accepted for the previous matrix of the sequence (Sec. 4.1)
  // Ruiz scaling (opt.ruiz_iters > 0): D, its scratch, ones, and the lower CSC pattern of H~
  double *d_D = nullptr, *d_Dtmp = nullptr, *d_ones = nullptr;
  // Krylov variants on S (opt.krylov): the J J^T handle of the preconditioner,
  // its value gather (pairs of J entries per lower entry), and workspace
  kkt_handle jjt = nullptr;
  int64_t* jjt_pp = nullptr;
  int32_t *jjt_pa = nullptr, *jjt_pb = nullptr;
  int64_t jjt_ne = 0;
  double* jjt_vals = nullptr;
  bool jjt_ok = false;
  double *kv = nullptr, *kpart = nullptr, *kdots = nullptr;
  int64_t* d_Hp = nullptr;
  int32_t* d_Hi = nullptr;
  // state
  bool on_device = false;   // false for a host-only (symbolic) handle
  bool factored = false;
  double delta = 0, gamma = 0;
  kkt_info info{};
  int inertia_ok = 0;
  Prof prof;
  Prof* profp = nullptr;   // non-null when opt.profile
  // the solve kernel is timed in every mode: one event pair per pass, read
  // after the pass's status read has synchronised the stream anyway
  cudaEvent_t cg_a = nullptr, cg_b = nullptr;
};

// Tensor maps of the pieces whose row tiles are staged as 2-D TMA boxes:
// the piece's pw columns of its supernode panel (ld rows each, rows past
// the panel read as zeros), box = pc_box rows x pw columns. The encoder is
// the driver's, fetched through the runtime (no link against libcuda).
static bool build_tensor_maps(const Plan& P, void* L, size_t es, int depth, std::vector<uint8_t>& out) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  out.assign((size_t)P.npieces * 128, 0);
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  for (int64_t p = 0; p < P.npieces; p++) {
    if (P.pc_box[p] <= 0) continue;
    const int32_t pw = P.pc_w[p], ld = P.pc_ld[p], box = P.pc_box[p];
    if (box > 256 || pw > 256 || (box * es) % 16 || ((size_t)ld * es) % 16 || (P.pc_colbase[p] * es) % 16) return false;
    // third dimension: the systems of a batch (panel sets panel_total apart)
    const cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)pw, (cuuint64_t)depth};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)P.panel_total * es};
    const cuuint32_t boxd[3] = {(cuuint32_t)box, (cuuint32_t)pw, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap* m = (CUtensorMap*)(out.data() + (size_t)p * 128);
    void* g = (char*)L + (size_t)P.pc_colbase[p] * es;
    if (encode(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g, dims, strides,
               boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

static kkt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KKT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
}
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

extern "C" {

void kkt_default_options(kkt_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gamma = 1e4;
  o->delta2 = 1e-9;
  o->cg_rtol = 0;      // by precision, resolved in the analysis
  o->cg_maxit = 1000;
  o->ir_maxit = -1;     // by precision, resolved in the analysis
  o->ir_rtol = 0;       // by precision, resolved in the analysis
  o->precision = KKT_FP64;
  o->ordering = 0;
  o->relax_small = 16;
  o->relax_num = 1;
  o->relax_den = 10;
  o->relax_wmax = 256;
  o->solve_w = 0;
  o->device = 0;
  o->debug_stall_piece = -1;
  o->spin_cycles = 0;
  o->profile = 0;
  o->nd_leaf = 64;
  o->tensor_cores = 1;
  o->ruiz_iters = 0;
  o->krylov = 0;
  o->solve_sms = 0;
  o->tc_panel_min = 0;
}

const char* kkt_status_string(kkt_status s) {
  switch (s) {
    case KKT_OK: return "ok";
    case KKT_ERR_INVALID: return "invalid argument or pattern";
    case KKT_ERR_NOT_SPD: return "H_delta is not positive definite (Cholesky pivot <= 0)";
    case KKT_ERR_CG_BREAKDOWN: return "CG breakdown on the Schur complement";
    case KKT_ERR_CG_MAXIT: return "CG reached its iteration limit";
    case KKT_ERR_OOM: return "device out of memory";
    case KKT_ERR_CUDA: return "CUDA error";
    case KKT_ERR_TIMEOUT: return "bounded wait in a persistent kernel timed out";
    case KKT_ERR_STATE: return "call out of order";
    case KKT_ERR_TOO_LARGE: return "n + m exceeds the no-allocation scratch (KKT_NOALLOC_MAX_ROWS)";
  }
  return "unknown status";
}

kkt_status kkt_destroy(kkt_handle h) {
  if (!h) return KKT_ERR_INVALID;
  if (!h->mem.ptrs.empty()) {
    cudaSetDevice(h->device);
    h->mem.release();
  }
  if (h->hst) cudaFreeHost(h->hst);
  if (h->h_dg) cudaFreeHost(h->h_dg);
  if (h->fac_graph) cudaGraphExecDestroy(h->fac_graph);
  if (h->reg_graph) cudaGraphExecDestroy(h->reg_graph);
  if (h->jjt) kkt_destroy(h->jjt);
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  if (h->bU) { cudaFree(h->bU); cudaFree(h->bDsc); cudaFree(h->bst); cudaFree(h->bs_maps); cudaFree(h->bWtc); }
  if (h->hbst) cudaFreeHost(h->hbst);
  if (h->hflag) cudaFreeHost(h->hflag);
  for (kkt_handle x : h->helpers) kkt_destroy(x);
  for (cudaStream_t x : h->hstreams) cudaStreamDestroy(x);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->prof.a) cudaEventDestroy(h->prof.a);
  if (h->prof.b) cudaEventDestroy(h->prof.b);
  if (h->bL) { cudaFree(h->bL); cudaFree(h->bLinv); cudaFree(h->bHv); cudaFree(h->bJv); }
  if (h->cg_a) cudaEventDestroy(h->cg_a);
  if (h->cg_b) cudaEventDestroy(h->cg_b);
  delete h;
  return KKT_OK;
}

static kkt_status analyse_host_impl(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                                    const int32_t* Ji, const kkt_options* opt, const Symbolic* reuse,
                                    kkt_handle* out) {
  if (!out) return KKT_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || m < 0 || !Hp || !Hi || (m > 0 && (!Jp || !Ji))) return KKT_ERR_INVALID;
  kkt_handle h = new (std::nothrow) kkt_handle_s();
  if (!h) return KKT_ERR_OOM;
  if (opt) h->opt = *opt; else kkt_default_options(&h->opt);
  const kkt_options& o = h->opt;
  if ((o.solve_w != 0 && (o.solve_w < 32 || o.solve_w > 256)) || o.relax_den <= 0 || o.precision < 0 ||
      o.precision > 1 || o.solve_ctas < 0 || o.solve_ctas == 1 || o.solve_ctas > 4 || o.refine < 0 ||
      o.refine > 2 || o.ruiz_iters < 0 || o.ruiz_iters > 100 || o.krylov < 0 || o.krylov > 2 || o.solve_sms < 0 ||
      (o.tc_panel_min != 0 && o.tc_panel_min < 128) ||
      (o.krylov != 0 && o.precision != KKT_FP64) ||
      (o.solve_ent != 0 && (o.solve_ent < 2048 || o.solve_ent > 32768))) {
    delete h;
    return KKT_ERR_INVALID;
  }
  // precision-dependent defaults: FP64 solves S to Sec. 5.1's 1e-12 in one
  // pass (refinement is a safety net); the FP32 factor bounds what one pass
  // can reach, so a mixed pass stops early and FP64 refinement does the rest
  const bool f64d = o.precision == KKT_FP64;
  if (!(h->opt.cg_rtol > 0)) h->opt.cg_rtol = f64d ? 1e-12 : 3e-3;
  if (h->opt.refine == 0) h->opt.refine = 2;
  if (h->opt.ir_maxit < 0) h->opt.ir_maxit = f64d ? 3 : (h->opt.refine == 2 ? 60 : 10);
  if (!(h->opt.ir_rtol > 0)) h->opt.ir_rtol = f64d ? 1e-10 : 1e-9;
  static const int64_t zero = 0;
  if (m == 0) Jp = &zero;
  RelaxParams rp;
  rp.small = o.relax_small; rp.num = o.relax_num; rp.den = o.relax_den; rp.wmax = o.relax_wmax;
  if (o.ordering < 0 || o.ordering > 2 || (o.ordering == 2 && o.nd_leaf < 1)) { delete h; return KKT_ERR_INVALID; }
  if (reuse) {
    h->S = *reuse;
  } else if (analyse_pattern(n, m, Hp, Hi, Jp, Ji, rp, o.ordering, o.nd_leaf, h->S) != 0) {
    delete h;
    return KKT_ERR_INVALID;
  }
  // host copies of the pattern: the device set-up and kkt_analyse_like read them
  h->hHp.assign(Hp, Hp + n + 1);
  h->hHi.assign(Hi, Hi + Hp[n]);
  h->hJp.assign(Jp, Jp + m + 1);
  h->hJi.assign(Ji, Ji + Jp[m]);
  // piece width and L entries per solve item. FP64: chunks, heads' chunk 0
  // and subtrees of 8192 entries, two solve CTAs per SM (about 98 KB of
  // shared memory each). FP32 factors of at least kSolveOverlapMin panel
  // entries: chunk tiles of 16000 entries share their region with the heads'
  // inverses (ent0 = subtree entries = 7680), about 73 KB per CTA, three per
  // SM (measured: 100^3, 1.2e10 entries, 15 % faster solves; 500 x 500,
  // 3.2e8, unchanged); smaller FP32 factors keep 16384 entries for all items
  // and two CTAs per SM (a 200 x 100 grid, 8e6 entries, was 5 % slower with
  // the smaller head and subtree items).
  constexpr int64_t kSolveOverlapMin = 100000000;
  const bool f64o = o.precision == KKT_FP64;
  const int sw = o.solve_w > 0 ? o.solve_w : (f64o ? 64 : 128);
  // the triangle inversion holds a piece's sw x sw triangle in shared memory
  if ((size_t)sw * sw * (f64o ? 8 : 4) > (size_t)200 * 1024) { delete h; return KKT_ERR_INVALID; }
  auto plan = [&](int ov) {
    const int ent = o.solve_ent > 0 ? o.solve_ent : (f64o ? 8192 : (ov ? 16000 : 16384));
    const int ent0 = ov ? std::min(ent, 7680) : ent;
    return build_plan(h->S, Hp, Hi, Jp, Ji, sw, ent, ent0, ent0, ov, !f64o && o.tensor_cores, !f64o,
                      o.tc_panel_min ? o.tc_panel_min : kTcPanelMinWidth, h->P);
  };
  int pr = plan(f64o ? 0 : 1);
  if (pr == 0 && h->P.solve_ov && h->P.panel_total < kSolveOverlapMin) pr = plan(0);
  if (pr != 0) {
    delete h;
    return KKT_ERR_INVALID;
  }
  if (o.debug_stall_piece >= 0 && o.debug_stall_piece < h->P.npieces) h->P.pc_need[o.debug_stall_piece] += 1;
  h->nnzH = Hp[n];
  h->nnzJ = Jp[m];
  *out = h;
  return KKT_OK;
}

static kkt_status analyse_host(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                               const int32_t* Ji, const kkt_options* opt, kkt_handle* out) {
  return analyse_host_impl(n, m, Hp, Hi, Jp, Ji, opt, nullptr, out);
}

static kkt_status device_stage(kkt_handle h, kkt_handle* out);

kkt_status kkt_analyse_host(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                            const int32_t* Ji, const kkt_options* opt, kkt_handle* out) {
  return analyse_host(n, m, Hp, Hi, Jp, Ji, opt, out);
}

kkt_status kkt_analyse(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                       const int32_t* Ji, const kkt_options* opt, kkt_handle* out) {
  kkt_status s0 = analyse_host(n, m, Hp, Hi, Jp, Ji, opt, out);
  if (s0) return s0;
  kkt_handle h = *out;
  *out = nullptr;
  return device_stage(h, out);
}

kkt_status kkt_analyse_like(kkt_handle src, const kkt_options* opt, kkt_handle* out) {
  if (!src || !out) return KKT_ERR_INVALID;
  *out = nullptr;
  kkt_options o;
  if (opt) o = *opt; else kkt_default_options(&o);
  const kkt_options& so = src->opt;
  if (o.ordering != so.ordering || (o.ordering == 2 && o.nd_leaf != so.nd_leaf) || o.relax_small != so.relax_small ||
      o.relax_num != so.relax_num || o.relax_den != so.relax_den || o.relax_wmax != so.relax_wmax)
    return KKT_ERR_INVALID;
  const int64_t n = src->S.n, m = src->S.m;
  kkt_status s0 = analyse_host_impl(n, m, src->hHp.data(), src->hHi.data(), src->hJp.data(), src->hJi.data(), &o,
                                    &src->S, out);
  if (s0) return s0;
  kkt_handle h = *out;
  *out = nullptr;
  return device_stage(h, out);
}

static kkt_status device_stage(kkt_handle h, kkt_handle* out) {
  const kkt_options& o = h->opt;
  const int64_t n = h->S.n, m = h->S.m;
  const int64_t* Jp = h->hJp.data();
  const int32_t* Ji = h->hJi.data();
  h->device = o.device;
  if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); delete h; return KKT_ERR_CUDA; }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
  if (!coop) { delete h; return KKT_ERR_CUDA; }
  const bool f64 = o.precision == KKT_FP64;
  const Plan& Pl = h->P;
  h->ctas = o.solve_ctas > 0 ? o.solve_ctas : (Pl.solve_ov ? 3 : 2);
  h->grid = f64 ? solve_grid_size<double>(h->device, Pl.solve_w, Pl.ent, Pl.ent0, Pl.esub, Pl.max_rows, Pl.solve_ov,
                                          h->ctas)
                : solve_grid_size<float>(h->device, Pl.solve_w, Pl.ent, Pl.ent0, Pl.esub, Pl.max_rows, Pl.solve_ov,
                                         h->ctas);
  h->grid2 = !Pl.solve_ov ? h->grid
                          : solve_grid_size<float>(h->device, Pl.solve_w, Pl.ent, Pl.ent0, Pl.esub, Pl.max_rows, 0, 2);
  if (h->grid <= 0 || h->grid2 <= 0) { delete h; return KKT_ERR_INVALID; }
  if (o.solve_sms > 0) {
    h->grid = std::min(h->grid, h->ctas * o.solve_sms);
    h->grid2 = std::min(h->grid2, 2 * o.solve_sms);
  }
  const Plan& P = h->P;
  DevArena& A = h->mem;
  auto as_int4 = [&](const std::vector<int32_t>& v) {
    int4* d = A.alloc<int4>(v.size() / 4);
    if (d && !v.empty() && cudaMemcpy(d, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice)) A.failed = true;
    return d;
  };
  h->sfirst = A.upload(P.sfirst); h->sw = A.upload(P.sw); h->snr = A.upload(P.snr); h->sld = A.upload(P.sld);
  h->sparent = A.upload(P.sparent); h->rel = A.upload(P.rel); h->sn_rows = A.upload(h->S.sn_rows);
  h->perm = A.upload(h->S.perm);
  h->srow = A.upload(P.srow); h->poff = A.upload(P.poff); h->uoff = A.upload(P.uoff);
  h->it_potrf = as_int4(P.it_potrf);
  h->it_trsm = as_int4(P.it_trsm); h->it_pupd = as_int4(P.it_pupd);
  h->it_syrk = as_int4(P.it_syrk); h->it_eadd = as_int4(P.it_eadd); h->it_syrk_tc = as_int4(P.it_syrk_tc);
  h->it_block = as_int4(P.it_block); h->it_syrk128 = as_int4(P.it_syrk128); h->it_dstore = as_int4(P.it_dstore);
  h->it_tc_split = as_int4(P.it_tc_split);
  h->slot_pos = A.upload(P.slot_pos); h->src_ptr = A.upload(P.src_ptr);
  h->srcA = A.upload(P.srcA); h->srcB = A.upload(P.srcB);
  h->Jcol_perm = A.upload(P.Jcol_perm); h->JT_ptr = A.upload(P.JT_ptr);
  h->JT_row = A.upload(P.JT_row); h->JT_vidx = A.upload(P.JT_vidx);
  h->Hs_ptr = A.upload(P.Hs_ptr); h->Hs_col = A.upload(P.Hs_col); h->Hs_vidx = A.upload(P.Hs_vidx);
  h->JTo_ptr = A.upload(P.JTo_ptr); h->JTo_row = A.upload(P.JTo_row); h->JTo_vidx = A.upload(P.JTo_vidx);
  h->J_rowptr = A.upload(std::vector<int64_t>(Jp, Jp + m + 1));
  h->J_colidx = A.upload(std::vector<int32_t>(Ji, Ji + h->nnzJ));
  // pieces: the triangle inversion's inputs, the inverses' offsets and the
  // target lists (the rest of each work item's description is in its descriptor)
  h->pc_w = A.upload(P.pc_w); h->pc_ld = A.upload(P.pc_ld); h->pc_c = A.upload(P.pc_c);
  h->pc_colbase = A.upload(P.pc_colbase); h->pc_inv = A.upload(P.pc_inv);
  h->hd_tgt = A.upload(P.hd_tgt); h->ch_tgt = A.upload(P.ch_tgt);
  h->fwd_items = A.upload(P.fwd_items); h->bwd_items = A.upload(P.bwd_items);
  h->st_first = A.upload(P.st_first); h->st_last = A.upload(P.st_last); h->st_clo = A.upload(P.st_clo);
  h->st_chi = A.upload(P.st_chi); h->st_tgt = A.upload(P.st_tgt); h->st_tptr = A.upload(P.st_tptr);
  h->st_lptr = A.upload(P.st_lptr); h->st_lev = A.upload(P.st_lev); h->st_sn = A.upload(P.st_sn);
  {
    std::vector<HeadDesc> hd = P.hdesc;
    for (size_t p = 0; p < hd.size(); p++) hd[p].need = P.pc_need[p];
    h->hdesc = A.upload(hd);
    h->cdesc = A.upload(P.cdesc);
  }
  h->sn_piece = A.upload(P.sn_piece);
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  h->Hv = A.alloc<double>(h->nnzH); h->Jv = A.alloc<double>(h->nnzJ);
  h->L = A.alloc<char>(es * (size_t)P.panel_total);
  h->U = A.alloc<char>(es * (size_t)P.u_total);
  h->Dsc = A.alloc<char>(es * (size_t)P.dsc_total);
  if (!f64 && P.tc_ws_tiles > 0) h->Wtc = A.alloc<float>((size_t)P.tc_ws_tiles * kTcTileFloats);
  h->v = A.alloc<char>(es * (size_t)n);
  h->Linv = A.alloc<char>(es * (size_t)P.inv_total);
  {
    std::vector<uint8_t> maps;
    if (!A.failed) {
      if (!build_tensor_maps(P, h->L, es, 1, maps)) { kkt_destroy(h); return KKT_ERR_CUDA; }
      h->tmaps = A.upload(maps);
      h->sv.L = h->L; h->sv.Linv = h->Linv; h->sv.Hv = h->Hv; h->sv.Jv = h->Jv; h->sv.tmaps = h->tmaps; h->sv.tz = 0;
    }
  }
  h->rhx = A.alloc<double>(n);
  h->wv = A.alloc<double>(n); h->xa = A.alloc<double>(n);
  h->p = A.alloc<double>(m); h->r = A.alloc<double>(m); h->y = A.alloc<double>(m);
  h->q = A.alloc<double>(m); h->bS = A.alloc<double>(m);
  h->red = A.alloc<double>((size_t)std::max(h->grid, 296) * kRedStride);
  h->rhs_stat = A.alloc<int32_t>(3 * kMaxRhs);
  h->res_x = A.alloc<double>(n); h->res_y = A.alloc<double>(m);
  h->stage_rx = A.alloc<double>(n); h->stage_ry = A.alloc<double>(m);
  h->stage_dx = A.alloc<double>(n); h->stage_dy = A.alloc<double>(m);
  h->counters = A.alloc<int>(4 * (size_t)P.npieces + 8);
  h->dst = A.alloc<DevStatus>(1);
  h->d_dg = A.alloc<double>(6);
  if (o.ruiz_iters > 0) {
    h->d_D = A.alloc<double>(n + m);
    h->d_Dtmp = A.alloc<double>(n + m);
    h->d_ones = A.upload(std::vector<double>(n + m, 1.0));
    h->d_Hp = A.upload(h->hHp);
    h->d_Hi = A.upload(h->hHi);
  }
  h->d_instr = A.alloc<unsigned long long>(32);
  if (o.profile) h->d_trace = A.alloc<unsigned long long>(6 * P.fwd_items.size() + 6);
  if (o.krylov == 1 && m > 0 && !A.failed) {
    // lower pattern of J J^T (column r2, rows r1 >= r2 that share a column of
    // J with r2) and, per entry, the pairs of J entries whose products sum to it
    struct Tri { int32_t r2, r1, qa, qb; };
    std::vector<Tri> tri;
    for (int64_t c = 0; c < n; c++)
      for (int64_t a1 = P.JTo_ptr[c]; a1 < P.JTo_ptr[c + 1]; a1++)
        for (int64_t a2 = P.JTo_ptr[c]; a2 < P.JTo_ptr[c + 1]; a2++)
          if (P.JTo_row[a1] >= P.JTo_row[a2]) tri.push_back({P.JTo_row[a2], P.JTo_row[a1], P.JTo_vidx[a1], P.JTo_vidx[a2]});
    std::sort(tri.begin(), tri.end(), [](const Tri& x, const Tri& y) {
      return x.r2 != y.r2 ? x.r2 < y.r2 : (x.r1 != y.r1 ? x.r1 < y.r1 : (x.qa != y.qa ? x.qa < y.qa : x.qb < y.qb));
    });
    std::vector<int64_t> cp(m + 1, 0), pp;
    std::vector<int32_t> ri, pa, pb;
    for (size_t t = 0; t < tri.size(); t++) {
      if (t == 0 || tri[t].r2 != tri[t - 1].r2 || tri[t].r1 != tri[t - 1].r1) {
        ri.push_back(tri[t].r1);
        cp[tri[t].r2 + 1]++;
        pp.push_back((int64_t)t);
      }
      pa.push_back(tri[t].qa);
      pb.push_back(tri[t].qb);
    }
    pp.push_back((int64_t)tri.size());
    for (int64_t r = 0; r < m; r++) cp[r + 1] += cp[r];
    kkt_options so;
    kkt_default_options(&so);
    so.precision = KKT_FP64;
    so.ordering = o.ordering;
    so.nd_leaf = o.nd_leaf;
    so.device = o.device;
    const kkt_status sj = kkt_analyse(m, 0, cp.data(), ri.data(), nullptr, nullptr, &so, &h->jjt);
    if (sj) { kkt_destroy(h); return sj; }
    h->jjt_ne = (int64_t)ri.size();
    h->jjt_pp = A.upload(pp);
    h->jjt_pa = A.upload(pa);
    h->jjt_pb = A.upload(pb);
    h->jjt_vals = A.alloc<double>(ri.size());
  }
  if (A.failed) { kkt_destroy(h); return KKT_ERR_OOM; }
  if (cudaMallocHost(&h->hst, sizeof(DevStatus)) != cudaSuccess) { cudaGetLastError(); h->hst = nullptr; kkt_destroy(h); return KKT_ERR_OOM; }
  if (cudaMallocHost(&h->h_dg, 6 * sizeof(double)) != cudaSuccess) { cudaGetLastError(); h->h_dg = nullptr; kkt_destroy(h); return KKT_ERR_OOM; }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); h->cap_stream = nullptr; kkt_destroy(h); return KKT_ERR_CUDA; }
  // (no device-wide synchronisation here: other threads may be capturing a
  // graph or running solves on their own streams; the uploads above are
  // synchronous copies)
  if (cudaEventCreate(&h->cg_a) != cudaSuccess || cudaEventCreate(&h->cg_b) != cudaSuccess) {
    cudaGetLastError();
    kkt_destroy(h);
    return KKT_ERR_CUDA;
  }
  if (o.profile) {
    if (cudaEventCreate(&h->prof.a) != cudaSuccess || cudaEventCreate(&h->prof.b) != cudaSuccess) {
      cudaGetLastError();
      kkt_destroy(h);
      return KKT_ERR_CUDA;
    }
    h->profp = &h->prof;
    if (cudaMemset(h->d_instr, 0, 32 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(h->d_trace, 0, (6 * h->P.fwd_items.size() + 6) * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      kkt_destroy(h);
      return KKT_ERR_CUDA;
    }
  }
  h->on_device = true;
  *out = h;
  return KKT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ drivers
// Ruiz scaling of the values just copied into h->Hv / h->Jv (in place)
static kkt_status apply_scaling(kkt_handle h, cudaStream_t st) {
  if (h->opt.ruiz_iters <= 0) return KKT_OK;
  const Plan& P = h->P;
  RuizArgs a;
  a.n = P.n; a.m = P.m;
  a.Hs_ptr = h->Hs_ptr; a.Hs_col = h->Hs_col; a.Hs_vidx = h->Hs_vidx;
  a.H_colptr = h->d_Hp; a.H_rowidx = h->d_Hi;
  a.JT_ptr = h->JTo_ptr; a.JT_row = h->JTo_row; a.JT_vidx = h->JTo_vidx;
  a.J_rowptr = h->J_rowptr; a.J_colidx = h->J_colidx;
  a.Hv = h->Hv; a.Jv = h->Jv; a.ones = h->d_ones;
  CK(launch_ruiz(a, h->opt.ruiz_iters, h->d_D, h->d_Dtmp, h->Hv, h->Jv, st));
  return KKT_OK;
}

static kkt_status reset_status(kkt_handle h, cudaStream_t st) {
  std::memset(h->hst, 0, sizeof(DevStatus));
  h->hst->fail_col = INT_MAX;
  CK(cudaMemcpyAsync(h->dst, h->hst, sizeof(DevStatus), cudaMemcpyHostToDevice, st));
  return KKT_OK;
}

static kkt_status read_status(kkt_handle h, cudaStream_t st) {
  CK(cudaMemcpyAsync(h->hst, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return KKT_OK;
}

template <typename T>
static cudaError_t factor_launches(kkt_handle h, cudaStream_t st, Prof* prof, int nb = 0) {
  // nb > 0: the batched form, nb systems in the batch slots (system b =
  // blockIdx.y of every launch); nb = 0: the single factor
  FacArgs<T> a;
  a.sfirst = h->sfirst; a.sw = h->sw; a.snr = h->snr; a.sld = h->sld; a.sparent = h->sparent; a.rel = h->rel;
  a.srow = h->srow; a.poff = h->poff; a.uoff = h->uoff;
  a.Hv = h->Hv; a.Jv = h->Jv;
  a.L = (T*)h->L; a.U = (T*)h->U; a.Dsc = (T*)h->Dsc; a.st = h->dst; a.W = h->Wtc;
  if (nb > 0) {
    a.Hv = h->bHv; a.Jv = h->bJv;
    a.L = (T*)h->bL; a.U = (T*)h->bU; a.Dsc = (T*)h->bDsc; a.st = h->bst; a.W = h->bWtc;
    a.bsL = h->P.panel_total; a.bsU = h->P.u_total; a.bsD = h->P.dsc_total;
    a.bsW = h->P.tc_ws_tiles * kTcTileFloats;
    a.bsH = h->nnzH; a.bsJ = h->nnzJ;
  }
  FacLists fl;
  fl.it_potrf = h->it_potrf; fl.it_trsm = h->it_trsm; fl.it_pupd = h->it_pupd;
  fl.it_syrk = h->it_syrk; fl.it_eadd = h->it_eadd; fl.it_syrk_tc = h->it_syrk_tc;
  fl.it_block = h->it_block; fl.it_syrk128 = h->it_syrk128; fl.it_dstore = h->it_dstore;
  fl.it_tc_split = h->it_tc_split;
  fl.slot_pos = h->slot_pos; fl.src_ptr = h->src_ptr; fl.srcA = h->srcA; fl.srcB = h->srcB;
  fl.nslot = (int64_t)h->P.slot_pos.size();
  fl.panel_total = h->P.panel_total; fl.u_total = h->P.u_total;
  fl.launches = &h->P.launches;
  cudaError_t e = launch_factor<T>(a, fl, h->d_dg, st, prof, nb > 0 ? nb : 1);
  if (e) return e;
  InvArgs<T> ia;
  ia.pc_w = h->pc_w; ia.pc_ld = h->pc_ld; ia.pc_c = h->pc_c;
  ia.pc_colbase = h->pc_colbase; ia.pc_inv = h->pc_inv;
  ia.L = (const T*)h->L; ia.Linv = (T*)h->Linv;
  if (nb > 0) {
    ia.L = (const T*)h->bL; ia.Linv = (T*)h->bLinv;
    ia.bsL = h->P.panel_total; ia.bsI = h->P.inv_total;
  }
  if ((e = prof_begin(prof, st))) return e;
  if ((e = launch_tri_inv<T>(ia, h->P.npieces, h->P.solve_w, st, nb > 0 ? nb : 1))) return e;
  return prof_end(prof, KKT_K_TRI_INV, st);
}

// The factorization's launch sequence depends only on the pattern, so it is
// captured once into a CUDA graph (on a private stream) and replayed on the
// caller's stream for every value update; delta and gamma are read from
// device memory. Profile mode launches kernel by kernel instead.
template <typename T>
static kkt_status factor_impl(kkt_handle h, cudaStream_t st) {
  h->h_dg[0] = h->delta;
  h->h_dg[1] = h->gamma;
  CK(cudaMemcpyAsync(h->d_dg, h->h_dg, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
  if (h->profp) {
    CK(factor_launches<T>(h, st, h->profp));
    return KKT_OK;
  }
  if (!h->fac_graph) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = factor_launches<T>(h, h->cap_stream, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e || e2) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return KKT_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&h->fac_graph, g, 0);
    cudaGraphDestroy(g);
    if (e) { h->fac_graph = nullptr; return cuda_status(e); }
  }
  CK(cudaGraphLaunch(h->fac_graph, st));
  return KKT_OK;
}

static kkt_status post_factor(kkt_handle h, cudaStream_t st);

static kkt_status factor_common(kkt_handle h, double delta, double gamma, cudaStream_t st) {
  h->factored = false;
  h->inertia_ok = 0;
  if (!(delta >= 0.0) || !std::isfinite(delta)) return KKT_ERR_INVALID;
  if (gamma < 0) gamma = h->opt.gamma;
  if (!std::isfinite(gamma)) return KKT_ERR_INVALID;
  h->delta = delta;
  h->gamma = gamma;
  kkt_status s = reset_status(h, st);
  if (s) return s;
  s = h->opt.precision == KKT_FP64 ? factor_impl<double>(h, st) : factor_impl<float>(h, st);
  if (s) return s;
  if ((s = read_status(h, st))) return s;
  if (h->hst->abort) return KKT_ERR_TIMEOUT;
  if (h->hst->fail_col != INT_MAX) return KKT_ERR_NOT_SPD;
  h->factored = true;
  return post_factor(h, st);
}

// Algorithm 1's regularization loop with the sequence rule of Sec. 4.1:
// delta_1 = 0; while the Cholesky fails and delta_1 <= delta_max / 2,
// delta_1 becomes the previous matrix's accepted value (delta_min when that
// was 0) on the first retry, then doubles. The loop runs on the device as
// one CUDA graph: a conditional WHILE node whose body is the captured
// factorization followed by k_reg_next, which reads the pivot status and
// either ends the loop or writes the next shift to device memory (the
// assembly reads it there) and clears the status for the next trial. One
// launch and one status read per call, whatever the number of trials.
__global__ void k_reg_next(cudaGraphConditionalHandle loop, double* dg, DevStatus* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double d1 = dg[0], dmin = dg[2], dmax = dg[3], prev = dg[4];
  unsigned go = 0;
  if (st->fail_col != INT_MAX && st->abort == 0 && d1 <= dmax / 2) {
    dg[0] = d1 == 0.0 ? (prev > 0.0 ? prev : dmin) : 2.0 * d1;
    st->fail_col = INT_MAX;
    go = 1;
  }
  cudaGraphSetConditional(loop, go);
}

template <typename T>
static kkt_status build_reg_graph(kkt_handle h) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle loop;
  cudaError_t e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
  // the parameter union has no default constructor: zero raw storage
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  std::memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (!e) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  if (!e) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (!e) {
      cudaError_t e1 = factor_launches<T>(h, h->cap_stream, nullptr);
      if (!e1) {
        k_reg_next<<<1, 32, 0, h->cap_stream>>>(loop, h->d_dg, h->dst);
        e1 = cudaGetLastError();
      }
      e = cudaStreamEndCapture(h->cap_stream, &body);
      if (!e) e = e1;
    }
  }
  if (!e) e = cudaGraphInstantiate(&h->reg_graph, g, 0);
  cudaGraphDestroy(g);
  if (e) {
    h->reg_graph = nullptr;
    cudaGetLastError();
    return cuda_status(e);
  }
  return KKT_OK;
}

template <typename T>
static SolveArgs<T> solve_args(kkt_handle h) {
  SolveArgs<T> a;
  const Plan& P = h->P;
  a.n = P.n; a.m = P.m;
  a.sn_rows = h->sn_rows;
  a.pc_inv = h->pc_inv; a.hd_tgt = h->hd_tgt;
  a.sw = P.solve_w; a.ent = P.ent; a.ent0 = P.ent0; a.max_rows = P.max_rows;
  a.esub = P.esub; a.ov = P.solve_ov;
  a.Linv = (const T*)h->sv.Linv;
  a.ch_tgt = h->ch_tgt;
  a.fwd_items = h->fwd_items; a.bwd_items = h->bwd_items;
  a.nitems = (int64_t)P.fwd_items.size();
  a.npieces = P.npieces;
  a.st_first = h->st_first; a.st_last = h->st_last; a.st_clo = h->st_clo; a.st_chi = h->st_chi;
  a.st_tgt = h->st_tgt; a.st_tptr = h->st_tptr; a.sn_piece = h->sn_piece;
  a.st_lptr = h->st_lptr; a.st_lev = h->st_lev; a.st_sn = h->st_sn;
  a.cdesc = h->cdesc; a.hdesc = h->hdesc; a.tmaps = h->sv.tmaps; a.tz = h->sv.tz;
  a.sfirst = h->sfirst; a.sw_ = h->sw; a.snr = h->snr; a.sld = h->sld; a.srow = h->srow; a.poff = h->poff;
  a.L = (const T*)h->sv.L;
  a.J_rowptr = h->J_rowptr; a.Jcol_perm = h->Jcol_perm; a.Jv = h->sv.Jv;
  a.JT_ptr = h->JT_ptr; a.JT_row = h->JT_row; a.JT_vidx = h->JT_vidx;
  a.perm = h->perm;
  a.gamma = h->gamma; a.delta2 = h->opt.delta2; a.rtol = h->opt.cg_rtol; a.maxit = h->opt.cg_maxit;
  a.v = (T*)h->v; a.rhx = h->rhx; a.p = h->p; a.r = h->r; a.y = h->y; a.q = h->q; a.bS = h->bS;
  a.wv = h->wv; a.xa = h->xa;
  a.xacc = h->opt.precision == KKT_MIXED ? 1 : 0;
  const int64_t np = P.npieces;
  a.fwd_arrive = h->counters; a.fwd_done = h->counters + np;
  a.bwd_arrive = h->counters + 2 * np; a.bwd_done = h->counters + 3 * np;
  a.disp = h->counters + 4 * np; a.bar = h->counters + 4 * np + 4;
  a.red = h->red; a.st = h->dst;
  a.nrhs = 1; a.rhs_stat = h->rhs_stat;
  a.spin = h->opt.spin_cycles > 0 ? h->opt.spin_cycles : kSpinCycles;
  a.instr = h->profp ? h->d_instr : nullptr;
  a.trace = h->profp ? h->d_trace : nullptr;
  return a;
}

template <typename T>
static kkt_status solve_pass(kkt_handle h, const double* bx, const double* by, double* ox, double* oy,
                             int accumulate, int mode, cudaStream_t st, int nrhs = 1, double rtol = 0.0) {
  CK(cudaMemsetAsync(h->counters, 0, sizeof(int) * (4 * (size_t)h->P.npieces + 8), st));
  SolveArgs<T> a = solve_args<T>(h);
  if (rtol > 0) a.rtol = rtol;
  a.bx = bx; a.by = by; a.ox = ox; a.oy = oy; a.accumulate = accumulate; a.mode = mode;
  if (nrhs > 1) {
    a.nrhs = nrhs;
    a.v = (T*)h->mv; a.rhx = h->mrhx;
    a.p = h->mp; a.r = h->mr; a.y = h->my; a.q = h->mq; a.bS = h->mbS;
    a.wv = h->mwv; a.xa = h->mxa;
  }
  // several right-hand sides use region A as scratch in their chunks: the
  // layout without overlap, two CTAs per SM
  int grid = h->grid, ctas = h->ctas;
  if (nrhs > 1 && a.ov) {
    a.ov = 0;
    grid = h->grid2;
    ctas = 2;
  }
  if (h->profp) {
    CK(prof_begin(h->profp, st));
    CK(launch_solve<T>(a, grid, ctas, st));
    CK(prof_end(h->profp, KKT_K_CG, st));
  } else {
    CK(cudaEventRecord(h->cg_a, st));
    CK(launch_solve<T>(a, grid, ctas, st));
    CK(cudaEventRecord(h->cg_b, st));
  }
  return KKT_OK;
}

static kkt_status residual(kkt_handle h, const double* bx, const double* by, const double* x,
                           const double* y, cudaStream_t st, double* res_x = nullptr, double* res_y = nullptr) {
  ResArgs r;
  r.n = h->P.n; r.m = h->P.m;
  r.Hs_ptr = h->Hs_ptr; r.Hs_col = h->Hs_col; r.Hs_vidx = h->Hs_vidx;
  r.J_rowptr = h->J_rowptr; r.J_colidx = h->J_colidx;
  r.JT_ptr = h->JTo_ptr; r.JT_row = h->JTo_row; r.JT_vidx = h->JTo_vidx;
  r.Hv = h->sv.Hv; r.Jv = h->sv.Jv; r.delta = h->delta;
  r.bx = bx; r.by = by; r.x = x; r.y = y;
  r.res_x = res_x ? res_x : h->res_x; r.res_y = res_y ? res_y : h->res_y;
  r.red = h->red; r.st = h->dst;
  CK(prof_begin(h->profp, st));
  CK(launch_residual(r, st));
  CK(prof_end(h->profp, KKT_K_RESIDUAL, st));
  return KKT_OK;
}

// Flexible GMRES on K_delta [dx; dy] = [r_x; r_y], right-preconditioned by
// the mixed solve M (one persistent solve pass: Schur CG with the FP32
// factor), restarted every kRestart iterations; classical Gram-Schmidt with
// one reorthogonalisation; the small Hessenberg problem by Givens rotations
// on the host. The mixed form's default refinement (opt.refine = 2).
constexpr int kRestart = 20;
constexpr double kInnerRtolMax = 0.5;   // loosest inner CG tolerance of a refinement pass
constexpr double kInnerRtolScale = 2.0; // inner tolerance per unit of the last step's contraction
static_assert(kRestart + 1 <= kMaxKrylov, "basis size");

static kkt_status solve_fgmres(kkt_handle h, const double* rx, const double* ry, double* dx, double* dy,
                               cudaStream_t st) {
  const int64_t n = h->P.n, m = h->P.m, N = n + m;
  if (!h->fV) {
    DevArena& A = h->mem;
    h->fV = A.alloc<double>((size_t)N * (kRestart + 1));
    h->fZ = A.alloc<double>((size_t)N * kRestart);
    h->fw = A.alloc<double>(N); h->fr = A.alloc<double>(N); h->fzero = A.alloc<double>(N);
    h->fpart = A.alloc<double>((size_t)296 * kMaxKrylov);
    h->fdots = A.alloc<double>(kMaxKrylov); h->fcoef = A.alloc<double>(kMaxKrylov);
    h->fgs = A.alloc<double>((size_t)(kRestart + 1) * kRestart + 2 * kRestart + 2 * (kRestart + 1) + 2);
    if (A.failed) { h->fV = nullptr; return KKT_ERR_OOM; }
    if (!h->hflag && cudaMallocHost((void**)&h->hflag, 2 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      h->fV = nullptr;
      return KKT_ERR_OOM;
    }
    CK(cudaMemsetAsync(h->fzero, 0, sizeof(double) * N, st));
  }
  kkt_status s = reset_status(h, st);
  if (s) return s;
  int total_it = 0, brk = 0, applications = 0;
  // The preconditioner's inner CG tolerance follows the outer iteration: an
  // application never needs to be more accurate than the contraction the
  // last FGMRES step achieved (where that is poor, a pass of one S product
  // serves as well as a converged one; where it is strong, passes stay
  // tight).
  double inner_rtol = h->opt.cg_rtol;
  auto apply_M = [&](const double* bx, const double* by, double* ox, double* oy) -> kkt_status {
    kkt_status e = solve_pass<float>(h, bx, by, ox, oy, 0, 0, st, 1, inner_rtol);
    if (e) return e;
    if ((e = read_status(h, st))) return e;
    if (!h->profp) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->cg_a, h->cg_b));
      h->prof.ms[KKT_K_CG] += ms;
      h->prof.n[KKT_K_CG] += 1;
    }
    const DevStatus& d = *h->hst;
    total_it += d.cg_iters;
    brk |= d.breakdown;
    applications++;
    if (d.abort) return KKT_ERR_TIMEOUT;
    if (d.cg_status == 3) return KKT_ERR_CG_BREAKDOWN;
    if (d.cg_status == 4) return KKT_ERR_CG_MAXIT;
    h->hst->cg_iters = 0;
    h->hst->breakdown = 0;
    CK(cudaMemcpyAsync(h->dst, h->hst, sizeof(DevStatus), cudaMemcpyHostToDevice, st));
    return KKT_OK;
  };
  auto true_residual = [&](double& rr, double& rnorm, double& bnorm) -> kkt_status {
    kkt_status e = residual(h, rx, ry, dx, dy, st, h->fr, h->fr + n);
    if (e) return e;
    if ((e = read_status(h, st))) return e;
    rr = h->hst->rr; rnorm = h->hst->res_norm; bnorm = h->hst->b_norm;
    h->info.rr = h->hst->rr;
    h->info.be = h->hst->be;
    return KKT_OK;
  };
  auto finish = [&](kkt_status e) {
    h->info.cg_iters = total_it;
    h->info.ir_steps = applications > 0 ? applications - 1 : 0;
    h->info.delta2_used = brk;
    if (e == KKT_OK) h->inertia_ok = brk ? 0 : 1;
    return e;
  };
  // x0 = M b
  if ((s = apply_M(rx, ry, dx, dy))) return finish(s);
  double rr, rnorm, bnorm;
  if ((s = true_residual(rr, rnorm, bnorm))) return finish(s);
  // Gram-Schmidt coefficients, the Hessenberg column, the rotations and the
  // stop test stay on the device (k_fgmres_coef); the host reads one flag
  // per step, and the preconditioner's status once per application
  const int R = kRestart;
  const double tol = 0.5 * h->opt.ir_rtol * bnorm;
  auto dots_dev = [&](const double* w, const double* V, int cnt) -> cudaError_t {
    return launch_multidot(w, V, N, N, cnt, h->fpart, h->fdots, st);
  };
  while (rr > h->opt.ir_rtol && applications - 1 < h->opt.ir_maxit) {
    // V0 = r / ||r|| (||r|| from the residual's status on the device)
    CK(launch_fgmres_coef(4, 0, R, h->fdots, h->dst, tol, h->fgs, h->fcoef, st));
    CK(launch_lincomb(h->fV, 0.0, h->fr, N, N, 1, h->fcoef, st));
    int k = 0;
    for (; k < kRestart && applications - 1 < h->opt.ir_maxit; k++) {
      double* Vk = h->fV + (size_t)k * N;
      double* Zk = h->fZ + (size_t)k * N;
      if ((s = apply_M(Vk, Vk + n, Zk, Zk + n))) return finish(s);
      // w = -K Z_k (the residual kernel with a zero right-hand side)
      if ((s = residual(h, h->fzero, h->fzero, Zk, Zk + n, st, h->fw, h->fw + n))) return finish(s);
      // u = K Z_k = -w; h_i = (u, V_i) = -(w, V_i); w <- w - sum (w, V_i) V_i (twice)
      CK(dots_dev(h->fw, h->fV, k + 1));
      CK(launch_fgmres_coef(0, k, R, h->fdots, h->dst, tol, h->fgs, h->fcoef, st));
      CK(launch_lincomb(h->fw, 1.0, h->fV, N, N, k + 1, h->fcoef, st));
      CK(dots_dev(h->fw, h->fV, k + 1));
      CK(launch_fgmres_coef(1, k, R, h->fdots, h->dst, tol, h->fgs, h->fcoef, st));
      CK(launch_lincomb(h->fw, 1.0, h->fV, N, N, k + 1, h->fcoef, st));
      CK(dots_dev(h->fw, h->fw, 1));
      // column k of H, rotations, g; coef[0] = -1/||w||: V_{k+1} = u / ||u|| = -w / ||w||
      CK(launch_fgmres_coef(2, k, R, h->fdots, h->dst, tol, h->fgs, h->fcoef, st));
      CK(launch_lincomb(h->fV + (size_t)(k + 1) * N, 0.0, h->fw, N, N, 1, h->fcoef, st));
      CK(cudaMemcpyAsync(h->hflag, h->fgs + (R + 1) * R + 2 * R + 2 * (R + 1), 2 * sizeof(double),
                         cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      inner_rtol = std::min(kInnerRtolMax, std::max(h->opt.cg_rtol, kInnerRtolScale * h->hflag[1]));
      if (h->hflag[0] != 0.0) { k++; break; }
    }
    // y = H^-1 g (upper triangular k x k); x += Z y
    if (k > 0) {
      CK(launch_fgmres_coef(3, k, R, h->fdots, h->dst, tol, h->fgs, h->fcoef, st));
      CK(launch_lincomb(dx, 1.0, h->fZ, N, n, k, h->fcoef, st));
      if (m) CK(launch_lincomb(dy, 1.0, h->fZ + n, N, m, k, h->fcoef, st));
    }
    if ((s = true_residual(rr, rnorm, bnorm))) return finish(s);
    if (k == 0) break;
  }
  return finish(KKT_OK);
}

// ------------------------------------------------ Krylov variants on S
// (opt.krylov = 1: CG preconditioned by M = (J J^T)^-1 J H_gamma J^T
// (J J^T)^-1; 2: MINRES), FP64 handles. The loop runs on the host; every
// vector lives on the device and every product is a device kernel: S p =
// J H^-1 J^T p with H^-1 from the persistent solve kernel (one H^-1
// application per launch), (J J^T)^-1 from the inner handle's.

// J J^T values from the current J and its Cholesky on the inner handle; a
// failure (J rank deficient) leaves the preconditioner off
static kkt_status post_factor(kkt_handle h, cudaStream_t st) {
  if (h->opt.krylov != 1 || !h->jjt) return KKT_OK;
  h->jjt_ok = false;
  CK(launch_jjt_values(h->jjt_ne, h->jjt_pp, h->jjt_pa, h->jjt_pb, h->Jv, h->jjt_vals, st));
  const kkt_status s = kkt_factor(h->jjt, h->jjt_vals, nullptr, 0.0, 0.0, st);
  if (s == KKT_OK) h->jjt_ok = true;
  else if (s != KKT_ERR_NOT_SPD) return s;
  return KKT_OK;
}

static kkt_status hinv(kkt_handle h, const double* b, double* x, cudaStream_t st) {
  return solve_pass<double>(h, b, b, x, x, 0, 1, st);
}

// host copies of cnt inner products <x, V[:, i]> (V columns of length N, ld N)
static kkt_status dots(kkt_handle h, const double* x, const double* V, int64_t N, int cnt, double* out,
                       cudaStream_t st) {
  CK(launch_multidot(x, V, N, N, cnt, h->kpart, h->kdots, st));
  CK(cudaMemcpyAsync(out, h->kdots, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return KKT_OK;
}

// one solve of K_delta [x; y] = [bx; by] through eqs. Schur1/Schur2 with the
// variant's Krylov method; ox, oy receive (accumulate = 0) or gain the result
static kkt_status variant_pass(kkt_handle h, const double* bx, const double* by, double* ox, double* oy,
                               int accumulate, int* iters, int* status, cudaStream_t st) {
  const Plan& P = h->P;
  const int64_t n = P.n, m = P.m;
  const double g = h->gamma, dl = h->delta;
  // workspace: n-vectors rhx, w, t1, t2, t3; m-vectors y, r, z (r and z adjacent), p, q, a, d,
  // v_old, v, w2, w1, wk
  double* rhx = h->kv;
  double* w = rhx + n;
  double* t1 = w + n;
  double* t2 = t1 + n;
  double* t3 = t2 + n;
  double* y = t3 + n;
  double* r = y + m;
  double* z = r + m;
  double* p = z + m;
  double* q = p + m;
  double* a = q + m;
  double* d = a + m;
  double* vo = d + m;
  double* v = vo + m;
  double* w2 = v + m;
  double* w1 = w2 + m;
  double* wk = w1 + m;
  auto jt = [&](const double* yy, double alpha, double beta, double* out) {
    return launch_jt_mult(n, h->JTo_ptr, h->JTo_row, h->JTo_vidx, h->Jv, yy, alpha, beta, out, st);
  };
  auto jm = [&](const double* xx, double alpha, double beta, double* out) {
    return launch_j_mult(m, h->J_rowptr, h->J_colidx, h->Jv, xx, alpha, beta, out, st);
  };
  kkt_status s;
  // r^_x = bx + gamma J^T by, w = H^-1 r^_x, b_S = J w - by (into r)
  CK(launch_axpby(n, 1.0, bx, 0.0, rhx, st));
  CK(jt(by, g, 1.0, rhx));
  if ((s = hinv(h, rhx, w, st))) return s;
  CK(launch_axpby(m, -1.0, by, 0.0, r, st));
  CK(jm(w, 1.0, 1.0, r));
  CK(cudaMemsetAsync(y, 0, sizeof(double) * m, st));
  double dd[2];
  if ((s = dots(h, r, r, m, 1, dd, st))) return s;
  const double nb = std::sqrt(dd[0]);
  const double tol = h->opt.cg_rtol * nb;
  const int maxit = h->opt.cg_maxit;
  int it = 0;
  *status = 0;
  // q = S p
  auto sprod = [&](const double* pp, double* qq) -> kkt_status {
    CK(jt(pp, 1.0, 0.0, t1));
    kkt_status e = hinv(h, t1, t2, st);
    if (e) return e;
    CK(jm(t2, 1.0, 0.0, qq));
    return KKT_OK;
  };
  // zz = M rr = (J J^T)^-1 J H_gamma J^T (J J^T)^-1 rr
  auto mprec = [&](const double* rr, double* zz) -> kkt_status {
    kkt_status e = kkt_hsolve(h->jjt, rr, a, st);
    if (e) return e;
    CK(jt(a, 1.0, 0.0, t1));
    CK(launch_hsym_mult(n, h->Hs_ptr, h->Hs_col, h->Hs_vidx, h->Hv, t1, dl, t3, st));
    CK(jm(t1, 1.0, 0.0, d));
    CK(jt(d, g, 1.0, t3));
    CK(jm(t3, 1.0, 0.0, d));
    return kkt_hsolve(h->jjt, d, zz, st);
  };
  if (nb > 0 && h->opt.krylov == 1) {
    const bool pre = h->jjt_ok;
    if (pre) { if ((s = mprec(r, z))) return s; }
    else CK(launch_axpby(m, 1.0, r, 0.0, z, st));
    CK(launch_axpby(m, 1.0, z, 0.0, p, st));
    if ((s = dots(h, r, z, m, 1, dd, st))) return s;
    double rho = dd[0];
    for (;;) {
      if (it >= maxit) { *status = 4; break; }
      if ((s = sprod(p, q))) return s;
      if ((s = dots(h, p, q, m, 1, dd, st))) return s;
      if (!(dd[0] > 0)) { *status = 3; break; }
      const double al = rho / dd[0];
      CK(launch_axpby(m, al, p, 1.0, y, st));
      CK(launch_axpby(m, -al, q, 1.0, r, st));
      it++;
      if (pre) { if ((s = mprec(r, z))) return s; }
      else CK(launch_axpby(m, 1.0, r, 0.0, z, st));
      if ((s = dots(h, r, r, m, 2, dd, st))) return s;   // r.r and r.z (z follows r)
      if (std::sqrt(dd[0]) <= tol) break;
      const double be = dd[1] / rho;
      rho = dd[1];
      CK(launch_axpby(m, 1.0, z, be, p, st));
    }
  } else if (nb > 0) {
    // MINRES: Lanczos on S from b_S / ||b_S||, Givens QR of the tridiagonal
    CK(cudaMemsetAsync(vo, 0, sizeof(double) * m, st));
    CK(cudaMemsetAsync(w2, 0, sizeof(double) * m, st));
    CK(cudaMemsetAsync(w1, 0, sizeof(double) * m, st));
    CK(launch_axpby(m, 1.0 / nb, r, 0.0, v, st));
    double beta = nb, eta = nb, c_old = 1.0, c = 1.0, s_old = 0.0, sn = 0.0;
    for (;;) {
      if (it >= maxit) { *status = 4; break; }
      if ((s = sprod(v, p))) return s;
      if ((s = dots(h, v, p, m, 1, dd, st))) return s;
      const double al = dd[0];
      CK(launch_axpby(m, -al, v, 1.0, p, st));
      CK(launch_axpby(m, -beta, vo, 1.0, p, st));
      if ((s = dots(h, p, p, m, 1, dd, st))) return s;
      const double bn = std::sqrt(dd[0]);
      const double dlt = c * al - c_old * sn * beta;
      const double r1 = std::hypot(dlt, bn);
      const double r2 = sn * al + c_old * c * beta;
      const double r3 = s_old * beta;
      if (!(r1 > 0)) { *status = 3; break; }
      const double cn = dlt / r1, snn = bn / r1;
      // wk = (v - r3 w2 - r2 w1) / r1
      CK(launch_axpby(m, 1.0 / r1, v, 0.0, wk, st));
      CK(launch_axpby(m, -r3 / r1, w2, 1.0, wk, st));
      CK(launch_axpby(m, -r2 / r1, w1, 1.0, wk, st));
      CK(launch_axpby(m, cn * eta, wk, 1.0, y, st));
      eta = -snn * eta;
      it++;
      if (std::fabs(eta) <= tol || bn == 0.0) break;
      std::swap(vo, v);                                   // v_old <- v
      CK(launch_axpby(m, 1.0 / bn, p, 0.0, v, st));       // v <- p / beta_new
      std::swap(w2, w1);                                  // w2 <- w1
      std::swap(w1, wk);                                  // w1 <- wk
      c_old = c; c = cn; s_old = sn; sn = snn;
      beta = bn;
    }
  }
  *iters = it;
  // x = H^-1 (r^_x - J^T y)
  CK(launch_axpby(n, 1.0, rhx, 0.0, t3, st));
  CK(jt(y, -1.0, 1.0, t3));
  if ((s = hinv(h, t3, t1, st))) return s;
  CK(launch_axpby(n, 1.0, t1, accumulate ? 1.0 : 0.0, ox, st));
  CK(launch_axpby(m, 1.0, y, accumulate ? 1.0 : 0.0, oy, st));
  return KKT_OK;
}

static kkt_status solve_variant(kkt_handle h, const double* rx, const double* ry, double* dx, double* dy,
                                cudaStream_t st) {
  const int64_t n = h->P.n, m = h->P.m;
  h->inertia_ok = 0;
  std::memset(&h->info, 0, sizeof(h->info));
  if (!h->kv) {
    h->kv = h->mem.alloc<double>(5 * (size_t)n + 12 * (size_t)std::max<int64_t>(m, 1));
    h->kpart = h->mem.alloc<double>(296 * (size_t)kMaxKrylov);
    h->kdots = h->mem.alloc<double>(kMaxKrylov);
    if (h->mem.failed) return KKT_ERR_OOM;
  }
  kkt_status s = reset_status(h, st);
  if (s) return s;
  int total = 0;
  for (int pass = 0;; pass++) {
    const double* bx = pass == 0 ? rx : h->res_x;
    const double* by = pass == 0 ? ry : h->res_y;
    int it = 0, cst = 0;
    if ((s = variant_pass(h, bx, by, dx, dy, pass > 0, &it, &cst, st))) return s;
    total += it;
    if ((s = residual(h, rx, ry, dx, dy, st))) return s;
    if ((s = read_status(h, st))) return s;
    const DevStatus& d = *h->hst;
    h->info.cg_iters = total;
    h->info.ir_steps = pass;
    h->info.cg_status = cst;
    h->info.rr = d.rr;
    h->info.be = d.be;
    if (d.abort) return KKT_ERR_TIMEOUT;
    if (cst == 3) return KKT_ERR_CG_BREAKDOWN;
    if (cst == 4) return KKT_ERR_CG_MAXIT;
    if (!(d.rr > h->opt.ir_rtol) || pass >= h->opt.ir_maxit) break;
  }
  h->inertia_ok = 1;
  return KKT_OK;
}

static kkt_status solve_common(kkt_handle h, const double* rx, const double* ry, double* dx, double* dy,
                               cudaStream_t st) {
  if (!h->factored) return KKT_ERR_STATE;
  if (h->opt.krylov != 0) return solve_variant(h, rx, ry, dx, dy, st);
  if (h->opt.precision == KKT_MIXED && h->opt.refine == 2) {
    h->inertia_ok = 0;
    std::memset(&h->info, 0, sizeof(h->info));
    return solve_fgmres(h, rx, ry, dx, dy, st);
  }
  h->inertia_ok = 0;
  std::memset(&h->info, 0, sizeof(h->info));
  const bool f64 = h->opt.precision == KKT_FP64;
  kkt_status s = reset_status(h, st);
  if (s) return s;
  int total_it = 0, brk = 0;
  for (int pass = 0;; pass++) {
    const double* bx = pass == 0 ? rx : h->res_x;
    const double* by = pass == 0 ? ry : h->res_y;
    s = f64 ? solve_pass<double>(h, bx, by, dx, dy, pass > 0, 0, st)
            : solve_pass<float>(h, bx, by, dx, dy, pass > 0, 0, st);
    if (s) return s;
    if ((s = residual(h, rx, ry, dx, dy, st))) return s;
    if ((s = read_status(h, st))) return s;
    if (!h->profp) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->cg_a, h->cg_b));
      h->prof.ms[KKT_K_CG] += ms;
      h->prof.n[KKT_K_CG] += 1;
    }
    const DevStatus& d = *h->hst;
    total_it += d.cg_iters;
    brk |= d.breakdown;
    h->info.cg_iters = total_it;
    h->info.ir_steps = pass;
    h->info.cg_status = d.cg_status;
    h->info.delta2_used = brk;
    h->info.rr = d.rr;
    h->info.be = d.be;
    if (d.abort) return KKT_ERR_TIMEOUT;
    if (d.cg_status == 3) return KKT_ERR_CG_BREAKDOWN;
    if (d.cg_status == 4) return KKT_ERR_CG_MAXIT;
    if (!(d.rr > h->opt.ir_rtol) || pass >= h->opt.ir_maxit) break;
    h->hst->cg_iters = 0;
    h->hst->breakdown = 0;
    CK(cudaMemcpyAsync(h->dst, h->hst, sizeof(DevStatus), cudaMemcpyHostToDevice, st));
  }
  h->inertia_ok = brk ? 0 : 1;
  return KKT_OK;
}

// Up to kMaxRhs right-hand sides in one persistent launch per refinement
// pass: the triangular sweeps stage each L tile once for all of them; CG
// runs independently per right-hand side (its own scalars and stop test).
// Refinement passes continue while any RR(K_delta) > ir_rtol.
static kkt_status solve_group(kkt_handle h, int R, const double* rx, const double* ry, double* dx, double* dy,
                              kkt_info* info, cudaStream_t st) {
  const bool f64 = h->opt.precision == KKT_FP64;
  const int64_t n = h->P.n, m = h->P.m;
  kkt_status s = reset_status(h, st);
  if (s) return s;
  int it_sum[kMaxRhs] = {0}, brk[kMaxRhs] = {0}, cst[kMaxRhs] = {0};
  double rr[kMaxRhs] = {0}, be[kMaxRhs] = {0};
  int32_t stat[3 * kMaxRhs];
  for (int pass = 0;; pass++) {
    const double* bx = pass == 0 ? rx : h->mres_x;
    const double* by = pass == 0 ? ry : h->mres_y;
    s = f64 ? solve_pass<double>(h, bx, by, dx, dy, pass > 0, 0, st, R)
            : solve_pass<float>(h, bx, by, dx, dy, pass > 0, 0, st, R);
    if (s) return s;
    CK(cudaMemcpyAsync(stat, h->rhs_stat, sizeof(int32_t) * 3 * R, cudaMemcpyDeviceToHost, st));
    if ((s = read_status(h, st))) return s;
    if (h->hst->abort) return KKT_ERR_TIMEOUT;
    if (!h->profp) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->cg_a, h->cg_b));
      h->prof.ms[KKT_K_CG] += ms;
      h->prof.n[KKT_K_CG] += 1;
    }
    double worst = 0.0;
    for (int j = 0; j < R; j++) {
      it_sum[j] += stat[3 * j];
      cst[j] = stat[3 * j + 1];
      brk[j] |= stat[3 * j + 2];
      if ((s = residual(h, rx + j * n, ry + j * m, dx + j * n, dy + j * m, st, h->mres_x + j * n,
                        h->mres_y + j * m)))
        return s;
      if ((s = read_status(h, st))) return s;
      rr[j] = h->hst->rr;
      be[j] = h->hst->be;
      worst = std::max(worst, rr[j]);
    }
    for (int j = 0; j < R; j++) {
      info[j].cg_iters = it_sum[j];
      info[j].ir_steps = pass;
      info[j].cg_status = cst[j];
      info[j].delta2_used = brk[j];
      info[j].rr = rr[j];
      info[j].be = be[j];
    }
    for (int j = 0; j < R; j++) {
      if (cst[j] == 3) return KKT_ERR_CG_BREAKDOWN;
      if (cst[j] == 4) return KKT_ERR_CG_MAXIT;
    }
    if (!(worst > h->opt.ir_rtol) || pass >= h->opt.ir_maxit) break;
  }
  return KKT_OK;
}

extern "C" {

// Batched form: nsys systems on the analysed pattern, factored one after
// another with the handle's factorization (its captured graph) and kept in
// per-system slots; each solve copies its system's factor back into the
// working buffers (a few microseconds of device copies) and runs the solve.
}  // extern "C"

// Restores the solve view of the single factor when a batched solve returns.
struct Handle_sv_saver {
  kkt_handle h;
  explicit Handle_sv_saver(kkt_handle hh) : h(hh) {}
  ~Handle_sv_saver() {
    h->sv.L = h->L; h->sv.Linv = h->Linv; h->sv.Hv = h->Hv; h->sv.Jv = h->Jv;
    h->sv.tmaps = h->tmaps; h->sv.tz = 0;
  }
};

// Batch slots for nsys systems: panels, inverses, update matrices, diagonal
// tile scratch and values, system after system, a status per system, and the
// tensor maps over them (third coordinate = system).
static kkt_status batch_reserve(kkt_handle h, int32_t nsys) {
  if (nsys <= h->batch_cap) return KKT_OK;
  const Plan& P = h->P;
  const bool f64 = h->opt.precision == KKT_FP64;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  void* old[] = {h->bL, h->bLinv, h->bHv, h->bJv, h->bU, h->bDsc, h->bst, h->bs_maps, h->bWtc};
  for (void* p : old) cudaFree(p);
  if (h->hbst) cudaFreeHost(h->hbst);
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  h->bL = h->bLinv = h->bU = h->bDsc = nullptr;
  h->bHv = h->bJv = nullptr;
  h->bst = h->hbst = nullptr;
  h->bs_maps = nullptr;
  h->bWtc = nullptr;
  h->bgraph = nullptr;
  h->bgraph_nb = 0;
  h->batch_cap = 0;
  auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
  bool ok = al(&h->bL, es * (size_t)P.panel_total * nsys) && al(&h->bLinv, es * (size_t)P.inv_total * nsys) &&
            al((void**)&h->bHv, sizeof(double) * (size_t)h->nnzH * nsys) &&
            al((void**)&h->bJv, sizeof(double) * (size_t)h->nnzJ * nsys) &&
            al(&h->bU, es * (size_t)P.u_total * nsys) && al(&h->bDsc, es * (size_t)P.dsc_total * nsys) &&
            al((void**)&h->bst, sizeof(DevStatus) * nsys) &&
            (f64 || P.tc_ws_tiles == 0 ||
             al((void**)&h->bWtc, sizeof(float) * (size_t)P.tc_ws_tiles * kTcTileFloats * nsys)) &&
            cudaMallocHost((void**)&h->hbst, sizeof(DevStatus) * nsys) == cudaSuccess;
  if (!ok) { cudaGetLastError(); return KKT_ERR_OOM; }
  std::vector<uint8_t> maps;
  if (!build_tensor_maps(P, h->bL, es, nsys, maps)) return KKT_ERR_CUDA;
  if (!maps.empty()) {
    if (!al((void**)&h->bs_maps, maps.size())) { cudaGetLastError(); return KKT_ERR_OOM; }
    CK(cudaMemcpy(h->bs_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice));
  }
  h->batch_cap = nsys;
  return KKT_OK;
}

// One graph for the whole batch: every factor launch covers all nsys systems
// (system b = blockIdx.y), so the level-by-level launch sequence is paid once.
template <typename T>
static kkt_status batch_graph(kkt_handle h, int32_t nsys) {
  if (h->bgraph && h->bgraph_nb == nsys) return KKT_OK;
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  h->bgraph = nullptr;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = factor_launches<T>(h, h->cap_stream, nullptr, nsys);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e || e2) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return KKT_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&h->bgraph, g, 0);
  cudaGraphDestroy(g);
  if (e) { h->bgraph = nullptr; return cuda_status(e); }
  h->bgraph_nb = nsys;
  return KKT_OK;
}

extern "C" {

kkt_status kkt_factor_batch(kkt_handle h, int32_t nsys, const double* H_vals, const double* J_vals,
                            double delta, double gamma, int32_t* status, void* stream) {
  if (!h || nsys < 1 || nsys > 65535 || !H_vals || (h->nnzJ > 0 && !J_vals)) return KKT_ERR_INVALID;
  if (!h->on_device || h->opt.ruiz_iters > 0 || h->opt.krylov != 0) return KKT_ERR_STATE;
  if (!(delta >= 0.0) || !std::isfinite(delta)) return KKT_ERR_INVALID;
  if (gamma < 0) gamma = h->opt.gamma;
  if (!std::isfinite(gamma)) return KKT_ERR_INVALID;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  kkt_status s = batch_reserve(h, nsys);
  if (s) return s;
  h->bstatus.assign((size_t)nsys, KKT_ERR_STATE);
  CK(cudaMemcpyAsync(h->bHv, H_vals, sizeof(double) * h->nnzH * nsys, cudaMemcpyDeviceToDevice, st));
  if (h->nnzJ) CK(cudaMemcpyAsync(h->bJv, J_vals, sizeof(double) * h->nnzJ * nsys, cudaMemcpyDeviceToDevice, st));
  for (int b = 0; b < nsys; b++) {
    std::memset(&h->hbst[b], 0, sizeof(DevStatus));
    h->hbst[b].fail_col = INT_MAX;
  }
  CK(cudaMemcpyAsync(h->bst, h->hbst, sizeof(DevStatus) * nsys, cudaMemcpyHostToDevice, st));
  h->h_dg[0] = delta;
  h->h_dg[1] = gamma;
  CK(cudaMemcpyAsync(h->d_dg, h->h_dg, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
  if (h->profp) {
    CK(h->opt.precision == KKT_FP64 ? factor_launches<double>(h, st, h->profp, nsys)
                                    : factor_launches<float>(h, st, h->profp, nsys));
  } else {
    s = h->opt.precision == KKT_FP64 ? batch_graph<double>(h, nsys) : batch_graph<float>(h, nsys);
    if (s) return s;
    CK(cudaGraphLaunch(h->bgraph, st));
  }
  CK(cudaMemcpyAsync(h->hbst, h->bst, sizeof(DevStatus) * nsys, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  kkt_status worst = KKT_OK;
  for (int b = 0; b < nsys; b++) {
    const kkt_status sb = h->hbst[b].abort ? KKT_ERR_TIMEOUT
                                           : (h->hbst[b].fail_col != INT_MAX ? KKT_ERR_NOT_SPD : KKT_OK);
    h->bstatus[b] = sb;
    if (status) status[b] = sb;
    if (sb == KKT_ERR_TIMEOUT) worst = KKT_ERR_TIMEOUT;
    else if (sb == KKT_ERR_NOT_SPD && worst == KKT_OK) worst = KKT_ERR_NOT_SPD;
  }
  h->factored = false;   // kkt_solve needs a kkt_factor; the batch is solved with kkt_solve_batch
  h->bdelta = delta;
  h->bgamma = gamma;
  return worst;
}

kkt_status kkt_solve_batch(kkt_handle h, int32_t nsys, const double* r_x, const double* r_y, double* dx,
                           double* dy, kkt_info* info, int32_t* status, void* stream) {
  if (!h || nsys < 1 || !r_x || !dx || (h->P.m > 0 && (!r_y || !dy))) return KKT_ERR_INVALID;
  if (!h->on_device || h->opt.ruiz_iters > 0 || h->opt.krylov != 0) return KKT_ERR_STATE;
  if (nsys > (int32_t)h->bstatus.size()) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->P.n, m = h->P.m;
  const size_t es = h->opt.precision == KKT_FP64 ? sizeof(double) : sizeof(float);
  // helpers: kBatchSolvers concurrent solves, each solve kernel on its share of the SMs
  const int K = std::min<int>(kBatchSolvers, nsys);
  while ((int)h->helpers.size() < K) {
    kkt_options o = h->opt;
    o.solve_sms = std::max(1, 148 / kBatchSolvers);
    o.profile = 0;
    kkt_handle x = nullptr;
    kkt_status s = kkt_analyse_like(h, &o, &x);
    if (s) return s;
    cudaStream_t xs = nullptr;
    if (cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      kkt_destroy(x);
      return KKT_ERR_CUDA;
    }
    h->helpers.push_back(x);
    h->hstreams.push_back(xs);
  }
  CK(cudaStreamSynchronize(st));   // the right-hand sides are written in the caller's stream order
  std::vector<kkt_status> res((size_t)nsys, KKT_OK);
  std::vector<kkt_info> inf((size_t)nsys);
  auto run = [&](int k) {
    kkt_handle x = h->helpers[k];
    cudaSetDevice(h->device);
    x->delta = h->bdelta;
    x->gamma = h->bgamma;
    for (int b = k; b < nsys; b += K) {
      kkt_status s = (kkt_status)h->bstatus[b];
      std::memset(&inf[b], 0, sizeof(kkt_info));
      if (s == KKT_OK) {
        // solve system b where the batch factored it: no copies
        x->sv.L = (char*)h->bL + es * (size_t)h->P.panel_total * b;
        x->sv.Linv = (char*)h->bLinv + es * (size_t)h->P.inv_total * b;
        x->sv.Hv = h->bHv + (int64_t)b * h->nnzH;
        x->sv.Jv = h->bJv + (int64_t)b * h->nnzJ;
        x->sv.tmaps = h->bs_maps;
        x->sv.tz = b;
        x->factored = true;
        s = solve_common(x, r_x + b * n, r_y + b * m, dx + b * n, dy + b * m, h->hstreams[k]);
        x->factored = false;
        inf[b] = x->info;
      }
      res[b] = s;
    }
    { const Handle_sv_saver restore(x); }
  };
  std::vector<std::thread> th;
  for (int k = 1; k < K; k++) th.emplace_back(run, k);
  run(0);
  for (std::thread& t : th) t.join();
  // a bounded wait that ran out while other solves were resident: solve
  // that system again alone (the persistent solve kernel's grid barriers need
  // all of its CTAs on the device at once)
  for (int b = 0; b < nsys; b++) {
    if (res[b] != KKT_ERR_TIMEOUT) continue;
    kkt_handle x = h->helpers[0];
    x->delta = h->bdelta;
    x->gamma = h->bgamma;
    x->sv.L = (char*)h->bL + es * (size_t)h->P.panel_total * b;
    x->sv.Linv = (char*)h->bLinv + es * (size_t)h->P.inv_total * b;
    x->sv.Hv = h->bHv + (int64_t)b * h->nnzH;
    x->sv.Jv = h->bJv + (int64_t)b * h->nnzJ;
    x->sv.tmaps = h->bs_maps;
    x->sv.tz = b;
    x->factored = true;
    res[b] = solve_common(x, r_x + b * n, r_y + b * m, dx + b * n, dy + b * m, h->hstreams[0]);
    x->factored = false;
    inf[b] = x->info;
    const Handle_sv_saver restore(x);
  }
  kkt_status worst = KKT_OK;
  for (int b = 0; b < nsys; b++) {
    if (info) info[b] = inf[b];
    if (status) status[b] = res[b];
    const kkt_status s = res[b];
    if (s == KKT_ERR_CUDA || s == KKT_ERR_TIMEOUT || s == KKT_ERR_OOM) return s;
    if (s != KKT_OK && worst == KKT_OK) worst = s;
  }
  return worst;
}

kkt_status kkt_solve_multi(kkt_handle h, int32_t nrhs, const double* r_x, const double* r_y, double* dx,
                           double* dy, kkt_info* info, void* stream) {
  if (!h || nrhs < 1 || !r_x || !dx || (h->P.m > 0 && (!r_y || !dy))) return KKT_ERR_INVALID;
  if (!h->on_device || h->opt.ruiz_iters > 0 || h->opt.krylov != 0) return KKT_ERR_STATE;
  if (!h->factored) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->P.n, m = h->P.m;
  if (!h->multi) {
    const size_t es = h->opt.precision == KKT_FP64 ? sizeof(double) : sizeof(float);
    DevArena& A = h->mem;
    h->mv = A.alloc<char>(es * (size_t)n * kMaxRhs);
    h->mrhx = A.alloc<double>((size_t)n * kMaxRhs);
    h->mwv = A.alloc<double>((size_t)n * kMaxRhs); h->mxa = A.alloc<double>((size_t)n * kMaxRhs);
    h->mp = A.alloc<double>((size_t)m * kMaxRhs); h->mr = A.alloc<double>((size_t)m * kMaxRhs);
    h->my = A.alloc<double>((size_t)m * kMaxRhs); h->mq = A.alloc<double>((size_t)m * kMaxRhs);
    h->mbS = A.alloc<double>((size_t)m * kMaxRhs);
    h->mres_x = A.alloc<double>((size_t)n * kMaxRhs); h->mres_y = A.alloc<double>((size_t)m * kMaxRhs);
    if (A.failed) return KKT_ERR_OOM;
    h->multi = true;
  }
  h->inertia_ok = 0;
  std::memset(&h->info, 0, sizeof(h->info));
  std::vector<kkt_info> all((size_t)nrhs);
  int brk = 0;
  kkt_status s = KKT_OK;
  for (int g0 = 0; g0 < nrhs && s == KKT_OK; g0 += kMaxRhs) {
    const int R = std::min(kMaxRhs, nrhs - g0);
    s = solve_group(h, R, r_x + g0 * n, r_y + g0 * m, dx + g0 * n, dy + g0 * m, all.data() + g0, st);
  }
  for (int j = 0; j < nrhs; j++) {
    h->info.cg_iters = std::max(h->info.cg_iters, all[j].cg_iters);
    h->info.ir_steps = std::max(h->info.ir_steps, all[j].ir_steps);
    h->info.cg_status = std::max(h->info.cg_status, all[j].cg_status);
    h->info.rr = std::max(h->info.rr, all[j].rr);
    h->info.be = std::max(h->info.be, all[j].be);
    brk |= all[j].delta2_used;
  }
  h->info.delta2_used = brk;
  if (info) std::memcpy(info, all.data(), sizeof(kkt_info) * (size_t)nrhs);
  if (s == KKT_OK) h->inertia_ok = brk ? 0 : 1;
  return s;
}

kkt_status kkt_factor(kkt_handle h, const double* H_vals, const double* J_vals, double delta, double gamma,
                      void* stream) {
  if (!h || !H_vals || (h->nnzJ > 0 && !J_vals)) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpyAsync(h->Hv, H_vals, sizeof(double) * h->nnzH, cudaMemcpyDeviceToDevice, st));
  if (h->nnzJ) CK(cudaMemcpyAsync(h->Jv, J_vals, sizeof(double) * h->nnzJ, cudaMemcpyDeviceToDevice, st));
  kkt_status sc = apply_scaling(h, st);
  if (sc) return sc;
  return factor_common(h, delta, gamma, st);
}

kkt_status kkt_factor_regularized(kkt_handle h, const double* H_vals, const double* J_vals, double gamma,
                                  double delta_min, double delta_max, double* delta_used, void* stream) {
  if (!h || !H_vals || (h->nnzJ > 0 && !J_vals)) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  if (!(delta_min > 0)) delta_min = 1e-9;
  if (!(delta_max > 0)) delta_max = 1e-6;
  if (!std::isfinite(delta_min) || !std::isfinite(delta_max) || delta_max < delta_min) return KKT_ERR_INVALID;
  if (gamma < 0) gamma = h->opt.gamma;
  if (!std::isfinite(gamma)) return KKT_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpyAsync(h->Hv, H_vals, sizeof(double) * h->nnzH, cudaMemcpyDeviceToDevice, st));
  if (h->nnzJ) CK(cudaMemcpyAsync(h->Jv, J_vals, sizeof(double) * h->nnzJ, cudaMemcpyDeviceToDevice, st));
  {
    kkt_status sc = apply_scaling(h, st);
    if (sc) return sc;
  }
  double d1 = 0.0;
  kkt_status s;
  if (h->profp) {
    // profile mode times kernel by kernel, so the loop stays on the host
    s = factor_common(h, d1, gamma, st);
    while (s == KKT_ERR_NOT_SPD && d1 <= delta_max / 2) {
      d1 = d1 == 0.0 ? (h->delta_prev > 0.0 ? h->delta_prev : delta_min) : 2.0 * d1;
      s = factor_common(h, d1, gamma, st);
    }
  } else {
    h->factored = false;
    h->inertia_ok = 0;
    if (!h->reg_graph) {
      s = h->opt.precision == KKT_FP64 ? build_reg_graph<double>(h) : build_reg_graph<float>(h);
      if (s) return s;
    }
    if ((s = reset_status(h, st))) return s;
    double* dg = h->h_dg;
    dg[0] = 0.0; dg[1] = gamma; dg[2] = delta_min; dg[3] = delta_max; dg[4] = h->delta_prev; dg[5] = 0.0;
    CK(cudaMemcpyAsync(h->d_dg, dg, 6 * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaGraphLaunch(h->reg_graph, st));
    CK(cudaMemcpyAsync(dg, h->d_dg, sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((s = read_status(h, st))) return s;   // synchronises the stream
    d1 = dg[0];
    h->delta = d1;
    h->gamma = gamma;
    if (h->hst->abort) s = KKT_ERR_TIMEOUT;
    else if (h->hst->fail_col != INT_MAX) s = KKT_ERR_NOT_SPD;
    else {
      h->factored = true;
      s = post_factor(h, st);
    }
  }
  if (s == KKT_OK) h->delta_prev = d1;
  if (delta_used) *delta_used = d1;
  return s;
}

kkt_status kkt_set_delta_prev(kkt_handle h, double delta_prev) {
  if (!h || !(delta_prev >= 0.0) || !std::isfinite(delta_prev)) return KKT_ERR_INVALID;
  h->delta_prev = delta_prev;
  return KKT_OK;
}

kkt_status kkt_solve(kkt_handle h, const double* r_x, const double* r_y, double* dx, double* dy, void* stream) {
  if (!h || !r_x || !dx || (h->P.m > 0 && (!r_y || !dy))) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  if (h->opt.ruiz_iters <= 0) return solve_common(h, r_x, r_y, dx, dy, (cudaStream_t)stream);
  // scaled handle: solve D K D x^ = D b, then x = D x^
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->P.n, m = h->P.m;
  CK(launch_scale_vec(n, m, h->d_D, r_x, r_y, h->stage_rx, h->stage_ry, st));
  kkt_status s = solve_common(h, h->stage_rx, h->stage_ry, h->stage_dx, h->stage_dy, st);
  CK(launch_scale_vec(n, m, h->d_D, h->stage_dx, h->stage_dy, dx, dy, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

kkt_status kkt_factor_solve_host(kkt_handle h, const double* H_vals, const double* J_vals, double delta,
                                 double gamma, const double* r_x, const double* r_y, double* dx, double* dy,
                                 void* stream) {
  if (!h || !H_vals || !r_x || !dx || (h->P.m > 0 && (!J_vals || !r_y || !dy))) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->P.n, m = h->P.m;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpyAsync(h->Hv, H_vals, sizeof(double) * h->nnzH, cudaMemcpyHostToDevice, st));
  if (h->nnzJ) CK(cudaMemcpyAsync(h->Jv, J_vals, sizeof(double) * h->nnzJ, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->stage_rx, r_x, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (m) CK(cudaMemcpyAsync(h->stage_ry, r_y, sizeof(double) * m, cudaMemcpyHostToDevice, st));
  kkt_status s = apply_scaling(h, st);
  if (s) return s;
  const bool scaled = h->opt.ruiz_iters > 0;
  if (scaled) CK(launch_scale_vec(n, m, h->d_D, h->stage_rx, h->stage_ry, h->stage_rx, h->stage_ry, st));
  s = factor_common(h, delta, gamma, st);
  if (s) return s;
  s = solve_common(h, h->stage_rx, h->stage_ry, h->stage_dx, h->stage_dy, st);
  if (scaled) CK(launch_scale_vec(n, m, h->d_D, h->stage_dx, h->stage_dy, h->stage_dx, h->stage_dy, st));
  CK(cudaMemcpyAsync(dx, h->stage_dx, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  if (m) CK(cudaMemcpyAsync(dy, h->stage_dy, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

kkt_status kkt_hsolve(kkt_handle h, const double* b, double* x, void* stream) {
  if (!h || !b || !x) return KKT_ERR_INVALID;
  if (!h->factored || h->opt.ruiz_iters > 0) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(h->device));
  kkt_status s = reset_status(h, st);
  if (s) return s;
  s = h->opt.precision == KKT_FP64 ? solve_pass<double>(h, b, b, x, x, 0, 1, st)
                                   : solve_pass<float>(h, b, b, x, x, 0, 1, st);
  if (s) return s;
  if ((s = read_status(h, st))) return s;
  return h->hst->abort ? KKT_ERR_TIMEOUT : KKT_OK;
}

kkt_status kkt_get_info(kkt_handle h, kkt_info* info) {
  if (!h || !info) return KKT_ERR_INVALID;
  *info = h->info;
  return KKT_OK;
}

kkt_status kkt_inertia(kkt_handle h, int32_t* ok) {
  if (!h || !ok) return KKT_ERR_INVALID;
  *ok = (h->factored && h->inertia_ok) ? 1 : 0;
  return KKT_OK;
}

kkt_status kkt_symbolic_info_get(kkt_handle h, kkt_symbolic_info* o) {
  if (!h || !o) return KKT_ERR_INVALID;
  std::memset(o, 0, sizeof(*o));
  o->n = h->S.n; o->m = h->S.m; o->nsuper = h->S.ns; o->nnz_l = h->S.nnzL;
  o->panel_entries = h->P.panel_total; o->update_entries = h->P.u_total;
  o->sn_rows_total = (int64_t)h->S.sn_rows.size();
  o->npieces = h->P.npieces; o->nchunks = h->P.nchunks; o->nlevels = h->P.nlevels;
  o->fwd_depth = h->P.fwd_depth; o->bwd_depth = h->P.bwd_depth;
  o->nsub = h->P.nsub; o->nitems = (int64_t)h->P.fwd_items.size();
  o->flops = h->S.flops;
  o->tc_flops = h->P.tc_flops;
  o->device_bytes = (double)h->mem.bytes;
  return KKT_OK;
}

kkt_status kkt_get_symbolic(kkt_handle h, int32_t* amd, int32_t* perm, int32_t* parent, int64_t* colcount,
                            int32_t* sn_start, int64_t* sn_rowptr, int32_t* sn_rows, int32_t* sn_parent) {
  if (!h) return KKT_ERR_INVALID;
  const Symbolic& S = h->S;
  auto cp = [](auto* dst, const auto& v) { if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(v[0]) * v.size()); };
  cp(amd, S.amd); cp(perm, S.perm); cp(parent, S.parent); cp(colcount, S.colcount);
  cp(sn_start, S.sn_start); cp(sn_rowptr, S.sn_rowptr); cp(sn_rows, S.sn_rows); cp(sn_parent, S.sn_parent);
  return KKT_OK;
}

kkt_status kkt_get_profile(kkt_handle h, double* ms, int64_t* launches, int32_t reset) {
  if (!h) return KKT_ERR_INVALID;
  static_assert(KKT_K_SYRK_TC == KKT_K_SYRK_TC_PROF && KKT_K_BLOCK == KKT_K_BLOCK_PROF, "profile slots");
  for (int k = 0; k < KKT_K_COUNT; k++) {
    if (ms) ms[k] = h->prof.ms[k];
    if (launches) launches[k] = h->prof.n[k];
  }
  if (reset) {
    for (int k = 0; k < KKT_K_COUNT; k++) { h->prof.ms[k] = 0; h->prof.n[k] = 0; }
  }
  return KKT_OK;
}

kkt_status kkt_get_scaling(kkt_handle h, double* D) {
  if (!h || !D) return KKT_ERR_INVALID;
  if (!h->on_device || h->opt.ruiz_iters <= 0) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpy(D, h->d_D, sizeof(double) * (size_t)(h->P.n + h->P.m), cudaMemcpyDeviceToHost));
  return KKT_OK;
}

kkt_status kkt_set_profile(kkt_handle h, int32_t on) {
  if (!h) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  if (!on) {
    h->profp = nullptr;
    return KKT_OK;
  }
  CK(cudaSetDevice(h->device));
  if (!h->prof.a) CK(cudaEventCreate(&h->prof.a));
  if (!h->prof.b) CK(cudaEventCreate(&h->prof.b));
  h->profp = &h->prof;
  return KKT_OK;
}

kkt_status kkt_get_solve_counters(kkt_handle h, uint64_t* out, int32_t reset) {
  if (!h || !out) return KKT_ERR_INVALID;
  if (!h->on_device) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpy(out, h->d_instr, 32 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (reset) CK(cudaMemset(h->d_instr, 0, 32 * sizeof(uint64_t)));
  return KKT_OK;
}

kkt_status kkt_get_solve_trace(kkt_handle h, uint64_t* out, int64_t cap) {
  if (!h || !out) return KKT_ERR_INVALID;
  if (!h->on_device || !h->d_trace) return KKT_ERR_STATE;
  const int64_t total = 6 * (int64_t)h->P.fwd_items.size();
  if (cap < total) return KKT_ERR_INVALID;
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpy(out, h->d_trace, (size_t)total * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return KKT_OK;
}

kkt_status kkt_get_solve_item_order(kkt_handle h, int32_t* fwd, int32_t* bwd, int64_t cap) {
  if (!h || !fwd || !bwd) return KKT_ERR_INVALID;
  const int64_t n = (int64_t)h->P.fwd_items.size();
  if (cap < n) return KKT_ERR_INVALID;
  std::copy(h->P.fwd_items.begin(), h->P.fwd_items.end(), fwd);
  std::copy(h->P.bwd_items.begin(), h->P.bwd_items.end(), bwd);
  return KKT_OK;
}

kkt_status kkt_get_factor_panels(kkt_handle h, double* out) {
  if (!h || !out) return KKT_ERR_INVALID;
  if (!h->factored) return KKT_ERR_STATE;
  CK(cudaSetDevice(h->device));
  const size_t cnt = (size_t)h->P.panel_total;
  if (h->opt.precision == KKT_FP64) {
    CK(cudaMemcpy(out, h->L, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(cnt);
    CK(cudaMemcpy(tmp.data(), h->L, sizeof(float) * cnt, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < cnt; i++) out[i] = tmp[i];
  }
  return KKT_OK;
}

}  // extern "C"
