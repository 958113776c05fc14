// Argument blocks passed by value to the KKT kernels, and the host launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "plan.hpp"

namespace kkt {

template <typename T>
struct FacArgs {
  const int32_t *sfirst, *sw, *snr, *sld, *sparent, *rel;
  const int64_t *srow, *poff, *uoff;
  const double *Hv, *Jv;
  T* L;
  T* U;
  T* Dsc;    // factored diagonal tiles of the current level's block steps (kPB x kPB each)
  DevStatus* st;
  float* W = nullptr;   // split operand tiles of the current tensor-core launch (FP32 factor)
  // batched form: system b = blockIdx.y works on these pointers advanced by
  // b times the strides (elements; DevStatus entries for st); 0 for one system
  int64_t bsL = 0, bsU = 0, bsD = 0, bsH = 0, bsJ = 0, bsW = 0;
};

// The view of system blockIdx.y of a batched launch (identity for one system).
template <typename T>
__device__ __forceinline__ void batch_view(FacArgs<T>& a) {
  const int64_t b = blockIdx.y;
  if (b) {
    a.L += b * a.bsL;
    a.U += b * a.bsU;
    a.Dsc += b * a.bsD;
    a.Hv += b * a.bsH;
    a.Jv += b * a.bsJ;
    if (a.W) a.W += b * a.bsW;
    a.st += b;
  }
}

// Optional per-launch timing (profile mode): events around each launch,
// elapsed time accumulated per kernel kind.
constexpr int KKT_K_TC_SPLIT_PROF = 6;   // profile slot of the tensor-core operand split
constexpr int KKT_K_SYRK_TC_PROF = 10;   // profile slot of the tensor-core SYRK
constexpr int KKT_K_BLOCK_PROF = 11;     // profile slot of the fused block step
struct Prof {
  cudaEvent_t a = nullptr, b = nullptr;
  double ms[12] = {0};
  long long n[12] = {0};
};
cudaError_t prof_begin(Prof* pr, cudaStream_t st);
cudaError_t prof_end(Prof* pr, int kind, cudaStream_t st);

struct FacLists {
  const int4 *it_potrf, *it_trsm, *it_pupd, *it_syrk, *it_eadd, *it_syrk_tc, *it_block, *it_syrk128, *it_dstore,
      *it_tc_split;
  const int64_t *slot_pos, *src_ptr;
  const int32_t *srcA, *srcB;
  int64_t nslot, panel_total, u_total;
  const std::vector<Launch>* launches;
};

template <typename T>
struct InvArgs {
  const int32_t *pc_w, *pc_ld, *pc_c;
  const int64_t *pc_colbase, *pc_inv;
  const T* L;
  T* Linv;
  int64_t bsL = 0, bsI = 0;   // batch strides (system blockIdx.y)
};
template <typename T>
cudaError_t launch_tri_inv(const InvArgs<T>& a, int64_t npieces, int max_pw, cudaStream_t st, int nb = 1);

// Tensor-core update tiles (tc_update.cu): items of kTcItem ints
// (Plan::it_syrk_tc), operands split beforehand by launch_tc_split
// (Plan::it_tc_split) into a.W.
cudaError_t launch_tc_split(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb = 1);
cudaError_t launch_tc_update(const int4* items, int64_t cnt, const FacArgs<float>& a, cudaStream_t st, int nb = 1);

template <typename T>
cudaError_t launch_factor(const FacArgs<T>& a, const FacLists& fl, const double* dg, cudaStream_t st,
                          Prof* prof = nullptr, int nb = 1);

// Persistent CG on the Schur complement (plus the two direct solves).
template <typename T>
struct SolveArgs {
  int64_t n, m;
  // solve DAG
  const int32_t* sn_rows;
  const int64_t* pc_inv;                 // packed triangle inverses of the pieces
  const int32_t *hd_tgt, *ch_tgt;        // target pieces of heads' chunk 0 and of chunks
  const int32_t *fwd_items, *bwd_items;
  int64_t nitems, npieces;
  int32_t sw, ent, ent0, max_rows;  // piece width, L entries per chunk / head chunk 0, max chunk rows
  int32_t esub;             // panel entries of a subtree item
  int32_t ov;               // 1: chunk tiles overlap the inverse region (one right-hand side only)
  // small subtrees solved whole by one CTA
  const int32_t *st_first, *st_last, *st_clo, *st_chi, *st_tgt, *sn_piece;
  const int64_t* st_tptr;
  const int32_t *st_lptr, *st_lev, *st_sn;
  const ChunkDesc* cdesc;
  const HeadDesc* hdesc;
  const uint8_t* tmaps;     // one 128-byte tensor map per piece (TMA pieces only)
  int32_t tz;               // the system's coordinate in the maps' third dimension (batched form)
  const int32_t *sfirst, *sw_, *snr, *sld;
  const int64_t *srow, *poff;
  const T* L;
  const T* Linv;
  // J (CSR, permuted column labels) and J^T (by permuted column)
  const int64_t* J_rowptr;
  const int32_t* Jcol_perm;
  const double* Jv;
  const int64_t* JT_ptr;
  const int32_t *JT_row, *JT_vidx;
  const int32_t* perm;
  // right-hand side and outputs (original labels)
  const double *bx, *by;
  double *ox, *oy;
  int32_t accumulate;   // 1: ox += result, oy += result
  int32_t mode;         // 0: full KKT solve; 1: ox = H^-1 bx only
  double gamma, delta2, rtol;
  int32_t maxit;
  // workspace
  // nrhs right-hand sides share every triangular sweep (each staged L tile
  // serves all of them); vector j of each workspace array starts at j times
  // its length (n for v, rhx, bx, ox; m for the CG vectors, by, oy)
  int32_t nrhs;
  int32_t* rhs_stat;   // [kMaxRhs * 3]: CG products, status, delta_2 restart per right-hand side
  T* v;
  double *rhx, *p, *r, *y, *q, *bS;
  double *wv, *xa;     // w = H^-1 r^_x and the accumulated dx (n each)
  int32_t xacc;        // 1: accumulate dx along CG (mixed form); 0: direct solve for dx
  int *fwd_arrive, *fwd_done, *bwd_arrive, *bwd_done;
  int* disp;   // [3]
  int* bar;    // [2]
  double* red; // [grid * kRedStride]
  DevStatus* st;
  long long spin;  // bound of every wait, in clock cycles
  unsigned long long* instr;  // optional per-kernel cycle counters (profile mode), else null
  unsigned long long* trace;  // optional item timeline of the first H^-1 application of each
                              // launch (profile mode): [sweep][item][start ns, end ns, CTA]
};

constexpr int kMaxRhs = 8;                // right-hand sides per solve-kernel launch
constexpr int kMaxKrylov = 24;            // basis vectors of the FGMRES refinement (restart length + 1)

// FP64 vector kernels of the FGMRES refinement (krylov.cu)
cudaError_t launch_multidot(const double* w, const double* V, int64_t ld, int64_t N, int cnt, double* part,
                            double* out, cudaStream_t st);
cudaError_t launch_lincomb(double* y, double alpha, const double* V, int64_t ld, int64_t N, int cnt, const double* c,
                           cudaStream_t st);
constexpr int kRedStride = 2 * kMaxRhs;   // doubles per CTA in the reduction buffer
// FGMRES coefficients, rotations and stop test on the device (krylov.cu);
// gs holds (R+1)R + 2R + 2(R+1) + 1 doubles
cudaError_t launch_fgmres_coef(int mode, int k, int R, const double* dots, const DevStatus* st, double tol, double* gs,
                               double* coef, cudaStream_t s);
// FP64 products of the Krylov variants on S (krylov.cu)
cudaError_t launch_jt_mult(int64_t n, const int64_t* tp, const int32_t* trow, const int32_t* tv, const double* Jv,
                           const double* y, double alpha, double beta, double* out, cudaStream_t st);
cudaError_t launch_j_mult(int64_t m, const int64_t* jp, const int32_t* jc, const double* Jv, const double* x,
                          double alpha, double beta, double* out, cudaStream_t st);
cudaError_t launch_hsym_mult(int64_t n, const int64_t* hp, const int32_t* hc, const int32_t* hv, const double* Hv,
                             const double* x, double delta, double* out, cudaStream_t st);
cudaError_t launch_axpby(int64_t N, double a, const double* x, double b, double* y, cudaStream_t st);
cudaError_t launch_jjt_values(int64_t ne, const int64_t* pp, const int32_t* pa, const int32_t* pb, const double* Jv,
                              double* out, cudaStream_t st);

template <typename T>
cudaError_t launch_solve(const SolveArgs<T>& a, int grid, int ctas, cudaStream_t st);
template <typename T>
int solve_grid_size(int device, int sw, int ent, int ent0, int esub, int max_rows, int ov, int ctas);
size_t solve_smem_bytes(size_t elem, int sw, int ent, int ent0, int esub, int max_rows, int ov);

// FP64 residual of K_delta = [H~ + delta I, J^T; J, 0] (original labels):
// res = b - K x, and norms into DevStatus (rr, be, ...).
struct ResArgs {
  int64_t n, m;
  const int64_t* Hs_ptr;
  const int32_t *Hs_col, *Hs_vidx;
  const int64_t* J_rowptr;
  const int32_t* J_colidx;
  const int64_t* JT_ptr;
  const int32_t *JT_row, *JT_vidx;
  const double *Hv, *Jv;
  double delta;
  const double *bx, *by, *x, *y;
  double *res_x, *res_y;
  double* red;   // scratch [blocks * 4]
  DevStatus* st;
};
cudaError_t launch_residual(const ResArgs& a, cudaStream_t st);

// Symmetrized Ruiz scaling (scale.cu): the pattern of K = [H~, J^T; J, 0] in
// original labels and the values it reads (and scales in place).
struct RuizArgs {
  int64_t n, m;
  const int64_t *Hs_ptr, *H_colptr, *JT_ptr, *J_rowptr;
  const int32_t *Hs_col, *Hs_vidx, *H_rowidx, *JT_row, *JT_vidx, *J_colidx;
  const double *Hv, *Jv;
  const double* ones;   // n + m ones (the initial D)
};
cudaError_t launch_ruiz(const RuizArgs& a, int iters, double* D, double* Dtmp, double* Hv, double* Jv,
                        cudaStream_t st);
cudaError_t launch_scale_vec(int64_t n, int64_t m, const double* D, const double* xx, const double* xy, double* yx,
                             double* yy, cudaStream_t st);

}  // namespace kkt
