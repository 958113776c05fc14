/*
 * kkt.h -- C ABI of the B300 hybrid direct-iterative KKT solver.
 *
 * Method (Regev, Chiang, Darve, Petra, Saunders, Swirydowicz, Peles,
 * "A Hybrid Direct-Iterative Method for Solving KKT Linear Systems"):
 * the 2x2 KKT system (Sec. 3, eq. linsys2x2)
 *
 *     [ H~ + delta I   J^T ] [dx]   [r_x]
 *     [ J              0   ] [dy] = [r_y]
 *
 * is solved through H_gamma = H~ + delta I + gamma J^T J (Sec. 4, eqs.
 * linsys2x2mod and gamma; delta is the delta_1 of Sec. 4.1), its sparse
 * Cholesky factor, and CG on the Schur complement S = J H_gamma^-1 J^T
 * (eqs. Schur1 and Schur2; Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Indices are 0-based. H~ is given by its LOWER triangle (diagonal
 *     included) in CSC form with rows strictly ascending inside each column;
 *     J (m x n) is given in CSR form with columns strictly ascending inside
 *     each row. Entries above the diagonal, out-of-range or repeated indices
 *     make kkt_analyse return KKT_ERR_INVALID.
 *   - "host" pointers are read or written on the host during the call only;
 *     "device" pointers are CUDA device memory on the handle's device and are
 *     read/written in stream order on `stream` (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream). The caller owns every buffer
 *     it passes; the handle owns its own copies of the pattern, the values it
 *     needs after kkt_factor returns, the factor and all workspace.
 *   - Every function returns a kkt_status; none aborts, traps or exits.
 *   - A handle is not thread safe; use one handle per host thread.
 */
#ifndef KKT_H_
#define KKT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kkt_status {
  KKT_OK = 0,
  KKT_ERR_INVALID = 1,       /* bad argument or pattern */
  KKT_ERR_NOT_SPD = 2,       /* Cholesky met a pivot <= 0 or non-finite (Sec. 4.1) */
  KKT_ERR_CG_BREAKDOWN = 3,  /* small quadratic form even after the delta_2 restart */
  KKT_ERR_CG_MAXIT = 4,      /* CG did not reach cg_rtol in cg_maxit products */
  KKT_ERR_OOM = 5,           /* device allocation failed */
  KKT_ERR_CUDA = 6,          /* a CUDA call failed */
  KKT_ERR_TIMEOUT = 7,       /* a bounded wait inside a persistent kernel gave up */
  KKT_ERR_STATE = 8,         /* call out of order (e.g. solve before a successful factor) */
  KKT_ERR_TOO_LARGE = 9      /* n + m exceeds KKT_NOALLOC_MAX_ROWS (kkt_residual_noalloc) */
} kkt_status;

typedef struct kkt_handle_s* kkt_handle;

enum { KKT_FP64 = 0, KKT_MIXED = 1 };

typedef struct kkt_options {
  double gamma;        /* default gamma when kkt_factor gets gamma < 0 (Algorithm 1: 1e4) */
  double delta2;       /* delta_2 of the CG restart on S + delta_2 I (Algorithm 1: 1e-9) */
  double cg_rtol;      /* CG stop: ||r|| <= cg_rtol ||b_S||; <= 0 selects by precision:
                          1e-12 for KKT_FP64 (Sec. 5.1), 3e-3 per refinement pass for
                          KKT_MIXED (the FP32 factor bounds what one pass can reach). With
                          the flexible-GMRES refinement (refine = 2) this is the tightest
                          per-pass tolerance: each pass after an FGMRES step uses
                          min(0.5, max(cg_rtol, 2 x that step's residual contraction)) */
  int32_t cg_maxit;    /* CG product limit (1000) */
  int32_t ir_maxit;    /* refinement passes on K_delta after the first solve; < 0 selects
                          by precision: 3 (KKT_FP64), 10 (KKT_MIXED) */
  double ir_rtol;      /* refine while RR(K_delta) > ir_rtol; <= 0 selects by precision:
                          1e-10 (KKT_FP64), 1e-9 (KKT_MIXED: a tenth of the 1e-8 target, so
                          the pass count does not hinge on rounding noise) */
  int32_t precision;   /* KKT_FP64: FP64 factor and solves; KKT_MIXED: FP32 factor and
                          triangular solves, FP64 CG recurrences, residual and refinement */
  int32_t ordering;    /* 0 = approximate minimum degree (Sec. 5.3), 1 = natural,
                          2 = nested dissection by level-structure separators (Sec. 5.3
                          compares it with AMD; its shallow elimination tree gives the GPU
                          far more parallel work) */
  int32_t relax_small; /* supernode relaxation: merge when merged width <= relax_small */
  int32_t relax_num;   /*   or explicit zeros * relax_den <= relax_num * panel entries */
  int32_t relax_den;
  int32_t relax_wmax;  /*   never beyond this width */
  int32_t solve_w;     /* column width of the triangular-solve pieces, 32..224 (KKT_MIXED) or
                          32..160 (KKT_FP64): a piece's triangle must fit in 200 KB of shared
                          memory; 0 = 128 (KKT_MIXED) / 64 (KKT_FP64) */
  int32_t device;      /* CUDA device ordinal */
  int32_t debug_stall_piece; /* test hook, -1 = off: makes one triangular-solve piece wait for
                                an arrival that never comes, so the bounded wait runs out */
  int64_t spin_cycles; /* limit of every wait on another CTA's flag, in SM clock cycles
                          (0 = default 4e9, about two seconds) */
  int32_t profile;     /* 1: time every kernel launch with CUDA events (serialises the
                          launches; for measurement runs only) */
  int32_t nd_leaf;     /* nested dissection stops at components of at most this many
                          vertices (ordered naturally); default 64 */
  int32_t tensor_cores;/* KKT_MIXED: 1 (default) = fronts with >= 128 update rows and >= 32
                          columns take their update-matrix product (SYRK), and fronts at
                          least tc_panel_min columns wide the in-panel update beyond each
                          128-column outer block, on the tcgen05 tensor cores: operands
                          split once per step into two TF32 parts, three partial products,
                          FP32 accumulation in tensor memory drained every 64 K and summed
                          with round-to-nearest adds; 0 = FP32 FMA units only */
  int32_t solve_ctas;  /* resident solve-kernel CTAs per SM, 2..4 (0 = 3 for KKT_MIXED factors
                          of at least 1e8 panel entries, else 2); the grid is this many per
                          SM or fewer if shared memory does not allow it (kkt_solve_multi
                          runs two per SM) */
  int32_t solve_ent;   /* L entries staged per triangular-solve chunk item, 2048..32768
                          (0 = 8192 for KKT_FP64; KKT_MIXED: 16000 for factors of at least
                          1e8 panel entries, else 16384). Those large KKT_MIXED factors
                          stage a head's first chunk and a subtree's panels in
                          min(solve_ent, 7680) entries and put chunk tiles where the heads'
                          inverses go, so that three solve CTAs fit on an SM */
  int32_t refine;      /* KKT_MIXED refinement on K_delta: 1 = plain passes x += M r;
                          2 = flexible GMRES (restart 20) preconditioned by the mixed
                          solve M: one M application per iteration, like a pass, and it
                          converges where the FP32 factor's error is too large for plain
                          passes (eps_32 kappa(H_gamma) > 1); 0 (default) = 2. ir_maxit
                          bounds the M applications after the first in both modes
                          (< 0: 10 for plain passes, 60 for GMRES) */
  int32_t ruiz_iters;  /* symmetrized Ruiz scaling of K = [H~, J^T; J, 0] before the
                          factorization (Sec. 4.1, so that gamma and delta are judged against
                          the scaled system): 0 (default) = none, k in 1..100 = k iterations
                          of D_i <- D_i / sqrt(max_j D_i |K_ij| D_j) from D = I. The handle
                          then factors and solves D K D (delta, gamma act on it), scales the
                          right-hand side by D and the solution back by D; kkt_info's RR and
                          BE are those of the scaled system. kkt_solve_multi, kkt_hsolve,
                          the batched and the 4x4 forms refuse a scaled handle
                          (KKT_ERR_STATE; the 4x4 analysis: KKT_ERR_INVALID) */
  int32_t krylov;      /* Krylov method on the Schur complement S (Sec. 4, after eqs.
                          Schur1-Schur2): 0 (default) = CG fused into the persistent solve
                          kernel (Algorithm 1); 1 = CG preconditioned by
                          M = (J J^T)^-1 J H_gamma J^T (J J^T)^-1, with J J^T factored by an
                          inner FP64 handle (plain CG if J J^T is not positive definite);
                          2 = MINRES. 1 and 2 need KKT_FP64, run the Krylov loop from the
                          host with device vectors, no delta_2 restart, and are not used by
                          kkt_solve_multi or the batched form (KKT_ERR_STATE) */
  int32_t solve_sms;   /* 0 (default): the persistent solve kernel's grid covers every SM;
                          k >= 1: at most k SMs' worth of its CTAs, so that several handles'
                          solves (one per stream, e.g. the request server's slots) can be
                          resident at once */
  int32_t tc_panel_min;/* narrowest front (columns) whose in-panel updates beyond each
                          128-column outer block run on the tensor cores (tensor_cores = 1):
                          0 = default 128 (every front), else >= 128; narrower fronts keep
                          them on the FMA units */
} kkt_options;

/* Kernel kinds reported by kkt_get_profile. Kinds a plan does not launch
 * stay zero: KKT_MIXED factors with KKT_K_BLOCK (fused POTRF + TRSM) instead
 * of KKT_K_POTRF and KKT_K_TRSM; KKT_K_TC_SPLIT (the TF32 hi/lo split of the
 * operands of each tensor-core launch) and KKT_K_SYRK_TC (the tensor-core
 * tiles) run only in KKT_MIXED with tensor_cores = 1. */
enum {
  KKT_K_ASSEMBLE = 0, KKT_K_POTRF = 1, KKT_K_TRSM = 2, KKT_K_PANEL_UPDATE = 3, KKT_K_SYRK = 4,
  KKT_K_EXTEND_ADD = 5, KKT_K_TC_SPLIT = 6, KKT_K_CG = 7, KKT_K_RESIDUAL = 8, KKT_K_TRI_INV = 9,
  KKT_K_SYRK_TC = 10, KKT_K_BLOCK = 11, KKT_K_COUNT = 12
};

/* Result of the last kkt_solve on a handle. */
typedef struct kkt_info {
  int32_t cg_iters;    /* products with S summed over all refinement passes */
  int32_t ir_steps;    /* refinement passes after the first */
  int32_t cg_status;   /* 0 converged, 3 breakdown, 4 max iterations (last pass) */
  int32_t delta2_used; /* 1 if the delta_2 restart was taken (inertia flag then false) */
  double rr;           /* ||b - K_delta x||_2 / ||b||_2 (Sec. 5.1, RR) */
  double be;           /* ||b - K_delta x||_2 / (||K_delta||_inf ||x||_2 + ||b||_2) (Sec. 5.1, BE) */
} kkt_info;

typedef struct kkt_symbolic_info {
  int64_t n, m;
  int64_t nsuper;      /* supernodes after relaxation */
  int64_t nnz_l;       /* nonzeros of L incl. diagonal (no explicit zeros) */
  int64_t panel_entries;  /* stored panel entries (supernodal storage, incl. zeros) */
  int64_t update_entries; /* multifrontal update-matrix workspace entries */
  int64_t sn_rows_total;  /* sum of supernode row-list lengths */
  int64_t npieces, nchunks;  /* triangular-solve work items */
  int32_t nlevels;     /* height of the supernodal tree */
  int32_t pad;
  double flops;        /* sum_j colcount_j^2 (factor flop count, no explicit zeros) */
  double device_bytes; /* device memory held by the handle */
  int64_t fwd_depth, bwd_depth;  /* longest dependency chains of the two triangular sweeps */
  int64_t nsub;        /* small subtrees solved whole by one CTA */
  int64_t nitems;      /* work items per triangular sweep */
  double tc_flops;     /* flops the factorization runs on the tensor cores (update-matrix
                          products and in-panel updates of the tensor-core fronts, counted
                          as 2 per multiply-add of the FP32 product they stand for) */
} kkt_symbolic_info;

/* Defaults: Algorithm 1's typical parameters (gamma 1e4, delta_2 1e-9), CG
 * tolerance 1e-12 (Sec. 5.1), AMD ordering. */
void kkt_default_options(kkt_options* opt);

/* Ordering and symbolic factorization, once per sparsity pattern (Sec. 2:
 * both are needed only once for the whole sequence; Sec. 5.3: AMD).
 *   n, m       dimensions of H~ (n x n) and J (m x n); n >= 1, m >= 0
 *   H_colptr   host int64[n+1], H_rowidx host int32[H_colptr[n]]
 *   J_rowptr   host int64[m+1], J_colidx host int32[J_rowptr[m]]
 *   opt        host, may be NULL for the defaults
 *   out        receives a new handle (NULL on failure)
 * Allocates all device memory the handle will use. Errors: KKT_ERR_INVALID,
 * KKT_ERR_OOM, KKT_ERR_CUDA. */
kkt_status kkt_analyse(int64_t n, int64_t m, const int64_t* H_colptr, const int32_t* H_rowidx,
                       const int64_t* J_rowptr, const int32_t* J_colidx, const kkt_options* opt,
                       kkt_handle* out);

/* Host-only variant of kkt_analyse: the same ordering, symbolic
 * factorization and numeric plan, but no CUDA call and no device memory.
 * The handle answers kkt_symbolic_info_get, kkt_get_symbolic and
 * kkt_destroy; factor/solve calls on it return KKT_ERR_STATE. */
kkt_status kkt_analyse_host(int64_t n, int64_t m, const int64_t* H_colptr, const int32_t* H_rowidx,
                            const int64_t* J_rowptr, const int32_t* J_colidx, const kkt_options* opt,
                            kkt_handle* out);

/* Numeric factorization L L^T = P (H~ + delta I + gamma J^T J) P^T on the
 * analysed pattern (Sec. 4 eq. gamma, Sec. 4.1 delta_1; Algorithm 1 "Try
 * L L^T = chol(H_delta)").
 *   H_vals  device double[nnz(H~)], in the order of H_rowidx
 *   J_vals  device double[nnz(J)], in the order of J_colidx
 *   delta   diagonal shift (>= 0); gamma >= 0 (gamma < 0 selects opt.gamma)
 * Synchronizes `stream` to read the pivot status. KKT_ERR_NOT_SPD when a
 * pivot is <= 0 or non-finite: the handle stays usable and the caller may
 * retry with a larger delta (the delta_1 loop of Algorithm 1 is the
 * caller's, Sec. 4.2). */
kkt_status kkt_factor(kkt_handle h, const double* H_vals, const double* J_vals, double delta,
                      double gamma, void* stream);

/* Algorithm 1's delta_1 loop around kkt_factor, with the sequence rule of
 * Sec. 4.1: delta_1 = 0 first; while the Cholesky fails (a pivot <= 0,
 * Thm 1: H~ not positive definite on null(J)) and delta_1 <= delta_max / 2,
 * delta_1 becomes, on the first retry, the value this handle accepted for
 * the previous matrix (delta_min if that was 0 or if there was none), and
 * doubles on each later retry (delta_min itself unchanged). A successful
 * call stores its delta_1 as the previous value for the next call; a failed
 * one leaves it. The loop runs on the device as one CUDA graph (a
 * conditional WHILE node around the captured factorization): one launch and
 * one status read per call, whatever the number of trials (profile handles
 * loop on the host instead).
 *   H_vals, J_vals  device, as kkt_factor
 *   gamma           as kkt_factor
 *   delta_min, delta_max  <= 0 selects Algorithm 1's typical 1e-9, 1e-6
 *   delta_used      host double* (may be NULL): the delta_1 of the last trial
 * Returns KKT_OK with the handle factored at delta_used, or KKT_ERR_NOT_SPD
 * when even the largest shift failed (Algorithm 1 then hands the system to
 * an LDL^T solver or back to the optimizer; that is the caller's). */
kkt_status kkt_factor_regularized(kkt_handle h, const double* H_vals, const double* J_vals, double gamma,
                                  double delta_min, double delta_max, double* delta_used, void* stream);

/* Sets the previous matrix's delta_1 that kkt_factor_regularized goes back
 * to (Sec. 4.1); 0 starts a new sequence (a new handle starts at 0).
 * Errors: KKT_ERR_INVALID for a negative or non-finite value. */
kkt_status kkt_set_delta_prev(kkt_handle h, double delta_prev);

/* Solve with the last successful factor (Algorithm 1 solve steps; eqs.
 * Schur1/Schur2), then FP64 refinement on K_delta while RR > ir_rtol
 * (flexible GMRES for KKT_MIXED unless opt.refine = 1 selects plain passes).
 *   r_x, r_y  device double[n], double[m] (may alias nothing written here)
 *   dx, dy    device double[n], double[m] outputs
 * Synchronizes `stream`. Errors: KKT_ERR_STATE (no successful factor),
 * KKT_ERR_CG_BREAKDOWN, KKT_ERR_CG_MAXIT, KKT_ERR_TIMEOUT, KKT_ERR_CUDA.
 * On an error the outputs hold the last iterate. KKT_OK with
 * kkt_info.rr > ir_rtol means the refinement budget (ir_maxit) ran out
 * first: the caller decides whether that residual is acceptable. */
kkt_status kkt_solve(kkt_handle h, const double* r_x, const double* r_y, double* dx, double* dy,
                     void* stream);

/* Several right-hand sides with the last successful factor (one factor
 * with many RHS): right-hand side j is r_x + j n, r_y + j m (device, RHS
 * after RHS), its solution dx + j n, dy + j m. Up to 8 right-hand sides
 * share each persistent solve launch: every triangular sweep stages each L
 * tile once and applies it to all of them, while CG runs independently per
 * right-hand side (own scalars, stop test and delta_2 restart; Algorithm 1
 * per right-hand side); refinement passes continue while any RR > ir_rtol.
 *   nrhs  >= 1
 *   info  host kkt_info[nrhs] (may be NULL): statistics per right-hand side;
 *         kkt_get_info then reports the worst of them
 * The first call allocates the multiple-RHS workspace (8 vectors of each
 * solve vector). Errors as kkt_solve. */
kkt_status kkt_solve_multi(kkt_handle h, int32_t nrhs, const double* r_x, const double* r_y, double* dx,
                           double* dy, kkt_info* info, void* stream);

/* Batched form: nsys systems with the analysed pattern (the symbolic
 * analysis is shared), e.g. the same network at several operating points.
 *   H_vals  device double[nsys * nnz(H~)], system after system
 *   J_vals  device double[nsys * nnz(J)]
 *   status  host int32[nsys] (may be NULL): KKT_OK or KKT_ERR_NOT_SPD per system
 * All systems are factored by one CUDA graph replay: every launch of the
 * factorization covers every system (the system is the launch's second grid
 * coordinate), into per-system slots of panels, inverses and update
 * matrices that the handle allocates (nsys <= 65535; a larger nsys later
 * reallocates them). Returns KKT_ERR_NOT_SPD if any system failed (the
 * others are usable), else the first other error. The single-system factor
 * is not changed: kkt_solve still solves with the last kkt_factor. */
kkt_status kkt_factor_batch(kkt_handle h, int32_t nsys, const double* H_vals, const double* J_vals,
                            double delta, double gamma, int32_t* status, void* stream);

/* Solves system b of the last kkt_factor_batch with right-hand side
 * r_x + b n, r_y + b m (device) into dx + b n, dy + b m, for b < nsys.
 * Up to four systems are solved at once, each by a helper handle made from
 * this analysis (own stream, host thread and workspace; its solve kernel on a
 * quarter of the SMs) that reads the system's factor in its batch slot; the
 * helpers are created by the first call. A system whose solve met
 * KKT_ERR_TIMEOUT while the others ran (the persistent solve kernel needs
 * all its CTAs resident at once) is solved again alone afterwards. The call
 * waits for `stream` first and returns when every solve is done.
 *   info    host kkt_info[nsys] (may be NULL)
 *   status  host int32[nsys] (may be NULL): per-system status (a system whose
 *           factorization failed reports KKT_ERR_NOT_SPD and is skipped)
 * Returns the first per-system error, KKT_OK if none. */
kkt_status kkt_solve_batch(kkt_handle h, int32_t nsys, const double* r_x, const double* r_y, double* dx,
                           double* dy, kkt_info* info, int32_t* status, void* stream);

/* Factor + solve with HOST buffers (copies in and out on `stream`):
 * H_vals/J_vals/r_x/r_y/dx/dy are host arrays of the sizes above. */
kkt_status kkt_factor_solve_host(kkt_handle h, const double* H_vals, const double* J_vals,
                                 double delta, double gamma, const double* r_x, const double* r_y,
                                 double* dx, double* dy, void* stream);

/* x = H_delta^-1 b with the current factor (device double[n] each; the two
 * triangular solves of Algorithm 1). Synchronizes `stream`. */
kkt_status kkt_hsolve(kkt_handle h, const double* b, double* x, void* stream);

/* Statistics of the last kkt_solve (host struct). */
kkt_status kkt_get_info(kkt_handle h, kkt_info* info);

/* 1 when the last factor succeeded and the last solve needed no delta_2
 * restart: then K_delta has inertia (n, m, 0) (Sec. 4.2, Thm 3; Thm 1). */
kkt_status kkt_inertia(kkt_handle h, int32_t* inertia_ok);

/* Sizes of the symbolic analysis and of the device storage (host struct). */
kkt_status kkt_symbolic_info_get(kkt_handle h, kkt_symbolic_info* out);

/* Copies of the symbolic outputs into host arrays (any pointer may be NULL):
 *   amd[n]        ordering before the etree postorder
 *   perm[n]       final permutation, perm[k] = original index at position k
 *   parent[n]     elimination tree in final labels (-1 = root)
 *   colcount[n]   nonzeros of each column of L incl. the diagonal
 *   sn_start[nsuper+1], sn_rowptr[nsuper+1], sn_rows[sn_rows_total],
 *   sn_parent[nsuper]  supernode partition, row lists and tree */
kkt_status kkt_get_symbolic(kkt_handle h, int32_t* amd, int32_t* perm, int32_t* parent,
                            int64_t* colcount, int32_t* sn_start, int64_t* sn_rowptr,
                            int32_t* sn_rows, int32_t* sn_parent);

/* The factor's supernode panels converted to FP64 into host double
 * [panel_entries] (column-major per supernode, ld = its row count rounded
 * up to a multiple of 4; the padding rows are not part of L). */
kkt_status kkt_get_factor_panels(kkt_handle h, double* panels);

/* Accumulated device time (ms) and launch count per kernel kind since the
 * last reset (host arrays of KKT_K_COUNT entries). Every kind is timed for
 * handles created with opt.profile = 1; otherwise only KKT_K_CG is (one
 * event pair around each solve pass, at no cost to the pass). reset != 0
 * clears the counters after reading. */
kkt_status kkt_get_profile(kkt_handle h, double* ms, int64_t* launches, int32_t reset);

/* The Ruiz scaling D = diag(D_x, D_y) of the last factorization (host
 * double[n + m]); KKT_ERR_STATE when the handle does not scale. */
kkt_status kkt_get_scaling(kkt_handle h, double* D);

/* Switches the per-kernel timing of kkt_get_profile on (1) or off (0) on an
 * existing handle, as opt.profile = 1 does at analysis: every launch is
 * bracketed by CUDA events and the factorization runs launch by launch
 * instead of as one graph (for measurement runs only). The item timeline of
 * kkt_get_solve_trace still needs opt.profile = 1 at analysis. */
kkt_status kkt_set_profile(kkt_handle h, int32_t on);

/* A new handle for the same pattern with other options (e.g. the other
 * precision), reusing src's ordering and symbolic factorization (Sec. 2:
 * they depend on the pattern only); only the numeric plan is rebuilt and
 * the device memory allocated. opt.ordering, opt.nd_leaf and the relaxation
 * parameters must equal src's (KKT_ERR_INVALID otherwise). src stays valid.
 * Errors as kkt_analyse. */
kkt_status kkt_analyse_like(kkt_handle src, const kkt_options* opt, kkt_handle* out);

/* Cycle counters of the persistent solve kernel summed over its CTAs (thread
 * 0 of each), for handles created with opt.profile = 1; host uint64_t[32]:
 * [0] item dispatch, [1] dependency waits, [2] bulk-copy waits, [3] whole
 * items, [4] grid barriers, [5] items processed, [6] CTA-launches,
 * [7]/[8] cycles/count of subtree items, [9]/[10] of piece heads,
 * [11]/[12] of row chunks, [13]/[14] cycles in / number of the level
 * loops of subtree items, [15] zero, [16..18] forward piece heads:
 * metadata and copy issue, dependency wait, vector load and copy wait;
 * [19..23] forward chunks: metadata and copy issue, dependency wait, vector
 * load and copy wait, mat-vec, publishing; [24..29] backward piece heads:
 * metadata and copy issue, dependency wait, vector loads and copy wait,
 * chunk-0 product, inverse product, storing and publishing; [30..31]
 * forward piece heads: inverse product and store, chunk-0 product and
 * publishing. */
kkt_status kkt_get_solve_counters(kkt_handle h, uint64_t* out, int32_t reset);

/* Item timeline of the persistent solve kernel, for handles created with
 * opt.profile = 1 (KKT_ERR_STATE otherwise): the forward and the backward
 * sweep of the first H_gamma^-1 application of the last solve-kernel launch.
 * Host uint64_t[6 * nitems] (nitems from kkt_symbolic_info.nitems; cap is
 * the array length, KKT_ERR_INVALID when smaller), laid out
 * [sweep 0 forward / 1 backward][dispatch ticket][3]: the device global
 * timer (ns) when the item was handed out and when it finished, and the CTA
 * that ran it. Entries of an item not run since the handle was created are
 * zero. */
kkt_status kkt_get_solve_trace(kkt_handle h, uint64_t* out, int64_t cap);

/* The two sweeps' dispatch orders (host int32_t[nitems] each, cap their
 * length): entry t is the item handed out at ticket t, coded as a row chunk
 * c >= 0, a piece head -1 - p (p < npieces), or a subtree item
 * -1 - npieces - s. Available after kkt_analyse_host; no device access. */
kkt_status kkt_get_solve_item_order(kkt_handle h, int32_t* fwd, int32_t* bwd, int64_t cap);

kkt_status kkt_destroy(kkt_handle h);

/* ---------------------------------------------------------------------------
 * Residual without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code whose
 * device memory belongs to another allocator (a framework's caching pool, an
 * application with a fixed memory budget), code running where allocating is
 * forbidden, or code that must not risk the device synchronisation that
 * cudaMalloc/cudaFree can cause. Every other entry point allocates in
 * kkt_analyse; this one allocates nothing.
 *
 * Computes res = b - K_delta [dx; dy] for K_delta = [H~ + delta I, J^T; J, 0]
 * and norms[0] = RR = ||res||_2/||b||_2, norms[1] = BE =
 * ||res||_2/(||K_delta||_inf ||[dx;dy]||_2 + ||b||_2), norms[2] = ||res||_2,
 * norms[3] = ||K_delta||_inf (the quantities of Sec. 5.1).
 *   H_colptr/H_rowidx/H_vals  device, H~ lower triangle (CSC, as for kkt_analyse)
 *   J_rowptr/J_colidx/J_vals  device, J (CSR); may be NULL when m == 0
 *   r_x, r_y, dx, dy          device inputs; res_x[n], res_y[m] device outputs
 *   norms                     device double[4] output
 * The work is queued on `stream`; the call does not synchronise.
 * Scratch: a fixed device array of (KKT_NOALLOC_MAX_ROWS + 1184) doubles
 * (about 8 MiB) that every GPU loading the library holds until the process
 * exits. n + m > KKT_NOALLOC_MAX_ROWS returns KKT_ERR_TOO_LARGE without
 * launching anything. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. Later calls look the address up again unless `stream` is
 * capturing, so a device reset between calls (which may reload the library's
 * module at another address) is picked up. The caller checks the arrays'
 * lengths and that they live on the current device: the kernels trust them.
 * All calls share the array and each clears what it needs,
 * so calls whose work overlaps on the GPU (different streams, different host
 * threads) race: serialise them. The residual accumulates with device
 * atomics, so its last bits may differ from run to run. */
#define KKT_NOALLOC_MAX_ROWS (1 << 20)
kkt_status kkt_residual_noalloc(int64_t n, int64_t m, const int64_t* H_colptr, const int32_t* H_rowidx,
                                const double* H_vals, const int64_t* J_rowptr, const int32_t* J_colidx,
                                const double* J_vals, double delta, const double* r_x, const double* r_y,
                                const double* dx, const double* dy, double* res_x, double* res_y,
                                double* norms, void* stream);

const char* kkt_status_string(kkt_status s);

/* ---------------------------------------------------------------------------
 * Request server: continuous batching of KKT solves over resident patterns.
 * The paper's method is a sequence of interior iterations on one sparsity
 * pattern (Sec. 2: analysis once, then value refactorizations and solves);
 * the server holds several patterns' analyses and, per pattern, "slots" --
 * handles with their factor storage and workspace resident on the device --
 * and runs the requests that arrive (one value refactorization + solve each)
 * as slots and device memory free up. Admission is by an HBM budget: a
 * request starts as soon as its pattern has an idle slot, or a new slot fits
 * the budget; the pending list is scanned in arrival order and a request
 * that cannot start does not block later ones of other patterns. Up to
 * max_inflight requests run at once, each on its slot's own CUDA stream and
 * host worker thread, so their kernels overlap on the device. Results do not
 * depend on what else runs (each slot is a separate handle). The persistent
 * solve kernel needs all of its CTAs resident at once (give the server's
 * options a solve_sms of about 148 / max_inflight); should one of its bounded
 * waits run out while other requests' kernels hold the device, the request
 * is run again with nothing else in flight (kkt_request_info.retried).
 * ------------------------------------------------------------------------ */
typedef struct kkt_server_s* kkt_server;

typedef struct kkt_request_info {
  int32_t status;      /* kkt_status of the factor + solve */
  int32_t pattern, slot;
  int32_t cg_iters, ir_steps;
  int32_t retried;     /* 1 if a bounded wait ran out while other requests were on the
                          device and the request was run again alone */
  double rr, be;       /* as kkt_info */
  double t_submit, t_start, t_end;  /* seconds on the server's clock (steady, from its creation) */
} kkt_request_info;

typedef struct kkt_server_stats {
  int64_t submitted, completed, failed;
  int64_t bytes_used, bytes_peak, budget;  /* device bytes of the slots (estimated before a
                                              slot's first solve allocates its refinement
                                              workspace, exact after) */
  int32_t patterns, slots, inflight, peak_inflight, waiting, pad;
} kkt_server_stats;

/* budget_bytes: device memory the slots may hold (<= 0: 90 % of the free
 * memory at creation); max_inflight: requests run at once (>= 1); opt: the
 * options of every slot (NULL: defaults), opt->device the GPU. */
kkt_status kkt_server_create(int64_t budget_bytes, int32_t max_inflight, const kkt_options* opt,
                             kkt_server* out);
/* Analyses a pattern (host, as kkt_analyse_host) and creates its first
 * slot; *pattern_id receives its index. KKT_ERR_OOM when that slot does not
 * fit the budget. Patterns as for kkt_analyse (host arrays). */
kkt_status kkt_server_add_pattern(kkt_server s, int64_t n, int64_t m, const int64_t* H_colptr,
                                  const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                                  int32_t* pattern_id);
/* Queues one request: factor H_vals/J_vals (delta, gamma) on a slot of the
 * pattern, then solve r_x, r_y into dx, dy. All six are DEVICE arrays of the
 * pattern's sizes that must stay valid (inputs unchanged) until the request
 * completes. Returns at once with *request_id. */
kkt_status kkt_server_submit(kkt_server s, int32_t pattern_id, const double* H_vals, const double* J_vals,
                             double delta, double gamma, const double* r_x, const double* r_y, double* dx,
                             double* dy, int64_t* request_id);
/* Blocks until the request completes and returns its record (once per id;
 * the id is then forgotten). The request's own status is in info->status. */
kkt_status kkt_server_wait(kkt_server s, int64_t request_id, kkt_request_info* info);
kkt_status kkt_server_get_stats(kkt_server s, kkt_server_stats* out);
/* Waits for every queued request, then releases all slots and patterns. */
kkt_status kkt_server_destroy(kkt_server s);

/* ------------------------------------------------------------------------
 * The 4x4 form (Sec. 3, eq. linsys4x4):
 *
 *   [ H + D_x   0     J^T   J_d^T ] [dx ]   [r~_x]
 *   [ 0         D_s   0     -I    ] [ds ]   [r_s ]
 *   [ J         0     0     0     ] [dy ] = [r_y ]
 *   [ J_d       -I    0     0     ] [dyd]   [r_yd]
 *
 * reduced to the 2x2 form by eliminating ds = J_d dx - r_yd and
 * dy_d = D_s ds - r_s (Sec. 3, eq. linsys2x2): H~ = H + D_x + J_d^T D_s J_d,
 * r_x = r~_x + J_d^T (D_s r_yd + r_s). The 2x2 system is then solved as
 * above (delta and gamma act on H~) and ds, dy_d are recovered from dx.
 * Shapes: H n_x x n_x (lower CSC, as H~ above; the diagonal may be absent),
 * J m_c x n_x and J_d m_d x n_x (CSR, columns strictly ascending in a row).
 * ------------------------------------------------------------------------ */
typedef struct kkt_handle4_s* kkt_handle4;

/* Pattern of H~ = pat(H) U pat(J_d^T J_d) U diag, then kkt_analyse on it.
 *   H_colptr host int64[n_x+1], H_rowidx host int32[H_colptr[n_x]]
 *   J_rowptr host int64[m_c+1], J_colidx host int32[J_rowptr[m_c]]
 *   Jd_rowptr host int64[m_d+1], Jd_colidx host int32[Jd_rowptr[m_d]]
 * Errors: KKT_ERR_INVALID (bad pattern), KKT_ERR_OOM, KKT_ERR_CUDA. */
kkt_status kkt_analyse_4x4(int64_t n_x, int64_t m_c, int64_t m_d, const int64_t* H_colptr,
                           const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                           const int64_t* Jd_rowptr, const int32_t* Jd_colidx, const kkt_options* opt,
                           kkt_handle4* out);

/* Host-only variant (no CUDA call; the inner handle is a kkt_analyse_host
 * handle): for the pattern and the symbolic analysis. */
kkt_status kkt_analyse_4x4_host(int64_t n_x, int64_t m_c, int64_t m_d, const int64_t* H_colptr,
                                const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                                const int64_t* Jd_rowptr, const int32_t* Jd_colidx, const kkt_options* opt,
                                kkt_handle4* out);

/* The 2x2 handle inside (owned by h): for kkt_get_info, kkt_inertia,
 * kkt_symbolic_info_get, kkt_get_symbolic. NULL for a NULL h. */
kkt_handle kkt_4x4_inner(kkt_handle4 h);

/* The lower CSC pattern of H~ into host arrays (any pointer may be NULL):
 * *nnz, colptr[n_x+1], rowidx[*nnz]. */
kkt_status kkt_get_4x4_pattern(kkt_handle4 h, int64_t* nnz, int64_t* colptr, int32_t* rowidx);

/* Forms H~ on the device and factors H~ + delta I + gamma J^T J.
 *   H_vals device double[nnz(H)], D_x device double[n_x],
 *   Jd_vals device double[nnz(J_d)], D_s device double[m_d] (D_s > 0),
 *   J_vals device double[nnz(J)]
 * J_d and D_s are copied into the handle for kkt_solve_4x4. Errors as
 * kkt_factor. */
kkt_status kkt_factor_4x4(kkt_handle4 h, const double* H_vals, const double* D_x, const double* Jd_vals,
                          const double* D_s, const double* J_vals, double delta, double gamma,
                          void* stream);

/* Solves eq. linsys4x4 with the last factor: device inputs r~_x[n_x],
 * r_s[m_d], r_y[m_c], r_yd[m_d]; device outputs dx[n_x], ds[m_d], dy[m_c],
 * dyd[m_d]. kkt_get_info(kkt_4x4_inner(h)) then reports the 2x2 solve
 * (its RR and BE are those of the reduced system). Errors as kkt_solve; on
 * KKT_ERR_CG_MAXIT / KKT_ERR_CG_BREAKDOWN ds and dyd are still recovered
 * from the last iterate. */
kkt_status kkt_solve_4x4(kkt_handle4 h, const double* r_xt, const double* r_s, const double* r_y,
                         const double* r_yd, double* dx, double* ds, double* dy, double* dyd, void* stream);

/* Releases the 4x4 handle and its inner 2x2 handle. */
kkt_status kkt_destroy_4x4(kkt_handle4 h);

#ifdef __cplusplus
}
#endif
#endif /* KKT_H_ */
