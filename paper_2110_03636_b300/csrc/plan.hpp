// Numeric plan: everything the device kernels need that depends only on the
// sparsity pattern, built once on the host after the symbolic analysis and
// copied to the device once (Sec. 2: the pattern is fixed over the sequence).
#pragma once
#include <cstdint>
#include <vector>

#include "symbolic.hpp"

namespace kkt {

// Everything a triangular-solve work item needs about its piece, packed so
// the solve kernel fetches it in one round trip (16-byte aligned vectors).
struct alignas(16) ChunkDesc {
  int32_t p, r0, nr, pw;        // piece, first row (piece-local), rows, piece width
  int32_t f, ld, c, k;          // piece's first column, panel ld, column offset in the supernode, chunk index
  int64_t colbase, rowbase;     // piece's first L entry; sn_rows index of the chunk's first row
  int64_t tp0, tp1;             // target pieces [tp0, tp1) in ch_tgt
  int32_t cs, tma;              // tile column stride in shared memory; 1 = one 2-D TMA box (else per column)
};
struct alignas(16) HeadDesc {
  int32_t pw, f, rn, need;      // width, first column, rows of chunk 0, arrivals expected per sweep
  int32_t c, ld, nch, cs;       // column offset in the supernode, panel ld, row chunks after chunk 0,
                                // chunk-0 tile column stride in shared memory
  int64_t colbase, rowbase;     // first L entry; sn_rows index of the piece's first row
  int64_t inv0, inv1;           // packed inverse [inv0, inv1) in Linv
  int64_t tp0, tp1;             // chunk-0 target pieces [tp0, tp1) in hd_tgt
  int32_t tma, pad;             // 1 = chunk 0 is one 2-D TMA box
};

// Pieces at least this wide stage their row tiles with one 2-D TMA box
// (rows x piece width, at most kTmaRows rows + 4 for the 16-byte start
// alignment); narrower pieces copy column by column.
constexpr int kTmaMinWidth = 32;
constexpr int kTmaRows = 252;

}  // namespace kkt

namespace kkt {

// Tile constants shared by the planner and the kernels.
constexpr int kPB = 32;      // panel column block of the front factorization
constexpr int kTR = 128;     // rows per TRSM item
constexpr int kUR = 64;      // rows per in-panel update item (x kPB columns)
constexpr int kST = 64;      // SYRK tile edge
constexpr int kEC = 32;      // columns per extend-add item
// Ints per block-step / in-panel-update item: (s, a, b, 0), (w, nr, ld,
// first column), (panel offset low, high, 0, 0) -- three int4 loads that
// do not depend on one another.
constexpr int kFItem = 12;

struct Launch {              // one batched kernel launch of the factorization
  int32_t kind;              // 0 potrf (diagonal tile), 1 trsm, 2 in-panel update, 3 syrk,
                             // 4 extend-add, 6 tensor-core tiles, 7 fused block step,
                             // 8 128 x 128 FP32 syrk, 9 diagonal-tile store,
                             // 10 operand split of the next tensor-core launch
  int32_t kb;                // column block (kinds 0-2)
  int64_t off, cnt;          // range in the item array of that kind
};

struct Plan {
  int64_t n = 0, m = 0, ns = 0;
  // supernodes
  std::vector<int32_t> sfirst, sw, snr;     // first column, width, rows
  std::vector<int32_t> sld;                 // panel leading dimension = snr rounded up to 4
  std::vector<int64_t> srow;                // offset of the row list in sn_rows
  std::vector<int64_t> poff;                // panel offset (column-major, ld = sld; multiple of 4)
  std::vector<int64_t> uoff;                // update-matrix offset (rb x rb, ld = rb)
  std::vector<int32_t> sparent;
  std::vector<int32_t> rel;                 // per sn_rows slot: position of a child's below
                                            // row inside the parent's row list
  int64_t panel_total = 0, u_total = 0;   // (dsc_total below)
  int32_t nlevels = 0;
  // factor work lists (items are int4: s, a, b, 0)
  std::vector<int32_t> it_potrf;            // (s) fronts whose column block kb is factored
  std::vector<int32_t> it_trsm;             // (s, row tile) pairs
  std::vector<int32_t> it_pupd;             // (s, row tile, col tile) triples (kFItem ints each)
  std::vector<int32_t> it_syrk;             // (s, ti, tj) triples, 64 x 64 tiles
  std::vector<int32_t> it_syrk_tc;          // tensor-core update tiles (128 rows x 256 columns), kTcItem
                                            // ints each: (A operand tile lo, hi, B operand tile lo, hi),
                                            // (chunks, mode, panel row of A, panel row of B), (ld, rows,
                                            // width, B has a second row block), (output offset lo, hi, 0, 0)
  std::vector<int32_t> it_tc_split;         // operand splits before each tensor-core launch, kTcItem
                                            // ints each: (ld, rows, first row, K begin), (K end, first
                                            // chunk, end chunk, 0), (panel offset lo, hi, first operand
                                            // tile lo, hi), 0 x 4
  int64_t tc_ws_tiles = 0;                  // operand tiles of the largest tensor-core launch
  double tc_flops = 0;                      // algorithmic flops of the tensor-core tiles per factorization
  std::vector<int32_t> it_block;            // (s, row tile, slot) per fused block step (kFItem ints each)
  std::vector<int32_t> it_syrk128;          // (s, ti, tj), 128 x 128 FP32 register-tiled SYRK
  std::vector<int32_t> it_dstore;           // (s, kb, slot): factored diagonal tile -> panel, per level
  int64_t dsc_total = 0;                    // entries of the diagonal-tile scratch (largest level)
  std::vector<int32_t> it_eadd;             // (child s, col tile) pairs, at the parent's level
  std::vector<Launch> launches;
  // assembly gather: panel slot <- sum of sources (H entry, delta, J pair)
  std::vector<int64_t> slot_pos;            // panel position of each slot
  std::vector<int64_t> src_ptr;             // [nslot+1]
  std::vector<int32_t> srcA, srcB;          // srcB == -1: H entry srcA; -2: delta; else J pair
  // J in permuted labels and its transpose (for J^T p without atomics)
  std::vector<int32_t> Jcol_perm;           // iperm of J's column indices
  std::vector<int64_t> JT_ptr;              // [n+1] by permuted column
  std::vector<int32_t> JT_row, JT_vidx;     // J row and index into J values
  // symmetric H~ (full, original labels) for the FP64 residual
  std::vector<int64_t> Hs_ptr;
  std::vector<int32_t> Hs_col, Hs_vidx;
  // J^T in original labels (residual)
  std::vector<int64_t> JTo_ptr;
  std::vector<int32_t> JTo_row, JTo_vidx;
  // solve DAG over column pieces of width <= solve_w. A piece's "head" applies
  // the inverse of its diagonal triangle and its first rc0 rows below ("chunk
  // 0"); the remaining rows form separate chunks of at most rc rows.
  int32_t solve_w = 128;
  int32_t ent = 16384, ent0 = 8192;         // L entries per chunk item / per head's chunk 0
  int32_t esub = 16384;                     // panel entries per subtree item
  int32_t solve_ov = 0;                     // chunk tiles overlap the inverse region (see solve.cu)
  int32_t max_rows = 1024;                  // rows of any chunk (gathered-vector limit)
  int64_t npieces = 0, nchunks = 0;
  std::vector<int32_t> pc_first, pc_w, pc_nr, pc_ld; // piece: first column, width, rows from its first row, ld
  std::vector<int32_t> pc_c;                // the piece's first row/column inside its supernode
  std::vector<int32_t> pc_rc0;              // rows of the fused chunk 0
  std::vector<int64_t> pc_row;              // offset in sn_rows of the piece's first row
  std::vector<int64_t> pc_colbase;          // panel offset of (supernode row 0, piece column 0)
  std::vector<int64_t> pc_inv;              // offset of the packed inverse of its triangle
  std::vector<int32_t> pc_nchunk;           // separate chunks
  std::vector<int32_t> pc_need;             // heads + chunks whose rows hit the piece (forward)
  std::vector<int64_t> hd_tptr;             // targets of each head's chunk 0
  std::vector<int32_t> hd_tgt;
  std::vector<int32_t> ch_piece, ch_r0, ch_nr, ch_k;  // chunk: piece, first row (piece-local), rows, index
  std::vector<int64_t> ch_tptr;             // targets of each chunk (distinct pieces)
  std::vector<int32_t> ch_tgt;
  // small subtrees solved whole by one CTA: supernodes [st_first, st_last]
  // (postorder ranges), their column range [st_clo, st_chi), and the pieces
  // outside the subtree that their rows hit
  int64_t nsub = 0;
  std::vector<int32_t> st_first, st_last, st_clo, st_chi;
  std::vector<int64_t> st_tptr;
  std::vector<int32_t> st_tgt;
  // supernodes of each subtree item grouped by height above its leaves:
  // item t's level boundaries are st_lev[st_lptr[t] .. st_lptr[t+1]) (offsets
  // into st_sn); supernodes of one level are independent of each other
  std::vector<int32_t> st_lptr, st_lev, st_sn;
  std::vector<ChunkDesc> cdesc;             // per chunk
  std::vector<HeadDesc> hdesc;              // per piece
  std::vector<int32_t> pc_box;              // per piece: TMA box rows (0 = per-column copies)
  std::vector<int32_t> sn_piece;            // first piece of each supernode
  std::vector<int32_t> fwd_items, bwd_items; // >= 0 chunk id; -1-p head of piece p (p < npieces);
                                            // -1-npieces-t subtree t
  int64_t inv_total = 0;
  int64_t fwd_depth = 0, bwd_depth = 0;     // longest dependency chains of the sweeps
  int32_t max_pw = 0;
};

// Rows of the packed inverse of a pw-wide triangle: column k holds rows
// k..pw-1, padded to a multiple of 4.
inline int64_t packed_inv_size(int64_t pw) {
  int64_t t = 0;
  for (int64_t k = 0; k < pw; k++) t += (pw - k + 3) & ~3;
  return t;
}

// tc_syrk: fronts with rb >= kTcMinRows and at least kTcMinWidth columns get
// 128 x 256 tensor-core SYRK tiles; the persistent kernel runs at most
// kTcGrid CTAs (one per SM). Before each tensor-core launch a split launch
// writes the launch's operands, rows [r0, rows) x K [K begin, K end) of each
// front, as operand tiles (kTcTileFloats floats each, in the layout the MMA
// reads) into a workspace of tc_ws_tiles tiles; a tile item names its A and
// B operand tiles and carries its front's geometry (kTcItem ints)
constexpr int kTcMinRows = 128;
constexpr int kTcPB = 128;        // outer column block of the tensor-core in-panel update
constexpr int kTcPanelMinWidth = 128;    // narrowest front that takes it (default of opt.tc_panel_min)
constexpr int kTcMinWidth = 32;
constexpr int kTcItem = 16;
constexpr int kTcK = 16;                      // K columns of one operand tile
constexpr int kTcTileFloats = 2 * 128 * kTcK; // one operand tile: TF32 hi and lo parts of 128 rows x kTcK
constexpr int kTcSplitChunks = 32;            // operand tiles of one row block per split item
constexpr int kTcGrid = 148;
// f32 (FP32 factor): fronts with rb >= kBigRows get 128 x 128 register-tiled SYRK
// tiles, and each block step fuses POTRF into the TRSM launch
constexpr int kBigRows = 128;
int build_plan(const Symbolic& S, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
               const int32_t* Ji, int32_t solve_w, int32_t ent, int32_t ent0, int32_t esub, int32_t ov,
               bool tc_syrk, bool f32, int32_t tc_panel_min, Plan& P);

}  // namespace kkt
