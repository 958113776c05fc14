#include "plan.hpp"

#include <algorithm>
#include <array>
#include <numeric>

namespace kkt {

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int build_plan(const Symbolic& S, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
               const int32_t* Ji, int32_t solve_w, int32_t ent, int32_t ent0, int32_t esub, int32_t ov,
               bool tc_syrk, bool f32, int32_t tc_panel_min, Plan& P) {
  P = Plan();
  const int64_t n = S.n, m = S.m, ns = S.ns;
  P.n = n; P.m = m; P.ns = ns;
  P.sfirst.resize(ns); P.sw.resize(ns); P.snr.resize(ns); P.sld.resize(ns); P.srow.resize(ns);
  P.poff.resize(ns); P.uoff.resize(ns); P.sparent = S.sn_parent;
  std::vector<int32_t> col2sn(n);
  int64_t po = 0, uo = 0;
  for (int64_t s = 0; s < ns; s++) {
    P.sfirst[s] = S.sn_start[s];
    P.sw[s] = S.sn_start[s + 1] - S.sn_start[s];
    P.snr[s] = (int32_t)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]);
    P.sld[s] = (P.snr[s] + 3) & ~3;
    P.srow[s] = S.sn_rowptr[s];
    P.poff[s] = po;
    po += (int64_t)P.sw[s] * P.sld[s];
    for (int32_t j = S.sn_start[s]; j < S.sn_start[s + 1]; j++) col2sn[j] = (int32_t)s;
  }
  P.panel_total = po;
  (void)uo;
  // relative indices of each child's below rows in its parent's row list
  P.rel.assign(S.sn_rows.size(), -1);
  for (int64_t s = 0; s < ns; s++) {
    const int32_t p = P.sparent[s];
    if (p < 0) continue;
    const int32_t* R = S.sn_rows.data() + P.srow[p];
    int64_t q = 0;
    for (int64_t k = P.sw[s]; k < P.snr[s]; k++) {
      const int32_t r = S.sn_rows[P.srow[s] + k];
      while (q < P.snr[p] && R[q] < r) q++;
      if (q >= P.snr[p] || R[q] != r) return 2;   // structure violated (cannot happen)
      P.rel[P.srow[s] + k] = (int32_t)q;
    }
  }
  std::vector<int64_t> kid_ptr(ns + 1, 0);
  std::vector<int32_t> kids;
  for (int64_t s = 0; s < ns; s++) if (P.sparent[s] >= 0) kid_ptr[P.sparent[s] + 1]++;
  for (int64_t s = 0; s < ns; s++) kid_ptr[s + 1] += kid_ptr[s];
  kids.resize(kid_ptr[ns]);
  {
    std::vector<int64_t> fill(kid_ptr.begin(), kid_ptr.end() - 1);
    for (int64_t s = 0; s < ns; s++) if (P.sparent[s] >= 0) kids[fill[P.sparent[s]]++] = (int32_t)s;
  }
  auto children_of = [&](int32_t p) {
    return std::vector<int32_t>(kids.begin() + kid_ptr[p], kids.begin() + kid_ptr[p + 1]);
  };
  // levels: as late as possible -- every front one level below its parent
  // (level = tree height - 1 - depth), so an update matrix lives for two
  // levels only and side subtrees run next to the long chains
  std::vector<int32_t> depth(ns, 0);
  for (int64_t s = ns - 1; s >= 0; s--)            // parents have larger indices
    depth[s] = P.sparent[s] >= 0 ? depth[P.sparent[s]] + 1 : 0;
  const int32_t height = ns ? *std::max_element(depth.begin(), depth.end()) + 1 : 0;
  std::vector<int32_t> level(ns, 0);
  for (int64_t s = 0; s < ns; s++) level[s] = height - 1 - depth[s];
  P.nlevels = height;
  std::vector<std::vector<int32_t>> bylev(P.nlevels);
  for (int64_t s = 0; s < ns; s++) bylev[level[s]].push_back((int32_t)s);
  // Update matrix U_s lives from s's level (cleared, children added, SYRK)
  // to its parent's level (extend-add). First-fit placement of these
  // intervals in one workspace, in order of start level.
  {
    struct Blk { int64_t off, size; int32_t end; };
    std::vector<Blk> live;                  // sorted by offset
    int64_t top = 0;
    for (int32_t L = 0; L < P.nlevels; L++) {
      live.erase(std::remove_if(live.begin(), live.end(), [&](const Blk& b) { return b.end < L; }), live.end());
      for (int32_t s : bylev[L]) {
        const int64_t rb = P.snr[s] - P.sw[s];
        const int64_t size = rb * rb;
        if (size == 0) { P.uoff[s] = 0; continue; }
        const int32_t end = P.sparent[s] >= 0 ? level[P.sparent[s]] : L;
        int64_t off = 0;
        size_t pos = 0;
        for (; pos < live.size(); pos++) {
          if (live[pos].off - off >= size) break;
          off = std::max(off, live[pos].off + live[pos].size);
        }
        live.insert(live.begin() + pos, Blk{off, size, end});
        P.uoff[s] = off;
        top = std::max(top, off + size);
      }
    }
    P.u_total = top;
  }
  // block-step and in-panel-update items carry their front's width, rows,
  // leading dimension, first column and panel offset, so their kernels reach
  // the panel after one load instead of two dependent ones
  // Tensor-core launches. tc_region: the split items of rows [r0, rows) x K
  // [klo, khi) of front sn, as operand tiles from ws on (row block by row
  // block, nch chunks each); returns the region's first tile. tc_item: the
  // tile C = A B^T of panel rows ra and rb of that region.
  int64_t ws = 0;
  auto lo32 = [](int64_t v) { return (int32_t)(uint32_t)(v & 0xffffffff); };
  auto hi32 = [](int64_t v) { return (int32_t)(v >> 32); };
  auto tc_region = [&](int32_t sn, int32_t r0, int32_t klo, int32_t khi) {
    const int64_t nrb = cdiv(P.snr[sn] - r0, 128), nch = cdiv(khi - klo, kTcK), base = ws;
    const int64_t po = P.poff[sn];
    for (int64_t rbi = 0; rbi < nrb; rbi++)
      for (int64_t c0 = 0; c0 < nch; c0 += kTcSplitChunks) {
        const int64_t dst = base + rbi * nch + c0;
        P.it_tc_split.insert(P.it_tc_split.end(),
                             {P.sld[sn], P.snr[sn], r0 + (int32_t)rbi * 128, klo, khi, (int32_t)c0,
                              (int32_t)std::min(nch, c0 + kTcSplitChunks), 0, lo32(po), hi32(po), lo32(dst),
                              hi32(dst), 0, 0, 0, 0});
      }
    ws += nrb * nch;
    return base;
  };
  // tc_item: the 128 x 256 tile of rows ra.. and the columns of row blocks
  // rb.. and rb + 128.. of that region (the second only if the front has it)
  auto tc_item = [&](int32_t sn, int32_t ra, int32_t rb, int32_t r0, int64_t base, int32_t klo, int32_t khi,
                     int32_t mode) {
    const int64_t nch = cdiv(khi - klo, kTcK);
    const int64_t ta = base + (ra - r0) / 128 * nch, tb = base + (rb - r0) / 128 * nch;
    const int64_t out = mode ? P.poff[sn] : P.uoff[sn];
    const int32_t two = rb + 128 < P.snr[sn] ? 1 : 0;
    P.it_syrk_tc.insert(P.it_syrk_tc.end(), {lo32(ta), hi32(ta), lo32(tb), hi32(tb), (int32_t)nch, mode, ra, rb,
                                             P.sld[sn], P.snr[sn], P.sw[sn], two, lo32(out), hi32(out), 0, 0});
  };
  // the split launch (kind 10) and the tile launch (kind 6) of the items
  // added since (o10, o6)
  auto tc_launch = [&](int32_t kb, int64_t o10, int64_t o6) {
    const int64_t c10 = (int64_t)P.it_tc_split.size() / kTcItem - o10;
    const int64_t c6 = (int64_t)P.it_syrk_tc.size() / kTcItem - o6;
    if (c6) {
      P.launches.push_back({10, kb, o10, c10});
      P.launches.push_back({6, kb, o6, c6});
    }
    P.tc_ws_tiles = std::max(P.tc_ws_tiles, ws);
    ws = 0;
  };
  // fronts at least tc_panel_min wide take the in-panel update beyond each
  // outer block on the tensor cores (the default, 128, is every front that
  // has columns beyond its first outer block)
  auto tc_panel = [&](int32_t sn) { return tc_syrk && P.sw[sn] >= tc_panel_min; };
  auto push_fitem = [&](std::vector<int32_t>& v, int32_t sn, int32_t x, int32_t y) {
    const int64_t po = P.poff[sn];
    v.insert(v.end(), {sn, x, y, 0, P.sw[sn], P.snr[sn], P.sld[sn], P.sfirst[sn],
                       (int32_t)(uint32_t)(po & 0xffffffff), (int32_t)(po >> 32), 0, 0});
  };
  for (int32_t L = 0; L < P.nlevels; L++) {
    const auto& F = bylev[L];
    // the children's update matrices split by column: columns landing in a
    // parent's panel are added before its block steps, columns landing in
    // its update matrix after its SYRK (which stores U = -L21 L21^T, so no
    // clearing pass is needed)
    std::vector<std::array<int32_t, 3>> ecols_u;   // (child, first column, end) of the U part
    const int64_t o3 = (int64_t)P.it_eadd.size() / 4;
    for (int32_t p : F)
      for (int32_t c : children_of(p)) {
        const int32_t rb = P.snr[c] - P.sw[c];
        const int32_t* relc = P.rel.data() + P.srow[c] + P.sw[c];
        int32_t split = 0;
        while (split < rb && relc[split] < P.sw[p]) split++;
        for (int32_t j = 0; j < split; j += kEC) P.it_eadd.insert(P.it_eadd.end(), {c, j, split, 0});
        if (split < rb) ecols_u.push_back({c, split, rb});
      }
    const int64_t c3 = (int64_t)P.it_eadd.size() / 4 - o3;
    if (c3) P.launches.push_back({4, 0, o3, c3});
    int32_t wmax = 0;
    for (int32_t s : F) wmax = std::max(wmax, P.sw[s]);
    // per 32-column block step: one fused POTRF + TRSM launch (every front
    // with columns left gets its row tiles below the block, at least one
    // item; every item factors the block's diagonal tile itself, tile 0
    // keeps the result in a per-level scratch slot, and one launch after the
    // level's last step stores the tiles into the panels, since a panel
    // write during the step would race with the other tiles' reads of A),
    // then the right-looking update of the later panel columns. FP64
    // fronts (f32 off) keep separate POTRF and TRSM launches: the
    // fused kernel's register footprint costs more than the launch it saves.
    int32_t slot = 0;
    const int64_t od = (int64_t)P.it_dstore.size() / 4;
    for (int32_t kb = 0; kb * kPB < wmax; kb++) {
      const int64_t ob = (int64_t)P.it_block.size() / kFItem;
      const int64_t opo = (int64_t)P.it_potrf.size() / 4, otr = (int64_t)P.it_trsm.size() / 4;
      for (int32_t s : F) {
        const int32_t c0 = kb * kPB;
        if (c0 >= P.sw[s]) continue;
        const int32_t bw = std::min(kPB, P.sw[s] - c0);
        const int64_t below = P.snr[s] - c0 - bw;
        const int64_t nt = std::max<int64_t>(1, cdiv(below, kTR));
        if (f32) {
          for (int64_t t = 0; t < nt; t++) push_fitem(P.it_block, s, (int32_t)t, slot);
          P.it_dstore.insert(P.it_dstore.end(), {s, kb, slot, 0});
          slot++;
        } else {
          P.it_potrf.insert(P.it_potrf.end(), {s, 0, 0, 0});
          for (int64_t t = 0; t < cdiv(below, kTR); t++) P.it_trsm.insert(P.it_trsm.end(), {s, (int32_t)t, 0, 0});
        }
      }
      const int64_t cb = (int64_t)P.it_block.size() / kFItem - ob;
      if (cb) P.launches.push_back({7, kb, ob, cb});
      const int64_t cpo = (int64_t)P.it_potrf.size() / 4 - opo, ctr = (int64_t)P.it_trsm.size() / 4 - otr;
      if (cpo) P.launches.push_back({0, kb, opo, cpo});
      if (ctr) P.launches.push_back({1, kb, otr, ctr});
      // right-looking update of the panel columns after the block; fronts
      // on the tensor-core path update only the columns of their current
      // kTcPB-column outer block here, and the columns beyond it once per
      // outer block (below)
      const int64_t o1 = (int64_t)P.it_pupd.size() / kFItem;
      for (int32_t s : F) {
        const int32_t c0 = kb * kPB;
        if (c0 >= P.sw[s]) continue;
        const int32_t bw = std::min(kPB, P.sw[s] - c0);
        const int32_t jstart = c0 + bw;
        const int32_t jend = tc_panel(s) ? std::min(P.sw[s], (c0 / kTcPB + 1) * kTcPB) : P.sw[s];
        for (int32_t ct = 0; jstart + ct * kPB < jend; ct++) {
          const int32_t cstart = jstart + ct * kPB;
          const int64_t nrt = cdiv(P.snr[s] - cstart, kUR);
          for (int64_t rt = 0; rt < nrt; rt++) push_fitem(P.it_pupd, s, (int32_t)rt, ct);
        }
      }
      const int64_t c1 = (int64_t)P.it_pupd.size() / kFItem - o1;
      if (c1) P.launches.push_back({2, kb, o1, c1});
      // end of an outer block: the columns beyond it -= L[rows, block] L[cols, block]^T,
      // K = the block's kTcPB columns, on the tensor cores (mode 1)
      if ((kb + 1) * kPB % kTcPB == 0) {
        const int64_t o6 = (int64_t)P.it_syrk_tc.size() / kTcItem, o10 = (int64_t)P.it_tc_split.size() / kTcItem;
        const int32_t oe = (kb + 1) * kPB;          // first column after the outer block
        for (int32_t s : F) {
          if (!tc_panel(s) || oe >= P.sw[s]) continue;
          const int64_t base = tc_region(s, oe, oe - kTcPB, oe);
          for (int32_t cs = oe; cs < P.sw[s]; cs += 256)
            for (int32_t rs = cs; rs < P.snr[s]; rs += 128) tc_item(s, rs, cs, oe, base, oe - kTcPB, oe, 1);
          // lower trapezoid of rows [oe, nr) x columns [oe, w), K = kTcPB
          const double cols = P.sw[s] - oe, top = P.snr[s] - oe;
          P.tc_flops += 2.0 * kTcPB * (cols * top - cols * (cols - 1) / 2);
        }
        tc_launch(kb, o10, o6);
      }
    }
    P.dsc_total = std::max(P.dsc_total, (int64_t)slot * kPB * kPB);
    const int64_t cd = (int64_t)P.it_dstore.size() / 4 - od;
    if (cd) P.launches.push_back({9, 0, od, cd});
    const int64_t o2 = (int64_t)P.it_syrk.size() / 4, o6 = (int64_t)P.it_syrk_tc.size() / kTcItem,
                  o8 = (int64_t)P.it_syrk128.size() / 4, o10 = (int64_t)P.it_tc_split.size() / kTcItem;
    // tensor-core tiles of the level's fronts, widest (longest K) first, so
    // the persistent kernel's round-robin hands every CTA a similar share
    std::vector<int32_t> tcf;
    for (int32_t s : F) {
      const int64_t rb = P.snr[s] - P.sw[s];
      const bool tcs = tc_syrk && rb >= kTcMinRows && P.sw[s] >= kTcMinWidth;
      if (tcs) { tcf.push_back(s); continue; }
      const bool big = f32 && rb >= kBigRows;
      const int64_t tile = big ? 128 : kST;
      const int64_t nt = cdiv(rb, tile);
      auto& list = big ? P.it_syrk128 : P.it_syrk;
      for (int64_t ti = 0; ti < nt; ti++)
        for (int64_t tj = 0; tj <= ti; tj++) list.insert(list.end(), {s, (int32_t)ti, (int32_t)tj, 0});
    }
    std::stable_sort(tcf.begin(), tcf.end(), [&](int32_t x, int32_t y) { return P.sw[x] > P.sw[y]; });
    for (int32_t s : tcf) {
      const int32_t w = P.sw[s];
      const int64_t nt = cdiv(P.snr[s] - w, 128);
      const double rbd = P.snr[s] - w;
      P.tc_flops += (double)w * rbd * (rbd + 1);   // U = -L21 L21^T, lower triangle
      const int64_t base = tc_region(s, w, 0, w);
      for (int64_t ti = 0; ti < nt; ti++)
        for (int64_t tj = 0; tj <= ti; tj += 2)
          tc_item(s, w + (int32_t)ti * 128, w + (int32_t)tj * 128, w, base, 0, w, 0);
    }
    const int64_t c2 = (int64_t)P.it_syrk.size() / 4 - o2, c8 = (int64_t)P.it_syrk128.size() / 4 - o8;
    tc_launch(0, o10, o6);
    if (c8) P.launches.push_back({8, 0, o8, c8});
    if (c2) P.launches.push_back({3, 0, o2, c2});
    const int64_t o4 = (int64_t)P.it_eadd.size() / 4;
    for (const auto& e : ecols_u)
      for (int32_t j = e[1]; j < e[2]; j += kEC) P.it_eadd.insert(P.it_eadd.end(), {e[0], j, e[2], 0});
    const int64_t c4 = (int64_t)P.it_eadd.size() / 4 - o4;
    if (c4) P.launches.push_back({4, 0, o4, c4});
  }
  // ---------------------------------------------------------- assembly map
  // slot of (row, col) in final labels (row >= col)
  auto slot_of = [&](int32_t r, int32_t c) -> int64_t {
    const int32_t s = col2sn[c];
    const int32_t* R = S.sn_rows.data() + P.srow[s];
    const int32_t* pos = std::lower_bound(R, R + P.snr[s], r);
    if (pos == R + P.snr[s] || *pos != r) return (int64_t)-1;   // not in the structure
    return P.poff[s] + (int64_t)(c - P.sfirst[s]) * P.sld[s] + (pos - R);
  };
  struct Src { int64_t slot; int32_t a, b; };
  std::vector<Src> src;
  src.reserve((size_t)Hp[n] + n);
  for (int64_t j = 0; j < n; j++)
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
      int32_t a = S.iperm[Hi[q]], b = S.iperm[j];
      if (a < b) std::swap(a, b);
      src.push_back({slot_of(a, b), (int32_t)q, -1});
    }
  for (int64_t j = 0; j < n; j++) src.push_back({slot_of(j, j), 0, -2});
  for (int64_t r = 0; r < m; r++)
    for (int64_t q1 = Jp[r]; q1 < Jp[r + 1]; q1++)
      for (int64_t q2 = q1; q2 < Jp[r + 1]; q2++) {
        int32_t a = S.iperm[Ji[q1]], b = S.iperm[Ji[q2]];
        if (a < b) std::swap(a, b);
        src.push_back({slot_of(a, b), (int32_t)q1, (int32_t)q2});
      }
  for (const Src& x : src)
    if (x.slot < 0) return 3;
  std::stable_sort(src.begin(), src.end(), [](const Src& x, const Src& y) { return x.slot < y.slot; });
  for (size_t t = 0; t < src.size(); t++) {
    if (t == 0 || src[t].slot != src[t - 1].slot) {
      P.slot_pos.push_back(src[t].slot);
      P.src_ptr.push_back((int64_t)t);
    }
    P.srcA.push_back(src[t].a);
    P.srcB.push_back(src[t].b);
  }
  P.src_ptr.push_back((int64_t)src.size());
  // ---------------------------------------------------------- J / J^T maps
  const int64_t nnzJ = m > 0 ? Jp[m] : 0;
  P.Jcol_perm.resize(nnzJ);
  for (int64_t q = 0; q < nnzJ; q++) P.Jcol_perm[q] = S.iperm[Ji[q]];
  auto transpose = [&](bool permuted, std::vector<int64_t>& tp, std::vector<int32_t>& trow, std::vector<int32_t>& tv) {
    tp.assign(n + 1, 0);
    for (int64_t q = 0; q < nnzJ; q++) tp[(permuted ? P.Jcol_perm[q] : Ji[q]) + 1]++;
    for (int64_t i = 0; i < n; i++) tp[i + 1] += tp[i];
    std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
    trow.resize(nnzJ); tv.resize(nnzJ);
    for (int64_t r = 0; r < m; r++)
      for (int64_t q = Jp[r]; q < Jp[r + 1]; q++) {
        const int64_t c = permuted ? P.Jcol_perm[q] : Ji[q];
        trow[fill[c]] = (int32_t)r;
        tv[fill[c]] = (int32_t)q;
        fill[c]++;
      }
  };
  transpose(true, P.JT_ptr, P.JT_row, P.JT_vidx);
  transpose(false, P.JTo_ptr, P.JTo_row, P.JTo_vidx);
  // symmetric H~ in original labels
  P.Hs_ptr.assign(n + 1, 0);
  for (int64_t j = 0; j < n; j++)
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
      P.Hs_ptr[Hi[q] + 1]++;
      if (Hi[q] != j) P.Hs_ptr[j + 1]++;
    }
  for (int64_t i = 0; i < n; i++) P.Hs_ptr[i + 1] += P.Hs_ptr[i];
  {
    std::vector<int64_t> fill(P.Hs_ptr.begin(), P.Hs_ptr.end() - 1);
    P.Hs_col.resize(P.Hs_ptr[n]); P.Hs_vidx.resize(P.Hs_ptr[n]);
    for (int64_t j = 0; j < n; j++)
      for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
        const int32_t i = Hi[q];
        P.Hs_col[fill[i]] = (int32_t)j; P.Hs_vidx[fill[i]++] = (int32_t)q;
        if (i != j) { P.Hs_col[fill[j]] = i; P.Hs_vidx[fill[j]++] = (int32_t)q; }
      }
  }
  // ---------------------------------------------------------- small subtrees
  // Maximal subtrees with at most kSubCols columns and kSubEntries panel
  // entries; supernode indices are a postorder, so a subtree is the index
  // range [root - size + 1, root].
  // The solve kernel stages a subtree's panels (stored entries, ld
  // included) into its row-tile region of esub entries and the inverses of
  // its triangles into the inverse region of one solve_w-wide piece (their
  // sum over <= solve_w columns never exceeds that piece's).
  const int64_t kSubCols = std::min<int64_t>(128, solve_w), kSubEntries = esub;
  std::vector<int64_t> sub_cols(ns, 0), sub_ent(ns, 0), sub_size(ns, 1);
  for (int64_t s = 0; s < ns; s++) {
    sub_cols[s] += P.sw[s];
    sub_ent[s] += (int64_t)P.sw[s] * P.sld[s];
    const int32_t p = P.sparent[s];
    if (p >= 0) { sub_cols[p] += sub_cols[s]; sub_ent[p] += sub_ent[s]; sub_size[p] += sub_size[s]; }
  }
  auto small_sub = [&](int64_t s) { return sub_cols[s] <= kSubCols && sub_ent[s] <= kSubEntries; };
  // maximal small subtrees, as supernode ranges in postorder
  std::vector<std::pair<int64_t, int64_t>> subs;
  for (int64_t s = 0; s < ns; s++) {
    if (!small_sub(s)) continue;
    const int32_t p = P.sparent[s];
    if (p >= 0 && small_sub(p)) continue;          // not maximal: the parent's subtree covers it
    subs.push_back({s - sub_size[s] + 1, s});
  }
  // bundle runs of adjacent subtrees (siblings are adjacent in postorder)
  // into one item while it stays within the same column/entry limits; rows
  // of a supernode inside the bundle's column range belong to its own subtree
  std::vector<int32_t> in_sub(ns, -1);
  for (size_t k = 0; k < subs.size();) {
    int64_t first = subs[k].first, last = subs[k].second;
    int64_t cols = sub_cols[last], ent = sub_ent[last];
    size_t q = k + 1;
    while (q < subs.size() && subs[q].first == last + 1 && cols + sub_cols[subs[q].second] <= kSubCols &&
           ent + sub_ent[subs[q].second] <= kSubEntries) {
      last = subs[q].second;
      cols += sub_cols[last];
      ent += sub_ent[last];
      q++;
    }
    const int32_t t = (int32_t)P.st_first.size();
    for (int64_t x = first; x <= last; x++) in_sub[x] = t;
    P.st_first.push_back((int32_t)first);
    P.st_last.push_back((int32_t)last);
    P.st_clo.push_back(P.sfirst[first]);
    P.st_chi.push_back(P.sfirst[last] + P.sw[last]);
    k = q;
  }
  P.nsub = (int64_t)P.st_first.size();
  {
    std::vector<int32_t> lvl(ns, 0);
    P.st_lptr.assign(1, 0);
    for (int64_t t = 0; t < P.nsub; t++) {
      const int32_t first = P.st_first[t], last = P.st_last[t];
      int32_t top = 0;
      for (int32_t s = first; s <= last; s++) lvl[s] = 0;
      for (int32_t s = first; s <= last; s++) {       // postorder: children before parents
        const int32_t p = P.sparent[s];
        if (p >= first && p <= last) lvl[p] = std::max(lvl[p], lvl[s] + 1);
        top = std::max(top, lvl[s]);
      }
      for (int32_t L = 0; L <= top; L++) {
        P.st_lev.push_back((int32_t)P.st_sn.size());
        for (int32_t s = first; s <= last; s++)
          if (lvl[s] == L) P.st_sn.push_back(s);
      }
      P.st_lev.push_back((int32_t)P.st_sn.size());
      P.st_lptr.push_back((int32_t)P.st_lev.size());
    }
  }
  // ---------------------------------------------------------- solve DAG
  P.solve_w = solve_w;
  P.ent = ent;
  P.ent0 = ent0;
  P.esub = esub;
  P.solve_ov = ov;
  // rows of an item holding at most e entries of a pw-wide piece: a multiple
  // of 4 (so the staged column segments stay 16-byte aligned) in [4, max_rows]
  auto rows_for = [&](int32_t e, int32_t pw) {
    int32_t r = e / std::max(pw, 1);
    r = std::min(r, P.max_rows);
    r &= ~3;
    return std::max(r, 4);
  };
  std::vector<int32_t> col2piece(n);
  for (int64_t s = 0; s < ns; s++) {
    for (int32_t c = 0; c < P.sw[s]; c += solve_w) {
      const int32_t pw = std::min(solve_w, P.sw[s] - c);
      const int32_t pid = (int32_t)P.pc_first.size();
      P.pc_first.push_back(P.sfirst[s] + c);
      P.pc_w.push_back(pw);
      P.pc_nr.push_back(P.snr[s] - c);
      P.pc_ld.push_back(P.sld[s]);
      P.pc_c.push_back(c);
      P.pc_row.push_back(P.srow[s] + c);
      P.pc_colbase.push_back(P.poff[s] + (int64_t)c * P.sld[s]);
      P.pc_inv.push_back(P.inv_total);
      P.inv_total += packed_inv_size(pw);
      for (int32_t j = 0; j < pw; j++) col2piece[P.sfirst[s] + c + j] = pid;
      if (c == 0) P.sn_piece.push_back(pid);
    }
  }
  P.npieces = (int64_t)P.pc_first.size();
  P.pc_inv.push_back(P.inv_total);               // [npieces + 1]: sizes by difference
  // the solve kernel's per-warp subtree scratch (8 x 160 entries) lives in
  // its gathered-vector region of max_rows + 256 entries
  if (P.max_rows + 256 < 8 * 160) return 2;
  // each subtree's staged ranges fit the solve kernel's tile regions
  for (int64_t t = 0; t < P.nsub; t++) {
    const int32_t s0 = P.st_first[t], s1 = P.st_last[t];
    const int64_t pe = P.poff[s1] + (int64_t)P.sw[s1] * P.sld[s1] - P.poff[s0];
    const int64_t ie = P.pc_inv[P.sn_piece[s1] + 1] - P.pc_inv[P.sn_piece[s0]];
    if (pe > esub || ie > packed_inv_size(solve_w) || P.sn_piece[s1] - P.sn_piece[s0] != s1 - s0) return 2;
  }
  P.pc_nchunk.resize(P.npieces);
  P.pc_rc0.resize(P.npieces);
  P.pc_need.assign(P.npieces, 0);
  P.pc_box.assign(P.npieces, 0);
  std::vector<int32_t> tg;
  auto targets = [&](int64_t p, int32_t r0, int32_t nr, std::vector<int32_t>& out) {
    out.clear();
    for (int32_t i = 0; i < nr; i++) out.push_back(col2piece[S.sn_rows[P.pc_row[p] + r0 + i]]);
    out.erase(std::unique(out.begin(), out.end()), out.end());   // rows ascending => pieces ascending
  };
  std::vector<int32_t> piece_sub(P.npieces, -1);
  for (int64_t s = 0; s < ns; s++)
    if (in_sub[s] >= 0) piece_sub[P.sn_piece[s]] = in_sub[s];   // subtree supernodes are single pieces
  for (int64_t p = 0; p < P.npieces; p++) {
    const int32_t pw = P.pc_w[p];
    const int32_t below = P.pc_nr[p] - pw;
    if (piece_sub[p] >= 0) {                      // solved inside its subtree item
      P.pc_rc0[p] = 0;
      P.hd_tptr.push_back((int64_t)P.hd_tgt.size());
      P.pc_nchunk[p] = 0;
      continue;
    }
    const bool tma = pw >= kTmaMinWidth;
    const int32_t rc0 = tma ? std::min(rows_for(ent0, pw), kTmaRows) : rows_for(ent0, pw);
    const int32_t rc = tma ? std::min(rows_for(ent, pw), kTmaRows) : rows_for(ent, pw);
    // one box height per piece (its tensor map): with the overlapped layout
    // it fits a chunk (heads then stage chunk 0 column by column, into the
    // smaller region B); otherwise both
    P.pc_box[p] = tma ? (ov ? rc : std::max(rc0, rc)) + 4 : 0;
    const int32_t r0n = std::min(below, rc0);
    P.pc_rc0[p] = r0n;
    P.hd_tptr.push_back((int64_t)P.hd_tgt.size());
    targets(p, pw, r0n, tg);
    for (int32_t t : tg) { P.hd_tgt.push_back(t); P.pc_need[t]++; }
    const int32_t rest = below - r0n;
    const int32_t nch = (int32_t)cdiv(rest, rc);
    P.pc_nchunk[p] = nch;
    for (int32_t k = 0; k < nch; k++) {
      const int32_t r0 = pw + r0n + k * rc;
      const int32_t nr = std::min(rc, P.pc_nr[p] - r0);
      P.ch_piece.push_back((int32_t)p);
      P.ch_r0.push_back(r0);
      P.ch_nr.push_back(nr);
      P.ch_k.push_back(k);
      P.ch_tptr.push_back((int64_t)P.ch_tgt.size());
      targets(p, r0, nr, tg);
      for (int32_t t : tg) { P.ch_tgt.push_back(t); P.pc_need[t]++; }
    }
  }
  P.hd_tptr.push_back((int64_t)P.hd_tgt.size());
  P.nchunks = (int64_t)P.ch_piece.size();
  P.ch_tptr.push_back((int64_t)P.ch_tgt.size());
  P.cdesc.resize(P.nchunks);
  for (int64_t c = 0; c < P.nchunks; c++) {
    ChunkDesc& d = P.cdesc[c];
    const int32_t p = P.ch_piece[c];
    d.p = p; d.r0 = P.ch_r0[c]; d.nr = P.ch_nr[c]; d.pw = P.pc_w[p];
    d.f = P.pc_first[p]; d.ld = P.pc_ld[p]; d.c = P.pc_c[p]; d.k = P.ch_k[c];
    d.colbase = P.pc_colbase[p]; d.rowbase = P.pc_row[p] + d.r0;
    d.tp0 = P.ch_tptr[c]; d.tp1 = P.ch_tptr[c + 1];
    d.tma = P.pc_box[p] > 0 ? 1 : 0;
    d.cs = d.tma ? P.pc_box[p] : ((d.nr + 3) & ~3) + 8;
  }
  P.hdesc.resize(P.npieces);
  for (int64_t p = 0; p < P.npieces; p++) {
    HeadDesc& d = P.hdesc[p];
    d.pw = P.pc_w[p]; d.f = P.pc_first[p]; d.rn = P.pc_rc0[p]; d.need = 0;   // need: set below
    d.c = P.pc_c[p]; d.ld = P.pc_ld[p]; d.nch = P.pc_nchunk[p];
    d.tma = P.pc_box[p] > 0 && !ov ? 1 : 0; d.pad = 0;
    d.cs = d.tma ? P.pc_box[p] : ((d.rn + 3) & ~3) + 8;
    d.colbase = P.pc_colbase[p]; d.rowbase = P.pc_row[p];
    d.inv0 = P.pc_inv[p]; d.inv1 = P.pc_inv[p + 1];
    d.tp0 = P.hd_tptr[p]; d.tp1 = P.hd_tptr[p + 1];
  }
  for (int64_t t = 0; t < P.nsub; t++) {
    P.st_tptr.push_back((int64_t)P.st_tgt.size());
    tg.clear();
    for (int64_t s = P.st_first[t]; s <= P.st_last[t]; s++)
      for (int64_t k = P.sw[s]; k < P.snr[s]; k++) {
        const int32_t r = S.sn_rows[P.srow[s] + k];
        if (r >= P.st_chi[t]) tg.push_back(col2piece[r]);
      }
    std::sort(tg.begin(), tg.end());
    tg.erase(std::unique(tg.begin(), tg.end()), tg.end());
    for (int32_t q : tg) { P.st_tgt.push_back(q); P.pc_need[q]++; }
  }
  P.st_tptr.push_back((int64_t)P.st_tgt.size());
  // dispatch order: by the longest dependency chain that still follows an
  // item (most first), ties by depth from the sweep's start. Every item then
  // comes after all of its inputs (the order is topological, so CTAs that
  // hold items waiting on inputs never hold up the items those inputs need),
  // and the items of the critical path are handed out as early as possible.
  {
    std::vector<int64_t> chunk_first(P.npieces + 1, 0);
    for (int64_t c = 0; c < P.nchunks; c++) chunk_first[P.ch_piece[c] + 1]++;
    for (int64_t p = 0; p < P.npieces; p++) chunk_first[p + 1] += chunk_first[p];
    // forward: head(p) after the heads/chunks whose rows hit p; chunk after its head
    std::vector<int64_t> hd(P.npieces, 0), cd(P.nchunks, 0);
    for (int64_t t = 0; t < P.nsub; t++)              // subtree items depend on nothing
      for (int64_t q = P.st_tptr[t]; q < P.st_tptr[t + 1]; q++) hd[P.st_tgt[q]] = std::max<int64_t>(hd[P.st_tgt[q]], 1);
    for (int64_t p = 0; p < P.npieces; p++) {       // pieces are in topological order
      if (piece_sub[p] >= 0) continue;
      for (int64_t t = P.hd_tptr[p]; t < P.hd_tptr[p + 1]; t++) {
        const int32_t q = P.hd_tgt[t];
        hd[q] = std::max(hd[q], hd[p] + 1);
      }
      for (int64_t c = chunk_first[p]; c < chunk_first[p + 1]; c++) {
        cd[c] = hd[p] + 1;
        for (int64_t t = P.ch_tptr[c]; t < P.ch_tptr[c + 1]; t++) {
          const int32_t q = P.ch_tgt[t];
          hd[q] = std::max(hd[q], cd[c] + 1);
        }
      }
    }
    // forward chains still to come: pieces in reverse topological order
    std::vector<int64_t> rh(P.npieces, 0), rc(P.nchunks, 0);
    for (int64_t p = P.npieces - 1; p >= 0; p--) {
      if (piece_sub[p] >= 0) continue;
      int64_t r = 0;
      for (int64_t t = P.hd_tptr[p]; t < P.hd_tptr[p + 1]; t++) r = std::max(r, rh[P.hd_tgt[t]] + 1);
      for (int64_t c = chunk_first[p]; c < chunk_first[p + 1]; c++) {
        int64_t q = 0;
        for (int64_t t = P.ch_tptr[c]; t < P.ch_tptr[c + 1]; t++) q = std::max(q, rh[P.ch_tgt[t]] + 1);
        rc[c] = q;
        r = std::max(r, q + 1);
      }
      rh[p] = r;
    }
    // (key: longest chain after the item, descending; then depth, ascending)
    std::vector<std::array<int64_t, 3>> ord;
    for (int64_t t = 0; t < P.nsub; t++) {
      int64_t r = 0;
      for (int64_t q = P.st_tptr[t]; q < P.st_tptr[t + 1]; q++) r = std::max(r, rh[P.st_tgt[q]] + 1);
      ord.push_back({-r, 0, -1 - P.npieces - t});
    }
    for (int64_t p = 0; p < P.npieces; p++) {
      if (piece_sub[p] >= 0) continue;
      ord.push_back({-rh[p], hd[p] * 2, -1 - p});
      P.fwd_depth = std::max(P.fwd_depth, hd[p]);
    }
    for (int64_t c = 0; c < P.nchunks; c++) ord.push_back({-rc[c], cd[c] * 2 + 1, c});
    auto by_key = [](const std::array<int64_t, 3>& a, const std::array<int64_t, 3>& b) {
      return a[0] != b[0] ? a[0] < b[0] : a[1] < b[1];
    };
    std::stable_sort(ord.begin(), ord.end(), by_key);
    for (auto& o : ord) P.fwd_items.push_back((int32_t)o[2]);
    // backward: chunk after the heads of its targets; head after its chunks and
    // after the heads of its chunk-0 targets
    std::vector<int64_t> bh(P.npieces, 0), bc(P.nchunks, 0);
    for (int64_t p = P.npieces - 1; p >= 0; p--) {
      if (piece_sub[p] >= 0) continue;
      int64_t d = 0;
      for (int64_t t = P.hd_tptr[p]; t < P.hd_tptr[p + 1]; t++) d = std::max(d, bh[P.hd_tgt[t]] + 1);
      for (int64_t c = chunk_first[p]; c < chunk_first[p + 1]; c++) {
        int64_t e = 0;
        for (int64_t t = P.ch_tptr[c]; t < P.ch_tptr[c + 1]; t++) e = std::max(e, bh[P.ch_tgt[t]] + 1);
        bc[c] = e;
        d = std::max(d, e + 1);
      }
      bh[p] = d;
      P.bwd_depth = std::max(P.bwd_depth, d);
    }
    // backward chains still to come: subtrees and lower pieces are the
    // later items, so pieces ascending give each head's final value before
    // it is passed on to its inputs (its chunks and chunk-0 targets)
    std::vector<int64_t> gh(P.npieces, 0), gc(P.nchunks, 0);
    for (int64_t t = 0; t < P.nsub; t++)
      for (int64_t q = P.st_tptr[t]; q < P.st_tptr[t + 1]; q++) gh[P.st_tgt[q]] = std::max<int64_t>(gh[P.st_tgt[q]], 1);
    for (int64_t p = 0; p < P.npieces; p++) {
      if (piece_sub[p] >= 0) continue;
      for (int64_t t = P.hd_tptr[p]; t < P.hd_tptr[p + 1]; t++) gh[P.hd_tgt[t]] = std::max(gh[P.hd_tgt[t]], gh[p] + 1);
      for (int64_t c = chunk_first[p]; c < chunk_first[p + 1]; c++) {
        gc[c] = gh[p] + 1;
        for (int64_t t = P.ch_tptr[c]; t < P.ch_tptr[c + 1]; t++) gh[P.ch_tgt[t]] = std::max(gh[P.ch_tgt[t]], gc[c] + 1);
      }
    }
    ord.clear();
    for (int64_t p = 0; p < P.npieces; p++)
      if (piece_sub[p] < 0) ord.push_back({-gh[p], bh[p] * 2 + 1, -1 - p});
    for (int64_t c = 0; c < P.nchunks; c++) ord.push_back({-gc[c], bc[c] * 2, c});
    for (int64_t t = 0; t < P.nsub; t++) {
      int64_t d = 0;
      for (int64_t q = P.st_tptr[t]; q < P.st_tptr[t + 1]; q++) d = std::max(d, bh[P.st_tgt[q]] + 1);
      ord.push_back({0, d * 2, -1 - P.npieces - t});
      P.bwd_depth = std::max(P.bwd_depth, d);
    }
    std::stable_sort(ord.begin(), ord.end(), by_key);
    for (auto& o : ord) P.bwd_items.push_back((int32_t)o[2]);
  }
  return 0;
}

}  // namespace kkt
