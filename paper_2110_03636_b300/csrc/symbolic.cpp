// Host symbolic analysis (pattern union, approximate minimum degree,
// elimination tree, postorder, column counts, supernodes).
//
// The ordering follows the approximate-minimum-degree method the paper uses
// (Sec. 5.3, "AMD"), with the approximate external degree of Amestoy, Davis
// and Duff (SIAM J. Matrix Anal. Appl. 17(4), 1996) and every choice pinned so
// that results are reproducible bit for bit:
//   pivot = argmin (degree, index); mass elimination; element absorption;
//   supervariables = variables of the new element with equal variable and
//   element adjacency, merged into the smallest index; no aggressive
//   absorption, no dense-row detection.
// Etree: Liu's algorithm with path compression. Column counts: row subtrees.
#include "symbolic.hpp"

#include <algorithm>
#include <thread>
#include <mutex>
#include <condition_variable>
#include <cstdlib>
#include <set>
#include <tuple>
#include <unordered_map>
#include <utility>

namespace kkt {

namespace {

// --------------------------------------------------------------- pattern
// Off-diagonal adjacency of pat(H~) U pat(J^T J), both halves, sorted.
bool build_graph(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                 const int32_t* Ji, std::vector<int64_t>& gp, std::vector<int32_t>& gi) {
  std::vector<uint64_t> keys;
  size_t est = 2 * (size_t)Hp[n];
  for (int64_t r = 0; r < m; r++) {
    int64_t k = Jp[r + 1] - Jp[r];
    est += (size_t)(k * (k - 1));
  }
  keys.reserve(est);
  for (int64_t j = 0; j < n; j++) {
    int32_t prev = -1;
    for (int64_t q = Hp[j]; q < Hp[j + 1]; q++) {
      int32_t i = Hi[q];
      if (i < j || i >= n || i <= prev) return false;
      prev = i;
      if (i == j) continue;
      keys.push_back(((uint64_t)i << 32) | (uint32_t)j);
      keys.push_back(((uint64_t)j << 32) | (uint32_t)i);
    }
  }
  for (int64_t r = 0; r < m; r++) {
    int32_t prev = -1;
    for (int64_t q = Jp[r]; q < Jp[r + 1]; q++) {
      int32_t a = Ji[q];
      if (a < 0 || a >= n || a <= prev) return false;
      prev = a;
      for (int64_t q2 = Jp[r]; q2 < q; q2++) {
        int32_t b = Ji[q2];
        keys.push_back(((uint64_t)a << 32) | (uint32_t)b);
        keys.push_back(((uint64_t)b << 32) | (uint32_t)a);
      }
    }
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  gp.assign(n + 1, 0);
  gi.resize(keys.size());
  for (size_t t = 0; t < keys.size(); t++) {
    gp[(keys[t] >> 32) + 1]++;
    gi[t] = (int32_t)(keys[t] & 0xffffffffu);
  }
  for (int64_t i = 0; i < n; i++) gp[i + 1] += gp[i];
  return true;
}

// --------------------------------------------------------------- AMD
struct Amd {
  int64_t n;
  std::vector<std::vector<int32_t>> A, E, L;   // variable adj., element adj., element lists
  std::vector<int64_t> deg, wt, lw;            // degree, supervariable weight, |L_e| (weighted)
  std::vector<std::vector<int32_t>> members;
  std::vector<uint8_t> state;                  // 0 variable, 1 element, 2 absorbed element, 3 merged
  std::vector<int64_t> mark, wstamp, wval;
  int64_t gen = 0;
  std::set<std::pair<int64_t, int32_t>> pq;

  void run(const std::vector<int64_t>& gp, const std::vector<int32_t>& gi, std::vector<int32_t>& order) {
    n = (int64_t)gp.size() - 1;
    A.resize(n); E.resize(n); L.resize(n);
    deg.assign(n, 0); wt.assign(n, 1); lw.assign(n, 0);
    members.resize(n);
    state.assign(n, 0);
    mark.assign(n, 0); wstamp.assign(n, 0); wval.assign(n, 0);
    for (int64_t i = 0; i < n; i++) {
      A[i].assign(gi.begin() + gp[i], gi.begin() + gp[i + 1]);
      deg[i] = (int64_t)A[i].size();
      members[i].push_back((int32_t)i);
      pq.insert({deg[i], (int32_t)i});
    }
    order.clear();
    order.reserve(n);
    int64_t nel = 0;
    std::vector<int32_t> Lp;
    std::vector<int64_t> newdeg;
    while (!pq.empty()) {
      const int32_t p = pq.begin()->second;
      pq.erase(pq.begin());
      // L_p = (A_p U union of L_e, e in E_p) \ {p}
      gen++;
      mark[p] = gen;
      Lp.clear();
      for (int32_t v : A[p])
        if (state[v] == 0 && mark[v] != gen) { mark[v] = gen; Lp.push_back(v); }
      for (int32_t e : E[p])
        for (int32_t v : L[e])
          if (state[v] == 0 && mark[v] != gen) { mark[v] = gen; Lp.push_back(v); }
      // p's members leave in ascending order
      std::sort(members[p].begin(), members[p].end());
      for (int32_t v : members[p]) order.push_back(v);
      nel += wt[p];
      state[p] = 1;
      // absorb the elements adjacent to p
      for (int32_t e : E[p]) { state[e] = 2; std::vector<int32_t>().swap(L[e]); }
      int64_t Lw = 0;
      for (int32_t i : Lp) {
        Lw += wt[i];
        auto& Ai = A[i];
        Ai.erase(std::remove_if(Ai.begin(), Ai.end(), [&](int32_t v) { return mark[v] == gen; }), Ai.end());
        auto& Ei = E[i];
        Ei.erase(std::remove_if(Ei.begin(), Ei.end(), [&](int32_t e) { return state[e] != 1; }), Ei.end());
        Ei.push_back(p);
      }
      std::vector<int32_t>().swap(A[p]);
      std::vector<int32_t>().swap(E[p]);
      L[p] = Lp;
      lw[p] = Lw;
      // |L_e \ L_p| = |L_e| - sum of weights of L_p's variables adjacent to e
      for (int32_t i : Lp)
        for (int32_t e : E[i]) {
          if (e == p) continue;
          if (wstamp[e] != gen) { wstamp[e] = gen; wval[e] = lw[e]; }
          wval[e] -= wt[i];
        }
      newdeg.resize(Lp.size());
      for (size_t t = 0; t < Lp.size(); t++) {
        const int32_t i = Lp[t];
        int64_t a = 0, c = 0;
        for (int32_t v : A[i]) a += wt[v];
        for (int32_t e : E[i])
          if (e != p) c += wval[e];
        const int64_t b = Lw - wt[i];
        newdeg[t] = std::min(std::min(n - nel - wt[i], deg[i] + b), a + b + c);
      }
      for (size_t t = 0; t < Lp.size(); t++) {
        const int32_t i = Lp[t];
        pq.erase({deg[i], i});
        deg[i] = newdeg[t];
      }
      detect_supervariables(Lp);
      for (int32_t i : Lp)
        if (state[i] == 0) pq.insert({deg[i], i});
    }
  }

  static uint64_t set_hash(const std::vector<int32_t>& a, const std::vector<int32_t>& e) {
    uint64_t h = 0x9e3779b97f4a7c15ull * (a.size() + 1) + e.size();
    uint64_t s1 = 0, s2 = 0;
    for (int32_t v : a) s1 += (uint64_t)v * 0x100000001b3ull + 7;
    for (int32_t v : e) s2 += (uint64_t)v * 0xc2b2ae3d27d4eb4full + 11;
    return h ^ s1 ^ (s2 << 1);
  }

  void detect_supervariables(const std::vector<int32_t>& Lp) {
    std::unordered_map<uint64_t, std::vector<int32_t>> buckets;
    buckets.reserve(Lp.size() * 2);
    for (int32_t i : Lp) buckets[set_hash(A[i], E[i])].push_back(i);
    std::vector<int32_t> sa, sb, ea, eb;
    for (auto& kv : buckets) {
      auto& cand = kv.second;
      if (cand.size() < 2) continue;
      std::sort(cand.begin(), cand.end());
      for (size_t x = 0; x < cand.size(); x++) {
        const int32_t r = cand[x];
        if (state[r] != 0) continue;
        sa = A[r]; std::sort(sa.begin(), sa.end());
        ea = E[r]; std::sort(ea.begin(), ea.end());
        for (size_t y = x + 1; y < cand.size(); y++) {
          const int32_t j = cand[y];
          if (state[j] != 0 || A[j].size() != sa.size() || E[j].size() != ea.size()) continue;
          sb = A[j]; std::sort(sb.begin(), sb.end());
          if (sb != sa) continue;
          eb = E[j]; std::sort(eb.begin(), eb.end());
          if (eb != ea) continue;
          // j joins r
          wt[r] += wt[j];
          deg[r] -= wt[j];
          members[r].insert(members[r].end(), members[j].begin(), members[j].end());
          std::vector<int32_t>().swap(members[j]);
          state[j] = 3;
          for (int32_t k : A[j]) {
            auto& Ak = A[k];
            Ak.erase(std::remove(Ak.begin(), Ak.end(), j), Ak.end());
          }
          std::vector<int32_t>().swap(A[j]);
          std::vector<int32_t>().swap(E[j]);
        }
      }
    }
  }
};


// --------------------------------------------------------------- nested dissection
// Level-structure nested dissection (George & Liu's automatic nested
// dissection) with the pinned choices: components by BFS from their smallest
// vertex; pseudo-peripheral root by repeated BFS from the smallest vertex
// (move to the fewest-neighbour vertex of the last level while the level
// structure grows); separator level = the smallest level in the middle
// third (ties: closest to the middle, then lowest); only separator-level
// vertices with a neighbour one level further stay in the separator; order
// = part before, part after, separator.
struct Nd {
  const std::vector<int64_t>& gp;
  const std::vector<int32_t>& gi;
  int32_t leaf;
  Nd(const std::vector<int64_t>& p, const std::vector<int32_t>& i, int32_t l) : gp(p), gi(i), leaf(l) {}

  // Per-thread scratch: stamps mark membership of the current set and BFS
  // visits (each thread counts its own stamps, so tasks on different threads
  // never see each other's marks as their own).
  struct Scratch {
    std::vector<int32_t> member, seen;
    int32_t stamp = 0;
    std::vector<std::vector<int32_t>> L, L2;
    explicit Scratch(size_t n) : member(n, 0), seen(n, 0) {}
  };
  // A subproblem and where its vertices go in the order: kind 0 = a set to
  // split into components, 2 = one connected component.
  struct Task {
    int kind;
    int64_t off;
    std::vector<int32_t> v;
  };

  // BFS level structure of the member set (stamp mst) from r
  void levels_from(Scratch& w, int32_t r, int32_t mst, std::vector<std::vector<int32_t>>& L) {
    L.clear();
    const int32_t st = ++w.stamp;
    L.push_back({r});
    w.seen[r] = st;
    for (size_t d = 0; d < L.size(); d++) {
      std::vector<int32_t> nxt;
      for (int32_t v : L[d])
        for (int64_t q = gp[v]; q < gp[v + 1]; q++) {
          const int32_t u = gi[q];
          if (w.member[u] == mst && w.seen[u] != st) { w.seen[u] = st; nxt.push_back(u); }
        }
      if (nxt.empty()) break;
      std::sort(nxt.begin(), nxt.end());
      L.push_back(std::move(nxt));
    }
  }

  // One task: writes the vertices it places into order[] and appends the
  // subtasks it creates to out (each with its final offset).
  void process(Task& t, Scratch& w, std::vector<int32_t>& order, std::vector<Task>& out) {
    if (t.kind == 0) {
      std::sort(t.v.begin(), t.v.end());
      const int32_t mst = ++w.stamp;
      for (int32_t v : t.v) w.member[v] = mst;
      const int32_t vst = ++w.stamp;
      int64_t off = t.off;
      for (int32_t s0 : t.v) {
        if (w.seen[s0] == vst) continue;
        std::vector<int32_t> c{s0};
        w.seen[s0] = vst;
        for (size_t h = 0; h < c.size(); h++)
          for (int64_t q = gp[c[h]]; q < gp[c[h] + 1]; q++) {
            const int32_t u = gi[q];
            if (w.member[u] == mst && w.seen[u] != vst) { w.seen[u] = vst; c.push_back(u); }
          }
        std::sort(c.begin(), c.end());
        const int64_t sz = (int64_t)c.size();
        out.push_back({2, off, std::move(c)});
        off += sz;
      }
      return;
    }
    std::vector<int32_t>& C = t.v;
    auto emit = [&](const std::vector<int32_t>& v, int64_t off) { std::copy(v.begin(), v.end(), order.begin() + off); };
    if ((int64_t)C.size() <= leaf) { emit(C, t.off); return; }
    const int32_t mst = ++w.stamp;
    for (int32_t v : C) w.member[v] = mst;
    auto deg_in = [&](int32_t v) {
      int64_t d = 0;
      for (int64_t q = gp[v]; q < gp[v + 1]; q++) d += w.member[gi[q]] == mst;
      return d;
    };
    std::vector<std::vector<int32_t>>& L = w.L;
    std::vector<std::vector<int32_t>>& L2 = w.L2;
    levels_from(w, C[0], mst, L);
    for (;;) {
      int32_t x = -1;
      int64_t bd = 0;
      for (int32_t v : L.back()) {
        const int64_t d = deg_in(v);
        if (x < 0 || d < bd || (d == bd && v < x)) { x = v; bd = d; }
      }
      levels_from(w, x, mst, L2);
      if (L2.size() > L.size()) std::swap(L, L2);
      else break;
    }
    const int64_t h = (int64_t)L.size() - 1;
    if (h < 2) { emit(C, t.off); return; }
    const int64_t lo = std::max<int64_t>(1, h / 3);
    const int64_t hi = std::min<int64_t>(h - 1, std::max<int64_t>(1, (2 * h + 2) / 3));
    const int64_t mid = (h + 1) / 2;
    int64_t k = lo;
    for (int64_t q = lo + 1; q <= hi; q++) {
      const auto key = std::make_tuple(L[q].size(), std::llabs(q - mid), q);
      const auto best = std::make_tuple(L[k].size(), std::llabs(k - mid), k);
      if (key < best) k = q;
    }
    const int32_t nst = ++w.stamp;            // marks level k+1
    for (int32_t v : L[k + 1]) w.seen[v] = nst;
    std::vector<int32_t> S, P1, P2;
    for (int64_t d = 0; d < k; d++) P1.insert(P1.end(), L[d].begin(), L[d].end());
    for (int32_t v : L[k]) {
      bool sep = false;
      for (int64_t q = gp[v]; q < gp[v + 1] && !sep; q++) sep = w.seen[gi[q]] == nst;
      (sep ? S : P1).push_back(v);
    }
    for (int64_t d = k + 1; d <= h; d++) P2.insert(P2.end(), L[d].begin(), L[d].end());
    // order = part before, part after, separator
    const int64_t n1 = (int64_t)P1.size(), n2 = (int64_t)P2.size();
    emit(S, t.off + n1 + n2);
    out.push_back({0, t.off, std::move(P1)});
    out.push_back({0, t.off + n1, std::move(P2)});
  }

  // Subproblems are independent and each knows its place in the order, so
  // they run on a pool of threads (a subproblem below kLocal vertices is
  // finished by the thread that made it); the order does not depend on the
  // schedule.
  void run(std::vector<int32_t>& order) {
    const int32_t n = (int32_t)gp.size() - 1;
    order.assign(n, -1);
    constexpr int64_t kLocal = 4096;
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 32u));
    if (n < 4 * kLocal) nt = 1;
    std::vector<Task> queue;
    std::vector<int32_t> all(n);
    for (int32_t i = 0; i < n; i++) all[i] = i;
    queue.push_back({0, 0, std::move(all)});
    std::mutex mu;
    std::condition_variable cv;
    int busy = 0;
    auto worker = [&]() {
      Scratch w((size_t)n);
      std::vector<Task> out, local;
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        cv.wait(lk, [&] { return !queue.empty() || busy == 0; });
        if (queue.empty()) return;   // busy == 0 and nothing queued: done
        Task t = std::move(queue.back());
        queue.pop_back();
        busy++;
        lk.unlock();
        local.clear();
        local.push_back(std::move(t));
        std::vector<Task> share;
        while (!local.empty()) {
          Task u = std::move(local.back());
          local.pop_back();
          out.clear();
          process(u, w, order, out);
          for (Task& o : out) ((int64_t)o.v.size() >= kLocal && nt > 1 ? share : local).push_back(std::move(o));
        }
        lk.lock();
        for (Task& o : share) queue.push_back(std::move(o));
        busy--;
        cv.notify_all();
      }
    };
    std::vector<std::thread> th;
    for (unsigned k = 1; k < nt; k++) th.emplace_back(worker);
    worker();
    for (std::thread& x : th) x.join();
  }
};


// --------------------------------------------------------------- etree
// Liu's algorithm on P A P^T given in the graph's labels and a permutation.
void etree_liu(int64_t n, const std::vector<int64_t>& gp, const std::vector<int32_t>& gi,
               const std::vector<int32_t>& perm, const std::vector<int32_t>& iperm,
               std::vector<int32_t>& parent) {
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int64_t k = 0; k < n; k++) {
    const int32_t ok = perm[k];
    for (int64_t q = gp[ok]; q < gp[ok + 1]; q++) {
      int32_t i = iperm[gi[q]];
      if (i >= k) continue;
      // climb from i to the root of its current subtree, compressing the path to k
      while (i != -1 && i < k) {
        const int32_t next = anc[i];
        anc[i] = (int32_t)k;
        if (next == -1) { parent[i] = (int32_t)k; break; }
        i = next;
      }
    }
  }
}

void postorder_tree(int64_t n, const std::vector<int32_t>& parent, std::vector<int32_t>& post) {
  std::vector<int32_t> head(n, -1), next(n, -1);
  for (int64_t j = n - 1; j >= 0; j--) {       // reverse insertion => ascending children lists
    if (parent[j] < 0) continue;
    next[j] = head[parent[j]];
    head[parent[j]] = (int32_t)j;
  }
  post.resize(n);
  std::vector<int32_t> stack;
  int64_t k = 0;
  for (int64_t r = 0; r < n; r++) {
    if (parent[r] >= 0) continue;
    stack.push_back((int32_t)r);
    while (!stack.empty()) {
      const int32_t v = stack.back();
      const int32_t c = head[v];
      if (c >= 0) {
        head[v] = next[c];
        stack.push_back(c);
      } else {
        post[k++] = v;
        stack.pop_back();
      }
    }
  }
}

}  // namespace

int analyse_pattern(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi, const int64_t* Jp,
                    const int32_t* Ji, const RelaxParams& rp, int ordering, int nd_leaf, Symbolic& S) {
  if (n <= 0 || m < 0 || n >= (int64_t)INT32_MAX) return 1;
  if (Hp[0] != 0 || (m > 0 && Jp[0] != 0)) return 1;
  for (int64_t j = 0; j < n; j++) if (Hp[j + 1] < Hp[j]) return 1;
  for (int64_t r = 0; r < m; r++) if (Jp[r + 1] < Jp[r]) return 1;
  std::vector<int64_t> gp;
  std::vector<int32_t> gi;
  if (!build_graph(n, m, Hp, Hi, Jp, Ji, gp, gi)) return 1;
  S = Symbolic();
  S.n = n;
  S.m = m;
  if (ordering == 0) {
    Amd amd;
    amd.run(gp, gi, S.amd);
  } else if (ordering == 2) {
    Nd nd(gp, gi, nd_leaf);
    nd.run(S.amd);
  } else {
    S.amd.resize(n);
    for (int64_t i = 0; i < n; i++) S.amd[i] = (int32_t)i;
  }
  // etree on the AMD order, postorder, relabel
  std::vector<int32_t> ia(n), par0, post;
  for (int64_t k = 0; k < n; k++) ia[S.amd[k]] = (int32_t)k;
  etree_liu(n, gp, gi, S.amd, ia, par0);
  postorder_tree(n, par0, post);
  std::vector<int32_t> ipost(n);
  for (int64_t k = 0; k < n; k++) ipost[post[k]] = (int32_t)k;
  S.perm.resize(n);
  S.iperm.resize(n);
  S.parent.resize(n);
  for (int64_t k = 0; k < n; k++) {
    S.perm[k] = S.amd[post[k]];
    S.iperm[S.perm[k]] = (int32_t)k;
    const int32_t pa = par0[post[k]];
    S.parent[k] = pa < 0 ? -1 : ipost[pa];
  }
  // Column counts without visiting L (Gilbert, Ng & Peyton, "An efficient
  // algorithm to compute row and column counts for sparse Cholesky
  // factorization", SIAM J. Matrix Anal. Appl. 15(4), 1994). Row i of L is
  // the row subtree T_i: the etree paths from i's neighbours k < i up to i.
  // cc(j) counts the row subtrees holding j. Give each T_i weights: +1 at
  // every neighbour k < i and at i, -1 at the lowest common ancestor of
  // consecutive ones (in postorder, i last) and -1 at parent(i); the weights
  // of T_i summed over the subtree of any j give 1 if j lies in T_i, else 0.
  // So cc(j) is the subtree sum of all weights. Columns are taken in
  // postorder; a disjoint-set forest over the finished columns (each linked
  // to its parent once done) answers lca(prev, j) = find(prev).
  {
    std::vector<int64_t> wgt(n, 1);            // +1: i as the last leaf of T_i
    std::vector<int32_t> prev(n, -1), anc(n);
    for (int64_t j = 0; j < n; j++) anc[j] = (int32_t)j;
    auto find = [&](int32_t x) {
      while (anc[x] != x) {                    // path halving
        anc[x] = anc[anc[x]];
        x = anc[x];
      }
      return x;
    };
    for (int64_t j = 0; j < n; j++) {
      const int32_t oj = S.perm[j];
      for (int64_t q = gp[oj]; q < gp[oj + 1]; q++) {
        const int32_t i = S.iperm[gi[q]];
        if (i <= j) continue;                  // j is a neighbour k < i of row i
        wgt[j] += 1;
        if (prev[i] >= 0) wgt[find(prev[i])] -= 1;
        prev[i] = (int32_t)j;
      }
      if (S.parent[j] >= 0) anc[j] = S.parent[j];
    }
    for (int64_t i = 0; i < n; i++) {
      if (prev[i] >= 0) wgt[i] -= 1;           // lca(last neighbour, i) = i
      if (S.parent[i] >= 0) wgt[S.parent[i]] -= 1;
    }
    S.colcount.assign(n, 0);
    for (int64_t j = 0; j < n; j++) {          // children precede parents
      S.colcount[j] += wgt[j];
      if (S.parent[j] >= 0) S.colcount[S.parent[j]] += S.colcount[j];
    }
  }
  S.nnzL = 0;
  S.flops = 0.0;
  for (int64_t j = 0; j < n; j++) {
    S.nnzL += S.colcount[j];
    S.flops += (double)S.colcount[j] * (double)S.colcount[j];
  }
  // fundamental supernodes
  std::vector<int32_t> nchild(n, 0);
  for (int64_t j = 0; j < n; j++) if (S.parent[j] >= 0) nchild[S.parent[j]]++;
  std::vector<int32_t> fund;   // first columns
  for (int64_t j = 0; j < n; j++) {
    const bool extend = j > 0 && S.parent[j - 1] == j && nchild[j] == 1 && S.colcount[j - 1] == S.colcount[j] + 1;
    if (!extend) fund.push_back((int32_t)j);
  }
  fund.push_back((int32_t)n);
  // relaxation in one left-to-right pass
  struct Span { int32_t f, l; int64_t nz; };
  std::vector<Span> rel;
  rel.reserve(fund.size());
  for (size_t s = 0; s + 1 < fund.size(); s++) {
    Span cur{fund[s], fund[s + 1] - 1, 0};
    for (int32_t j = cur.f; j <= cur.l; j++) cur.nz += S.colcount[j];
    if (!rel.empty()) {
      const Span& t = rel.back();
      if (t.l == cur.f - 1 && S.parent[t.l] == cur.f) {
        const int64_t w = (int64_t)cur.l - t.f + 1;
        const int64_t below = S.colcount[cur.l] - 1;
        const int64_t panel = w * (w + 1) / 2 + w * below;
        const int64_t zeros = panel - (t.nz + cur.nz);
        if (w <= rp.wmax && (w <= rp.small || zeros * (int64_t)rp.den <= (int64_t)rp.num * panel)) {
          rel.back().l = cur.l;
          rel.back().nz += cur.nz;
          continue;
        }
      }
    }
    rel.push_back(cur);
  }
  S.ns = (int64_t)rel.size();
  S.sn_start.resize(S.ns + 1);
  std::vector<int32_t> col2sn(n), last_of(n, -1);
  for (int64_t s = 0; s < S.ns; s++) {
    S.sn_start[s] = rel[s].f;
    for (int32_t j = rel[s].f; j <= rel[s].l; j++) col2sn[j] = (int32_t)s;
    last_of[rel[s].l] = (int32_t)s;
  }
  S.sn_start[S.ns] = (int32_t)n;
  // rows below each supernode = structure of its last column l: the rows
  // > l adjacent to any of its columns, joined with the rows > l of its
  // child supernodes (a supernode's columns form one etree chain, and every
  // other etree child of those columns ends a child supernode). Children
  // precede parents, so one pass in supernode order suffices; it touches
  // the row lists, not the entries of L.
  std::vector<std::vector<int32_t>> below(S.ns);
  {
    std::vector<std::vector<int32_t>> kids(S.ns);
    for (int64_t s = 0; s < S.ns; s++) {
      const int32_t pl = S.parent[rel[s].l];
      if (pl >= 0) kids[col2sn[pl]].push_back((int32_t)s);
    }
    std::vector<int32_t> mark(n, -1);
    for (int64_t s = 0; s < S.ns; s++) {
      const int32_t l = rel[s].l;
      std::vector<int32_t>& B = below[s];
      auto add = [&](int32_t r) {
        if (r > l && mark[r] != (int32_t)s) {
          mark[r] = (int32_t)s;
          B.push_back(r);
        }
      };
      for (int32_t j = rel[s].f; j <= l; j++) {
        const int32_t oj = S.perm[j];
        for (int64_t q = gp[oj]; q < gp[oj + 1]; q++) add(S.iperm[gi[q]]);
      }
      for (int32_t c : kids[s])
        for (int32_t r : below[c]) add(r);
      std::sort(B.begin(), B.end());
    }
  }
  S.sn_rowptr.assign(S.ns + 1, 0);
  for (int64_t s = 0; s < S.ns; s++)
    S.sn_rowptr[s + 1] = S.sn_rowptr[s] + (rel[s].l - rel[s].f + 1) + (int64_t)below[s].size();
  S.sn_rows.resize(S.sn_rowptr[S.ns]);
  S.sn_parent.resize(S.ns);
  for (int64_t s = 0; s < S.ns; s++) {
    int64_t q = S.sn_rowptr[s];
    for (int32_t j = rel[s].f; j <= rel[s].l; j++) S.sn_rows[q++] = j;
    for (int32_t r : below[s]) S.sn_rows[q++] = r;
    const int32_t pl = S.parent[rel[s].l];
    S.sn_parent[s] = pl < 0 ? -1 : col2sn[pl];
  }
  return 0;
}

}  // namespace kkt
