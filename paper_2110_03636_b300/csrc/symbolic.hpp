// Host symbolic analysis for the supernodal Cholesky of
//   H_gamma = H~ + delta I + gamma J^T J            (Sec. 4, eq. gamma)
// computed once per sparsity pattern and reused for every value update
// (Sec. 2: ordering and symbolic factorization are needed only once).
#pragma once
#include <cstdint>
#include <vector>

namespace kkt {

struct RelaxParams {
  int32_t small = 16;   // merge child into parent when merged width <= small
  int32_t num = 1;      // ... or added explicit zeros * den <= num * panel entries
  int32_t den = 10;
  int32_t wmax = 256;   // never relax beyond this width
};

struct Symbolic {
  int64_t n = 0, m = 0;
  std::vector<int32_t> amd;       // fill-reducing order (AMD, natural or ND) before postordering
  std::vector<int32_t> perm;      // perm[k] = original index of position k
  std::vector<int32_t> iperm;     // iperm[perm[k]] = k
  std::vector<int32_t> parent;    // elimination tree in final labels (-1 = root)
  std::vector<int64_t> colcount;  // nnz of each column of L incl. diagonal
  int64_t nnzL = 0;
  double flops = 0.0;             // sum_j colcount_j^2
  // supernodes (contiguous column ranges in final labels)
  int64_t ns = 0;
  std::vector<int32_t> sn_start;  // [ns+1]
  std::vector<int64_t> sn_rowptr; // [ns+1] offsets into sn_rows
  std::vector<int32_t> sn_rows;   // rows of each supernode: its columns, then rows below, ascending
  std::vector<int32_t> sn_parent; // supernodal tree
};

// Pattern-only inputs: H~ lower CSC (diagonal optional in the input, always
// added), J CSR. Returns 0 on success, 1 on invalid pattern (out of range,
// entry above the diagonal, duplicates, unsorted indices).
// ordering: 0 approximate minimum degree, 1 natural, 2 nested dissection
// with leaves of at most nd_leaf vertices.
int analyse_pattern(int64_t n, int64_t m, const int64_t* Hp, const int32_t* Hi,
                    const int64_t* Jp, const int32_t* Ji, const RelaxParams& rp,
                    int ordering, int nd_leaf, Symbolic& out);

}  // namespace kkt
