"""Pins of the supernode partition (S5) against hand-worked cases and the
definition of fundamental supernodes, for the oracle and for the library's
host analysis (CPU only).

The paper (Sec. 5.3) fixes the ordering only; the partition rule is pinned
in ``tests/golden/supernodes_hand_worked.md``: fundamental supernodes by
their definition, then one relaxation pass with the constants (relax_small,
num/den, wmax) as inputs. Each golden case exercises one clause (width limit,
zero fraction at and just beyond equality, the wmax cap, the last-child
condition), so a wrong comparison, a wrong panel count or a merge of a
non-last child fails one of them."""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_2110_03636_b300 as K
import workloads as W
from test_oracle import adjacency_dense, brute_symbolic, graph_sys

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

with open(os.path.join(GOLDEN, "supernodes_hand_worked.json")) as _f:
    _CASES = json.load(_f)
_PARAMS = [(name, p) for name, c in _CASES.items() if not name.startswith("_") for p in c["params"]]


def _case_sys(c):
    # edges are (row, column) of the strictly lower pattern
    return graph_sys(c["n"], [(int(a), int(b)) for a, b in c["edges"]])


def _oracle_partition(sys, relax):
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, ordering="natural",
                     relax_small=relax[0], relax_num=relax[1], relax_den=relax[2], wmax=relax[3])
    st, rp, rows, par = sym.supernodes()
    return sym, st, [rows[rp[s]:rp[s + 1]].tolist() for s in range(len(st) - 1)], par


def _library_partition(sys, relax):
    o = K.kkt_default_options(ordering=1, relax_small=relax[0], relax_num=relax[1], relax_den=relax[2],
                              relax_wmax=relax[3])
    h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, o)
    try:
        g = K.kkt_get_symbolic(h)
    finally:
        K.kkt_destroy(h)
    st, rp = g["sn_start"], g["sn_rowptr"]
    rows = [g["sn_rows"][rp[s]:rp[s + 1]].tolist() for s in range(len(st) - 1)]
    return g, st, rows, g["sn_parent"]


@pytest.mark.parametrize("name,pname", _PARAMS)
def test_oracle_partition_hand_worked(name, pname):
    c = _CASES[name]
    want = c["params"][pname]
    sym, st, rows, par = _oracle_partition(_case_sys(c), want["relax"])
    assert sym.perm.tolist() == list(range(c["n"]))
    assert sym.parent.tolist() == c["parent"]
    assert sym.colcount.tolist() == c["colcount"]
    assert st.tolist() == want["start"]
    assert par.tolist() == want["sparent"]
    assert rows == want["rows"]


@pytest.mark.parametrize("name,pname", _PARAMS)
def test_library_partition_hand_worked(name, pname):
    c = _CASES[name]
    want = c["params"][pname]
    g, st, rows, par = _library_partition(_case_sys(c), want["relax"])
    assert g["parent"].tolist() == c["parent"]
    assert st.tolist() == want["start"]
    assert par.tolist() == want["sparent"]
    assert rows == want["rows"]


def _fundamental_by_definition(parent, cc):
    """Starts of the fundamental supernodes from their definition."""
    n = len(parent)
    kids = np.zeros(n, int)
    for j in range(n):
        if parent[j] >= 0:
            kids[parent[j]] += 1
    starts = [j for j in range(n) if not (j > 0 and parent[j - 1] == j and kids[j] == 1 and cc[j - 1] == cc[j] + 1)]
    return starts + [n]


@pytest.mark.parametrize("seed", range(30))
def test_fundamental_supernodes_are_maximal(seed):
    """With merging switched off (wmax = 1) the partition is exactly the
    fundamental one of the definition, computed here from a brute-force
    boolean elimination (etree = first row below the diagonal, cc = column
    counts): every adjacent pair that may join does, and no other."""
    rng = np.random.default_rng(seed)
    sys = W.random_tiny_system(seed + 3100, n_lo=10, n_hi=70, density=float(rng.uniform(0.03, 0.2)))
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx,
                     relax_small=1, relax_num=0, relax_den=1, wmax=1)
    Lb = brute_symbolic(sys.n, adjacency_dense(sys), sym.perm)
    parent = [int(np.nonzero(Lb[:, j])[0].min()) if Lb[:, j].any() else -1 for j in range(sys.n)]
    cc = (Lb.sum(0) + 1).tolist()
    want = _fundamental_by_definition(parent, cc)
    assert sym.supernodes()[0].tolist() == want
    g, st, _, _ = _library_partition_any(sys, (1, 0, 1, 1), ordering=0)
    assert st.tolist() == want


def _library_partition_any(sys, relax, ordering):
    o = K.kkt_default_options(ordering=ordering, relax_small=relax[0], relax_num=relax[1], relax_den=relax[2],
                              relax_wmax=relax[3])
    h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, o)
    try:
        g = K.kkt_get_symbolic(h)
    finally:
        K.kkt_destroy(h)
    return g, g["sn_start"], None, g["sn_parent"]


@pytest.mark.parametrize("seed", range(20))
def test_relaxed_partition_coarsens_fundamental_and_every_boundary_is_refused(seed):
    """A relaxed partition is a union of consecutive fundamental supernodes,
    and at every boundary between relaxed supernodes where the left one is
    the right one's last child, the rule refuses the merge of the left
    relaxed supernode with the right one's first fundamental supernode (the
    pass is greedy, so that is the merge it considered). Quantities come
    from the brute-force elimination."""
    rng = np.random.default_rng(seed)
    sys = W.random_tiny_system(seed + 3300, n_lo=20, n_hi=80, density=float(rng.uniform(0.02, 0.12)))
    relax = (int(rng.integers(1, 6)), int(rng.integers(0, 3)), int(rng.integers(1, 6)), int(rng.integers(2, 9)))
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, relax_small=relax[0],
                     relax_num=relax[1], relax_den=relax[2], wmax=relax[3])
    Lb = brute_symbolic(sys.n, adjacency_dense(sys), sym.perm)
    parent = [int(np.nonzero(Lb[:, j])[0].min()) if Lb[:, j].any() else -1 for j in range(sys.n)]
    cc = (Lb.sum(0) + 1).tolist()
    fund = _fundamental_by_definition(parent, cc)
    st = sym.supernodes()[0].tolist()
    assert set(st) <= set(fund)
    for s in range(1, len(st) - 1):
        f = st[s]
        l = fund[fund.index(f) + 1] - 1              # last column of the first fundamental piece
        if parent[f - 1] != f:
            continue                                 # not the last child: no merge was considered
        Wd = l - st[s - 1] + 1
        panel = Wd * (Wd + 1) // 2 + Wd * (cc[l] - 1)
        z = panel - sum(cc[st[s - 1]:l + 1])
        ok = Wd <= relax[3] and (Wd <= relax[0] or z * relax[2] <= relax[1] * panel)
        assert not ok, (s, f, l, Wd, panel, z)
