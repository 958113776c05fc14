"""Host symbolic analysis of the library vs the oracle: bit-exact on the
ordering, etree, column counts and supernodes (CPU only; the library's
kkt_analyse_host makes no CUDA call). Also checks the C ABI surface."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2110_03636_b300 as K
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def lib_symbolic(sys, **opt):
    o = K.kkt_default_options(**opt)
    h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, o)
    try:
        return K.kkt_get_symbolic(h), K.kkt_symbolic_info_get(h)
    finally:
        K.kkt_destroy(h)


def assert_same(sys, relax=(16, 1, 10, 256), ordering=0, nd_leaf=64):
    g, info = lib_symbolic(sys, relax_small=relax[0], relax_num=relax[1], relax_den=relax[2],
                           relax_wmax=relax[3], ordering=ordering, nd_leaf=nd_leaf)
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx,
                     relax_small=relax[0], relax_num=relax[1], relax_den=relax[2], wmax=relax[3],
                     ordering={0: "amd", 1: "natural", 2: "nd"}[ordering], nd_leaf=nd_leaf)
    np.testing.assert_array_equal(g["amd"], sym.amd_order)
    np.testing.assert_array_equal(g["perm"], sym.perm)
    np.testing.assert_array_equal(g["parent"], sym.parent)
    np.testing.assert_array_equal(g["colcount"], sym.colcount)
    st, rp, rows, par = sym.supernodes()
    np.testing.assert_array_equal(g["sn_start"], st)
    np.testing.assert_array_equal(g["sn_rowptr"], rp)
    np.testing.assert_array_equal(g["sn_rows"], rows)
    np.testing.assert_array_equal(g["sn_parent"], par)
    assert info.nnz_l == sym.nnzL and info.flops == sym.flops and info.nsuper == sym.nsuper
    return info


@pytest.mark.parametrize("seed", range(120))
def test_random_tiny_patterns_bit_exact(seed):
    rng = np.random.default_rng(seed)
    sys = W.random_tiny_system(seed + 1000, n_lo=2, n_hi=90, density=float(rng.uniform(0.01, 0.3)))
    assert_same(sys)


@pytest.mark.parametrize("relax", [(1, 0, 1, 1), (1, 0, 1, 256), (4, 1, 4, 8), (32, 3, 10, 64), (16, 1, 10, 256)])
def test_relaxation_parameters_bit_exact(relax):
    for seed in range(6):
        assert_same(W.random_tiny_system(seed + 2000, n_lo=30, n_hi=120, density=0.05), relax=relax)


@pytest.mark.parametrize("seed", range(60))
def test_nested_dissection_random_bit_exact(seed):
    rng = np.random.default_rng(seed)
    sys = W.random_tiny_system(seed + 3000, n_lo=2, n_hi=120, density=float(rng.uniform(0.01, 0.2)))
    assert_same(sys, ordering=2, nd_leaf=int(rng.integers(1, 20)))


@pytest.mark.parametrize("name", ["grid2d_n2000", "grid2d_n20k"])
def test_nested_dissection_workloads_bit_exact(name):
    assert_same(W.make_config(name), ordering=2)


@pytest.mark.slow
def test_nested_dissection_n250k_bit_exact():
    info = assert_same(W.make_config("grid2d_n250k"), ordering=2)
    assert info.nnz_l > 1e8


def test_natural_ordering_bit_exact():
    assert_same(W.make_config("grid2d_n2000"), ordering=1)


def test_grid_n2000_bit_exact():
    assert_same(W.make_config("grid2d_n2000"))


def test_grid_n20k_bit_exact():
    assert_same(W.make_config("grid2d_n20k"))


def test_serving_pattern_bit_exact():
    assert_same(W.serving_pattern(100))


@pytest.mark.slow
def test_grid_n250k_bit_exact():
    """The full 500 x 500 workload (oracle symbolic takes ~20 s)."""
    info = assert_same(W.make_config("grid2d_n250k"))
    assert info.nnz_l > 1e8


def test_trees_and_cliques():
    from test_oracle import graph_sys
    for n in (1, 2, 7, 40):
        edges = [(a, b) for a in range(n) for b in range(a)]
        assert_same(graph_sys(n, edges))
        path = [(i, i + 1) for i in range(n - 1)]
        assert_same(graph_sys(n, path))


def test_invalid_patterns_rejected():
    sys = W.random_tiny_system(5)
    bad = [
        (sys.H_colptr, np.where(np.arange(sys.H_rowidx.size) == 1, 0, sys.H_rowidx)),  # an entry above the diagonal
    ]
    Hi = sys.H_rowidx.copy()
    Hi[-1] = sys.n + 5                                                                  # out of range
    bad.append((sys.H_colptr, Hi))
    for Hp, Hi in bad:
        with pytest.raises(K.KKTError) as e:
            K.kkt_analyse_host(sys.n, sys.m, Hp, Hi, sys.J_rowptr, sys.J_colidx)
        assert e.value.code == 1
    Jc = sys.J_colidx.copy()
    if sys.J_rowptr[1] - sys.J_rowptr[0] >= 2:
        Jc[1] = Jc[0]                                                                   # duplicate column
        with pytest.raises(K.KKTError):
            K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, Jc)
    with pytest.raises(K.KKTError):
        K.kkt_analyse_host(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int64),
                           np.zeros(0, np.int32))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "kkt.h")).read()
    names = set(re.findall(r"\b(kkt_[a-z0-9_]+)\s*\(", hdr))
    lib = ctypes.CDLL(K.LIB_PATH)
    missing = [nm for nm in sorted(names) if not hasattr(lib, nm)]
    assert not missing, missing
    assert set(K.EXPORTED) <= names


def test_host_handle_refuses_device_calls():
    sys = W.random_tiny_system(3)
    h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    try:
        code = K._lib.kkt_factor(h, None, None, 0.0, 1.0, None)
        assert code in (1, 8)
        code = K._lib.kkt_solve(h, None, None, None, None, None)
        assert code in (1, 8)
        buf = np.zeros(6 * max(K.kkt_symbolic_info_get(h).nitems, 1), np.uint64)
        assert K._lib.kkt_get_solve_trace(h, buf.ctypes.data, buf.size) == 8   # no device state
    finally:
        K.kkt_destroy(h)


@pytest.mark.parametrize("name,precision", [("grid2d_n2000", 1), ("grid2d_n20k", 1), ("grid2d_n20k", 0)])
def test_solve_item_orders_cover_every_item_once(name, precision):
    """Both sweeps hand out every work item exactly once: each row chunk, each
    subtree item and the same set of piece heads, nitems in all; the forward
    sweep starts with an item that has no inputs (a subtree or a head)."""
    sys = W.make_config(name)
    o = K.kkt_default_options(precision=precision, ordering=2)
    h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, o)
    try:
        info = K.kkt_symbolic_info_get(h)
        f, b = K.kkt_get_solve_item_order(h)
    finally:
        K.kkt_destroy(h)
    npc = info.npieces
    assert len(f) == len(b) == info.nitems
    for order in (f, b):
        assert len(set(order.tolist())) == len(order)
        chunks = np.sort(order[order >= 0])
        np.testing.assert_array_equal(chunks, np.arange(info.nchunks))
        subs = order[order < -npc]
        assert len(subs) == info.nsub and set((-1 - npc - subs).tolist()) == set(range(info.nsub))
        heads = order[(order < 0) & (order >= -npc)]
        assert len(heads) == info.nitems - info.nchunks - info.nsub
    assert set(f.tolist()) == set(b.tolist())
    # forward: subtree items depend on nothing; some of them come first
    assert f[0] < 0


# ----------------------------------------------------------------- 4x4 form (Sec. 3)
@pytest.mark.parametrize("seed", range(8))
def test_4x4_pattern_and_symbolic_match_oracle_reduction(seed):
    """The library's H~ pattern of the 4x4 form (pat(H) U pat(J_d^T J_d) U
    diag) equals the oracle's reduction, and the symbolic analysis of the
    inner 2x2 system is bit-exact."""
    p = W.random_4x4_parts(seed, n_x=25 + 7 * seed, m_c=6 + seed, m_d=4 + 2 * seed)
    h = K.kkt_analyse_4x4(p["n_x"], p["m_c"], p["m_d"], p["H_colptr"], p["H_rowidx"], p["J_rowptr"],
                          p["J_colidx"], p["Jd_rowptr"], p["Jd_colidx"], host=True)
    try:
        ptr, row = K.kkt_get_4x4_pattern(h, p["n_x"])
        Hp, Hi, _, _ = O.reduce4x4(p)
        np.testing.assert_array_equal(ptr, Hp)
        np.testing.assert_array_equal(row, Hi)
        g = K.kkt_get_symbolic(K.kkt_4x4_inner(h))
        sym = O.Symbolic(p["n_x"], p["m_c"], Hp, Hi, p["J_rowptr"], p["J_colidx"])
        np.testing.assert_array_equal(g["perm"], sym.perm)
        np.testing.assert_array_equal(g["colcount"], sym.colcount)
    finally:
        K.kkt_destroy_4x4(h)


def test_4x4_grid_pattern_matches_oracle_reduction():
    p = W.grid_4x4_parts("grid2d_n2000")
    h = K.kkt_analyse_4x4(p["n_x"], p["m_c"], p["m_d"], p["H_colptr"], p["H_rowidx"], p["J_rowptr"],
                          p["J_colidx"], p["Jd_rowptr"], p["Jd_colidx"], host=True)
    try:
        ptr, row = K.kkt_get_4x4_pattern(h, p["n_x"])
        Hp, Hi, _, _ = O.reduce4x4(p)
        np.testing.assert_array_equal(ptr, Hp)
        np.testing.assert_array_equal(row, Hi)
    finally:
        K.kkt_destroy_4x4(h)


def test_4x4_invalid_jd_rejected():
    p = W.random_4x4_parts(1, n_x=20, m_c=5, m_d=4)
    for bad in ("range", "dup"):
        Jc = p["Jd_colidx"].copy()
        if bad == "range":
            Jc[0] = p["n_x"]
        else:
            r = int(np.argmax(np.diff(p["Jd_rowptr"]) >= 2))
            Jc[p["Jd_rowptr"][r] + 1] = Jc[p["Jd_rowptr"][r]]
        with pytest.raises(K.KKTError) as e:
            K.kkt_analyse_4x4(p["n_x"], p["m_c"], p["m_d"], p["H_colptr"], p["H_rowidx"], p["J_rowptr"],
                              p["J_colidx"], p["Jd_rowptr"], Jc, host=True)
        assert e.value.code == 1


@pytest.mark.parametrize("wa,wc", [(300, 300), (700, 260)])
def test_dense_front_probe_system(wa, wc):
    """The profiling probe's dense-front system (workloads.probe): natural
    order gives exactly three fronts, A (wa columns, wc rows below), B (100
    columns, wc below) and the root C (wc columns), with the library's
    analysis bit-exact against the oracle's."""
    from workloads.probe import dense_fronts
    sys = dense_fronts(wa, wc)
    assert_same(sys, ordering=1)
    g, _ = lib_symbolic(sys, ordering=1)
    w = np.diff(g["sn_start"])
    nr = np.diff(g["sn_rowptr"])
    np.testing.assert_array_equal(w, [wa, 100, wc])
    np.testing.assert_array_equal(nr - w, [wc, wc, 0])
