"""Pins for the CPU oracle, against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a dense
LU/Cholesky/eigenvalue computation (numpy), a closed form, a theorem of the
paper, or a brute-force symbolic elimination.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def dense_H(sys):
    n = sys.n
    H = np.zeros((n, n))
    for j in range(n):
        for q in range(sys.H_colptr[j], sys.H_colptr[j + 1]):
            i = sys.H_rowidx[q]
            H[i, j] += sys.H_vals[q]
            if i != j:
                H[j, i] += sys.H_vals[q]
    return H


def dense_J(sys):
    J = np.zeros((sys.m, sys.n))
    for r in range(sys.m):
        for q in range(sys.J_rowptr[r], sys.J_rowptr[r + 1]):
            J[r, sys.J_colidx[q]] += sys.J_vals[q]
    return J


def dense_K(sys, delta=None):
    d = sys.delta if delta is None else delta
    H, J = dense_H(sys), dense_J(sys)
    n, m = sys.n, sys.m
    K = np.zeros((n + m, n + m))
    K[:n, :n] = H + d * np.eye(n)
    K[:n, n:] = J.T
    K[n:, :n] = J
    return K


def make_sys(H, J, rx, ry, delta=0.0, gamma=1e2):
    """KKTSystem from dense H (symmetric) and J."""
    n, m = H.shape[0], J.shape[0]
    rows, cols = np.nonzero(np.tril(H, -1))
    Hp, Hi, Hv = W.lower_csc(n, rows, cols, H[rows, cols], np.diag(H))
    Jr, Jc = np.nonzero(J)
    Jp = np.zeros(m + 1, np.int64)
    np.add.at(Jp, Jr + 1, 1)
    Jp = np.cumsum(Jp)
    return W.KKTSystem(n, m, Hp, Hi, Hv, Jp, Jc.astype(np.int32), J[Jr, Jc], rx, ry, delta, gamma)


def brute_symbolic(n, adj_dense, perm):
    """Dense boolean elimination of P A P^T: returns the strictly-lower
    pattern of L as a boolean matrix (B[i, j] True for i > j)."""
    B = adj_dense[np.ix_(perm, perm)].copy()
    np.fill_diagonal(B, False)
    B = B | B.T
    L = np.zeros((n, n), bool)
    for k in range(n):
        nb = np.nonzero(B[k, k + 1:])[0] + k + 1
        L[nb, k] = True
        for a in nb:
            B[a, nb] = True
        B[nb, nb] = False  # no self loops
        for a in nb:
            for b in nb:
                if a != b:
                    B[a, b] = True
    return L


def adjacency_dense(sys):
    A = np.zeros((sys.n, sys.n), bool)
    for j in range(sys.n):
        for q in range(sys.H_colptr[j], sys.H_colptr[j + 1]):
            i = sys.H_rowidx[q]
            A[i, j] = A[j, i] = True
    for r in range(sys.m):
        cols = sys.J_colidx[sys.J_rowptr[r]:sys.J_rowptr[r + 1]]
        for a in cols:
            for b in cols:
                A[a, b] = True
    np.fill_diagonal(A, False)
    return A


def graph_sys(n, edges):
    """KKT system whose H~ pattern is the given graph and J is empty (m=0)."""
    rows = [max(a, b) for a, b in edges]
    cols = [min(a, b) for a, b in edges]
    Hp, Hi, Hv = W.lower_csc(n, rows, cols, -np.ones(len(edges)), np.full(n, float(n)))
    return W.KKTSystem(n, 0, Hp, Hi, Hv, np.zeros(1, np.int64), np.zeros(0, np.int32),
                       np.zeros(0), np.zeros(n), np.zeros(0), 0.0, 0.0)


def sym_of(sys, **kw):
    return O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, **kw)


# ----------------------------------------------------------------- solution
@pytest.mark.parametrize("seed", range(25))
def test_solution_matches_dense_lu(seed):
    """Solution of the 2x2 KKT system (eq. linsys2x2) equals a dense LU solve."""
    sys = W.random_tiny_system(seed)
    sym, fac, dx, dy, info = O.solve_system(sys)
    assert info["status"] == 0 and info["inertia_ok"]
    K = dense_K(sys)
    ref = np.linalg.solve(K, np.concatenate([sys.r_x, sys.r_y]))
    got = np.concatenate([dx, dy])
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    assert info["rr"] <= 1e-10


@pytest.mark.parametrize("seed", range(8))
def test_gamma_invariance(seed):
    """H_gamma = H~ + gamma J^T J does not change the solution (Sec. 4, Q = gamma I)."""
    sys = W.random_tiny_system(seed + 100)
    ref = np.linalg.solve(dense_K(sys), np.concatenate([sys.r_x, sys.r_y]))
    for gamma in (0.0, 1.0, 1e2, 1e4, 1e6):
        s = sys.copy()
        s.gamma = gamma
        _, _, dx, dy, info = O.solve_system(s)
        assert info["status"] == 0
        err = np.linalg.norm(np.concatenate([dx, dy]) - ref) / np.linalg.norm(ref)
        assert err <= 1e-7, (gamma, err)


@pytest.mark.parametrize("alpha,gamma", [(1.0, 1e2), (3.0, 1e4), (0.25, 1.0), (7.0, 0.0)])
def test_closed_form_identity_blocks(alpha, gamma):
    """H~ = alpha I, J = [I 0]: dx1 = r_y, dy = r_x1 - alpha r_y, dx2 = r_x2/alpha,
    and S = I/(alpha+gamma) so CG stops after exactly one product."""
    n, m = 12, 5
    rng = np.random.default_rng(7)
    rx, ry = rng.standard_normal(n), rng.standard_normal(m)
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    sys = make_sys(alpha * np.eye(n), J, rx, ry, gamma=gamma)
    _, _, dx, dy, info = O.solve_system(sys)
    np.testing.assert_allclose(dx[:m], ry, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(dx[m:], rx[m:] / alpha, rtol=1e-13)
    np.testing.assert_allclose(dy, rx[:m] - alpha * ry, rtol=1e-12, atol=1e-12)
    assert info["iters"] == 1


def test_zero_rhs_gives_zero_and_no_iterations():
    sys = W.random_tiny_system(3)
    sys.r_x[:] = 0
    sys.r_y[:] = 0
    _, _, dx, dy, info = O.solve_system(sys)
    assert info["iters"] == 0 and not dx.any() and not dy.any()


# ----------------------------------------------------------------- inertia
@pytest.mark.parametrize("seed", range(10))
def test_inertia_when_cholesky_succeeds(seed):
    """Cholesky success + full-rank J  =>  inertia (n, m, 0) (Thm 1 and Thm 3)."""
    sys = W.random_tiny_system(seed + 200, spd=False)
    sys.gamma = 1e4
    sym = sym_of(sys)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, sys.gamma)
    ev = np.linalg.eigvalsh(dense_K(sys, 0.0))
    J = dense_J(sys)
    full_rank = np.linalg.matrix_rank(J) == sys.m
    Hg = dense_H(sys) + sys.gamma * J.T @ J
    spd = np.linalg.eigvalsh(Hg).min() > 0
    assert fac.ok == spd
    if fac.ok and full_rank:
        assert (ev > 0).sum() == sys.n and (ev < 0).sum() == sys.m
        _, _, info = fac.solve(sys.r_x, sys.r_y)
        assert info["inertia_ok"]


def test_thm1_gamma_threshold():
    """H~ = diag(-1, 1, ...), J = [I_m 0]: lambda_min(H~) = -1 and
    lambda_min*(J^T J) = 1, so H_gamma is SPD exactly when gamma > 1 (Thm 1)."""
    n, m = 8, 3
    H = np.eye(n)
    H[0, 0] = -1.0
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    sys = make_sys(H, J, np.ones(n), np.ones(m))
    sym = sym_of(sys)
    for gamma, ok in ((0.5, False), (0.999, False), (1.001, True), (10.0, True), (1e6, True)):
        assert O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, gamma).ok == ok, gamma


def test_indefinite_on_nullspace_fails_for_every_gamma():
    """H~ negative on a null(J) direction: no gamma makes H_gamma SPD (Thm 1)."""
    n, m = 8, 3
    H = np.eye(n)
    H[5, 5] = -0.5                 # e_5 is in null(J)
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    sys = make_sys(H, J, np.ones(n), np.ones(m))
    sym = sym_of(sys)
    for gamma in (0.0, 1.0, 1e4, 1e8):
        f = O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, gamma)
        assert not f.ok
    # a diagonal shift delta > 0.5 restores SPD (Sec. 4.1, H_delta = H_gamma + delta_1 I)
    assert O.Factor(sym, sys.H_vals, sys.J_vals, 0.6, 1e4).ok


def test_rank_deficient_J_triggers_delta2_and_clears_inertia():
    """A duplicated J row makes S singular; an inconsistent r_y makes CG meet a
    small quadratic form, restart on S + delta_2 I, and drop the inertia flag
    (Sec. 4.1 delta_2; Thm 3 needs delta_2 = 0)."""
    n, m = 10, 4
    rng = np.random.default_rng(3)
    J = np.zeros((m, n))
    J[np.arange(3), np.arange(3)] = 1.0
    J[:3, 3:6] = rng.standard_normal((3, 3))
    J[3] = J[0]
    sys = make_sys(np.eye(n) * 2.0, J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e2)
    sym = sym_of(sys)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, sys.gamma)
    assert fac.ok
    dx, dy, info = fac.solve(sys.r_x, sys.r_y, delta2=1e-6)
    assert info["delta2"] == 1e-6 and not info["inertia_ok"]
    # the restarted CG solved (S + delta2 I) dy = J w - r_y
    S = J @ np.linalg.solve(2 * np.eye(n) + sys.gamma * J.T @ J, J.T)
    rhat = sys.r_x + sys.gamma * J.T @ sys.r_y
    w = np.linalg.solve(2 * np.eye(n) + sys.gamma * J.T @ J, rhat)
    ref = np.linalg.solve(S + 1e-6 * np.eye(m), J @ w - sys.r_y)
    assert np.linalg.norm(dy - ref) <= 1e-6 * np.linalg.norm(ref)


# ----------------------------------------------------------------- convergence theory
def test_thm4_eigenvalues_cluster_at_one():
    """eig(gamma S) -> 1 with an error O(1/gamma) (Thm 4)."""
    sys = W.random_tiny_system(11, n_lo=30, n_hi=30)
    H, J = dense_H(sys), dense_J(sys)
    errs = []
    for gamma in (1e3, 1e4, 1e5, 1e6):
        S = J @ np.linalg.solve(H + gamma * J.T @ J, J.T)
        ev = np.linalg.eigvalsh(gamma * (S + S.T) / 2)
        errs.append(np.abs(ev - 1).max())
    for a, b in zip(errs, errs[1:]):
        assert 5.0 <= a / b <= 20.0          # decays like 1/gamma


@pytest.mark.parametrize("gamma", [1e2, 1e4])
def test_cg_iterations_within_cgconv_bound(gamma):
    """CG iterations obey eq. CGconv: ||r_k||/||r_0|| <= sqrt(k(S)) * 2((sqrt k - 1)/(sqrt k + 1))^k."""
    sys = W.random_tiny_system(21, n_lo=40, n_hi=40, gamma=gamma)
    H, J = dense_H(sys), dense_J(sys)
    S = J @ np.linalg.solve(H + gamma * J.T @ J, J.T)
    ev = np.linalg.eigvalsh((S + S.T) / 2)
    kappa = ev.max() / ev.min()
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    k_bound = 1
    while 2 * np.sqrt(kappa) * q ** k_bound > 1e-12:
        k_bound += 1
    _, _, _, _, info = O.solve_system(sys)
    assert 1 <= info["iters"] <= k_bound + 1


# ----------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("seed", range(10))
def test_cholesky_equals_dense_cholesky(seed):
    """L L^T = P (H~ + delta I + gamma J^T J) P^T; L equals numpy's Cholesky."""
    sys = W.random_tiny_system(seed + 300)
    delta, gamma = 1e-3, 50.0
    sym = sym_of(sys)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, delta, gamma)
    assert fac.ok
    Lp, Li, Lx = fac.L_csc()
    n = sys.n
    L = np.zeros((n, n))
    for j in range(n):
        L[Li[Lp[j]:Lp[j + 1]], j] = Lx[Lp[j]:Lp[j + 1]]
    J = dense_J(sys)
    A = dense_H(sys) + delta * np.eye(n) + gamma * J.T @ J
    p = sym.perm
    PA = A[np.ix_(p, p)]
    Lref = np.linalg.cholesky(PA)
    assert np.abs(L - Lref).max() <= 1e-12 * np.abs(Lref).max()
    assert np.linalg.norm(L @ L.T - PA) <= 1e-14 * n * np.linalg.norm(PA)


def test_hsolve_is_inverse():
    sys = W.random_tiny_system(5)
    sym = sym_of(sys)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, sys.gamma)
    J = dense_J(sys)
    A = dense_H(sys) + sys.gamma * J.T @ J
    b = np.arange(sys.n, dtype=float)
    np.testing.assert_allclose(fac.hsolve(b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------- symbolic
@pytest.mark.parametrize("seed", range(40))
def test_symbolic_equals_bruteforce_elimination(seed):
    """Pattern of L, etree (= first off-diagonal row per column) and column
    counts match dense boolean elimination in the oracle's permutation."""
    sys = W.random_tiny_system(seed + 400, n_lo=5, n_hi=45, density=0.1)
    sym = sym_of(sys)
    p = sym.perm
    assert sorted(p.tolist()) == list(range(sys.n))
    Lb = brute_symbolic(sys.n, adjacency_dense(sys), p)
    Lp, Li = sym.l_pattern()
    got = np.zeros_like(Lb)
    for j in range(sys.n):
        got[Li[Lp[j]:Lp[j + 1]], j] = True
    assert (got == Lb).all()
    par = sym.parent
    for j in range(sys.n):
        rows = np.nonzero(Lb[:, j])[0]
        assert par[j] == (rows.min() if rows.size else -1)
    np.testing.assert_array_equal(sym.colcount, Lb.sum(0) + 1)


@pytest.mark.parametrize("seed", range(15))
def test_postorder_makes_subtrees_contiguous(seed):
    sys = W.random_tiny_system(seed + 500, n_lo=20, n_hi=60, density=0.05)
    sym = sym_of(sys)
    par = sym.parent
    n = sys.n
    size = np.ones(n, int)
    for j in range(n):          # children precede parents
        assert par[j] == -1 or par[j] > j
        if par[j] >= 0:
            size[par[j]] += size[j]
    for j in range(n):
        # the descendants of j are exactly j-size+1 .. j
        lo = j - size[j] + 1
        for k in range(lo, j):
            a = k
            while a != -1 and a < j:
                a = par[a]
            assert a == j


def _amd_case(name):
    with open(os.path.join(GOLDEN, "amd_hand_worked.json")) as f:
        return json.load(f)[name]


@pytest.mark.parametrize("name", ["path5", "star5", "clique4", "two_triangles", "grid2x3"])
def test_amd_hand_worked(name):
    """Hand-worked orders of the pinned AMD rules (Sec. 5.3 names AMD;
    the rules are those of Amestoy, Davis and Duff 1996 with pinned ties)."""
    case = _amd_case(name)
    sys = graph_sys(case["n"], [tuple(e) for e in case["edges"]])
    assert sym_of(sys).amd_order.tolist() == case["order"]


@pytest.mark.parametrize("name", ["nd_path10_leaf2", "nd_star7_leaf2"])
def test_nd_hand_worked(name):
    case = _amd_case(name)
    sys = graph_sys(case["n"], [tuple(e) for e in case["edges"]])
    assert sym_of(sys, ordering="nd", nd_leaf=case["leaf"]).amd_order.tolist() == case["order"]


@pytest.mark.parametrize("seed", range(10))
def test_nd_is_a_permutation_and_separators_come_last(seed):
    """Every ND separator vertex is numbered after both parts it separates:
    so no vertex is adjacent to a later-numbered vertex of a *different*
    earlier part. Checked through the symbolic result: the etree built on
    the ND order is valid and the fill matches brute-force elimination."""
    sys = W.random_tiny_system(seed + 700, n_lo=30, n_hi=90, density=0.05)
    sym = sym_of(sys, ordering="nd", nd_leaf=4)
    assert sorted(sym.amd_order.tolist()) == list(range(sys.n))
    Lb = brute_symbolic(sys.n, adjacency_dense(sys), sym.perm)
    np.testing.assert_array_equal(sym.colcount, Lb.sum(0) + 1)


def test_nd_shortens_the_elimination_tree_on_the_grid():
    """On the 200 x 100 grid workload nested dissection gives a much shorter
    elimination tree than AMD (the reason to offer it on a GPU)."""
    sys = W.make_config("grid2d_n20k")
    def height(sym):
        par = sym.parent
        d = np.zeros(sys.n, int)
        for j in range(sys.n - 1, -1, -1):
            d[j] = d[par[j]] + 1 if par[j] >= 0 else 1
        return d.max()
    assert 2 * height(sym_of(sys, ordering="nd")) < height(sym_of(sys))


@pytest.mark.parametrize("seed", range(10))
def test_amd_zero_fill_on_trees(seed):
    """Minimum degree eliminates leaves first, so a tree gets no fill."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 80))
    lab = rng.permutation(n)
    edges = [(int(lab[i]), int(lab[rng.integers(0, i)])) for i in range(1, n)]
    sys = graph_sys(n, edges)
    sym = sym_of(sys)
    assert sym.nnzL == n + len(edges)


def test_amd_clique_is_identity_and_one_supernode():
    n = 9
    edges = [(a, b) for a in range(n) for b in range(a)]
    sym = sym_of(graph_sys(n, edges))
    assert sym.amd_order.tolist() == list(range(n))
    assert sym.nsuper == 1


def test_amd_beats_natural_on_grid():
    """AMD gives less fill than the natural order (Sec. 5.3 comparison)."""
    sys = W.make_config("grid2d_n2000")
    a = sym_of(sys)
    b = sym_of(sys, ordering="natural")
    assert a.nnzL < b.nnzL


# ----------------------------------------------------------------- supernodes
@pytest.mark.parametrize("seed", range(12))
def test_supernodes_cover_structure(seed):
    """Supernodes partition the columns into contiguous ranges; each row
    list holds its columns and contains the structure of every column; the
    supernodal parent is the supernode of the etree parent of its last column."""
    sys = W.random_tiny_system(seed + 600, n_lo=20, n_hi=60, density=0.08)
    for relax in ((1, 0, 1, 256), (16, 1, 10, 256), (4, 1, 2, 8)):
        sym = sym_of(sys, relax_small=relax[0], relax_num=relax[1], relax_den=relax[2], wmax=relax[3])
        start, rowptr, rows, spar = sym.supernodes()
        Lp, Li = sym.l_pattern()
        par = sym.parent
        assert start[0] == 0 and start[-1] == sys.n and (np.diff(start) > 0).all()
        col2sn = np.repeat(np.arange(sym.nsuper), np.diff(start))
        zeros = 0
        for s in range(sym.nsuper):
            f, l = start[s], start[s + 1] - 1
            R = rows[rowptr[s]:rowptr[s + 1]]
            assert (np.diff(R) > 0).all()
            assert R[:l - f + 1].tolist() == list(range(f, l + 1))
            for j in range(f, l + 1):
                assert set(Li[Lp[j]:Lp[j + 1]].tolist()) <= set(R.tolist())
            W_ = l - f + 1
            panel = W_ * (W_ + 1) // 2 + W_ * (len(R) - W_)
            zeros_s = panel - sum(Lp[j + 1] - Lp[j] + 1 for j in range(f, l + 1))
            zeros += zeros_s
            if relax[0] == 1 and relax[1] == 0:
                assert zeros_s == 0           # fundamental supernodes hold no explicit zeros
            assert W_ <= max(relax[3], 1) or zeros_s == 0
            assert spar[s] == (col2sn[par[l]] if par[l] >= 0 else -1)


# ----------------------------------------------------------------- residual definitions
def test_rr_be_definitions():
    """RR = ||K x - b|| / ||b||, BE = ||K x - b|| / (||K||_inf ||x|| + ||b||) (Sec. 5.1)."""
    sys = W.random_tiny_system(8)
    K = dense_K(sys)
    b = np.concatenate([sys.r_x, sys.r_y])
    x = np.linalg.solve(K, b)
    sym = sym_of(sys)
    exact = O.residual(sym, sys.H_vals, sys.J_vals, sys.delta, sys.r_x, sys.r_y, x[:sys.n], x[sys.n:])
    assert exact["rr"] < 1e-13 and exact["be"] <= exact["rr"]
    assert exact["knorm"] == pytest.approx(np.abs(K).sum(1).max(), rel=1e-14)
    e = np.zeros_like(x)
    e[0] = 1e-3
    pert = O.residual(sym, sys.H_vals, sys.J_vals, sys.delta, sys.r_x, sys.r_y, (x + e)[:sys.n], (x + e)[sys.n:])
    res = np.linalg.norm(K @ (x + e) - b)
    assert pert["rr"] == pytest.approx(res / np.linalg.norm(b), rel=1e-8)
    assert pert["be"] == pytest.approx(res / (np.abs(K).sum(1).max() * np.linalg.norm(x + e) + np.linalg.norm(b)), rel=1e-8)


# ----------------------------------------------------------------- 4x4 reduction
@pytest.mark.parametrize("seed", range(5))
def test_4x4_reduction_matches_dense(seed):
    """Eliminating ds, dy_d (Sec. 3, eq. linsys2x2) and recovering them
    reproduces the dense solve of the 4x4 system (eq. linsys4x4)."""
    p = W.random_4x4_parts(seed, n_x=20, m_c=6, m_d=5)
    Hp, Hi, Hv, r_x = O.reduce4x4(p)
    n, mc, md = p["n_x"], p["m_c"], p["m_d"]
    sys = W.KKTSystem(n, mc, Hp, Hi, Hv, p["J_rowptr"], p["J_colidx"], p["J_vals"], r_x,
                      p["r_y"], 0.0, 1e2)
    _, _, dx, dy, info = O.solve_system(sys)
    assert info["status"] == 0
    ds, dyd = O.recover4x4(p, dx)
    # dense 4x4
    H = np.zeros((n, n))
    for j in range(n):
        for q in range(Hp.size and p["H_colptr"][j], p["H_colptr"][j + 1]):
            i = p["H_rowidx"][q]
            H[i, j] += p["H_vals"][q]
            if i != j:
                H[j, i] += p["H_vals"][q]
    J = np.zeros((mc, n))
    for r in range(mc):
        for q in range(p["J_rowptr"][r], p["J_rowptr"][r + 1]):
            J[r, p["J_colidx"][q]] = p["J_vals"][q]
    Jd = np.zeros((md, n))
    for r in range(md):
        for q in range(p["Jd_rowptr"][r], p["Jd_rowptr"][r + 1]):
            Jd[r, p["Jd_colidx"][q]] = p["Jd_vals"][q]
    N = n + md + mc + md
    K = np.zeros((N, N))
    K[:n, :n] = H + np.diag(p["D_x"])
    K[n:n + md, n:n + md] = np.diag(p["D_s"])
    K[:n, n + md:n + md + mc] = J.T
    K[:n, n + md + mc:] = Jd.T
    K[n:n + md, n + md + mc:] = -np.eye(md)
    K[n + md:n + md + mc, :n] = J
    K[n + md + mc:, :n] = Jd
    K[n + md + mc:, n:n + md] = -np.eye(md)
    rhs = np.concatenate([p["r_xt"], p["r_s"], p["r_y"], p["r_yd"]])
    ref = np.linalg.solve(K, rhs)
    got = np.concatenate([dx, ds, dy, dyd])
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


# ----------------------------------------------------------------- the small workload
def test_small_grid_workload_against_sparse_lu():
    """50x40 grid workload: RR <= 1e-8 on K_delta, CG iterations O(10)
    (Sec. 5: < 20 on average), inertia flag set, and agreement with a
    sparse LU solve of the full KKT matrix (scipy SuperLU)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    sys = W.make_config("grid2d_n2000")
    sym, fac, dx, dy, info = O.solve_system(sys)
    assert info["status"] == 0 and info["inertia_ok"]
    assert info["rr"] <= 1e-8 and info["iters"] <= 20
    n, m = sys.n, sys.m
    H = sp.csc_matrix((sys.H_vals, sys.H_rowidx, sys.H_colptr), shape=(n, n))
    H = H + sp.tril(H, -1).T + sys.delta * sp.eye(n)
    J = sp.csr_matrix((sys.J_vals, sys.J_colidx, sys.J_rowptr), shape=(m, n))
    K = sp.bmat([[H, J.T], [J, None]]).tocsc()
    ref = spl.spsolve(K, np.concatenate([sys.r_x, sys.r_y]))
    got = np.concatenate([dx, dy])
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)


def test_grid_4x4_reduction_matches_sparse_lu():
    """The 4x4 form on the 50x40 grid (J_d with n/4 local rows, D_s over
    eight decades): reduction + 2x2 solve + recovery (Sec. 3) equals a
    sparse LU solve of the full eq. linsys4x4 matrix with delta on the
    H + D_x block."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    p = W.grid_4x4_parts("grid2d_n2000")
    Hp, Hi, Hv, r_x = O.reduce4x4(p)
    n, mc, md = p["n_x"], p["m_c"], p["m_d"]
    s = W.KKTSystem(n, mc, Hp, Hi, Hv, p["J_rowptr"], p["J_colidx"], p["J_vals"], r_x, p["r_y"], p["delta"],
                    p["gamma"])
    _, _, dx, dy, info = O.solve_system(s)
    assert info["status"] == 0
    ds, dyd = O.recover4x4(p, dx)
    H = sp.csc_matrix((p["H_vals"], p["H_rowidx"], p["H_colptr"]), shape=(n, n))
    H = H + sp.tril(H, -1).T
    J = sp.csr_matrix((p["J_vals"], p["J_colidx"], p["J_rowptr"]), shape=(mc, n))
    Jd = sp.csr_matrix((p["Jd_vals"], p["Jd_colidx"], p["Jd_rowptr"]), shape=(md, n))
    I = sp.eye(md)
    K4 = sp.bmat([[H + sp.diags(p["D_x"]) + p["delta"] * sp.eye(n), None, J.T, Jd.T],
                  [None, sp.diags(p["D_s"]), None, -I], [J, None, None, None], [Jd, -I, None, None]]).tocsc()
    b = np.concatenate([p["r_xt"], p["r_s"], p["r_y"], p["r_yd"]])
    ref = spl.splu(K4).solve(b)
    got = np.concatenate([dx, ds, dy, dyd])
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(b - K4 @ got) <= 1e-10 * np.linalg.norm(b)


# ----------------------------------------------------------------- Algorithm 1's delta_1 loop
def nullspace_indefinite_system(lam, n=30, m=10, seed=3):
    """H~ with eigenvalue lam along a unit v in null(J) (all other eigenvalues
    >= 1), so H_gamma has lam as its smallest eigenvalue for every gamma."""
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((m, n))
    _, _, Vt = np.linalg.svd(J)
    v = Vt[m]                                   # in null(J)
    P = np.eye(n) - np.outer(v, v)
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)
    H = P @ A @ P + lam * np.outer(v, v)
    H = (H + H.T) / 2
    return make_sys(H, J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e2), H, J


@pytest.mark.parametrize("lam,expect_delta,expect_ok", [(0.5, 0.0, True), (-2.5e-8, 3.2e-8, True),
                                                        (-1e-5, 5.12e-7, False)])
def test_factor_regularized_loop(lam, expect_delta, expect_ok):
    """delta_1 = 0, then delta_min = 1e-9 doubling while the Cholesky fails and
    delta_1 <= delta_max / 2 = 5e-7: the first trial value above -lam."""
    sys, H, J = nullspace_indefinite_system(lam)
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    fac, d1 = O.factor_regularized(sym, sys.H_vals, sys.J_vals, sys.gamma)
    assert fac.ok == expect_ok
    assert d1 == pytest.approx(expect_delta, rel=1e-12, abs=0)
    # Thm 1: the smallest eigenvalue of H_gamma + delta_1 I decides
    lmin = np.linalg.eigvalsh(H + sys.gamma * J.T @ J + d1 * np.eye(sys.n)).min()
    assert (lmin > 0) == expect_ok


def test_factor_regularized_sequence_carries_delta():
    """Sec. 4.1: for each next matrix delta_1 starts at 0 and, if that
    Cholesky fails, is set back to the previous matrix's value (then doubled
    while it still fails); after a matrix that needed no shift the first
    retry is delta_min, as in Algorithm 1. The smallest eigenvalue of H_gamma
    is lam along a null(J) direction, so the accepted shifts follow by hand:
    -2.5e-8 -> 1e-9 * 2^5 = 3.2e-8; -1e-8 -> back to 3.2e-8 (from scratch it
    would be 1.6e-8); 0.5 -> 0; -5e-9 -> 1e-9 * 2^3 = 8e-9; -5e-8 -> 8e-9 *
    2^3 = 6.4e-8."""
    lams = [-2.5e-8, -1e-8, 0.5, -5e-9, -5e-8]
    want = [3.2e-8, 3.2e-8, 0.0, 8e-9, 6.4e-8]
    prev = 0.0
    for lam, w in zip(lams, want):
        sys, H, J = nullspace_indefinite_system(lam)
        sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
        fac, d1 = O.factor_regularized(sym, sys.H_vals, sys.J_vals, sys.gamma, delta_prev=prev)
        assert fac.ok
        assert d1 == pytest.approx(w, rel=1e-12, abs=0)
        assert np.linalg.eigvalsh(H + sys.gamma * J.T @ J + d1 * np.eye(sys.n)).min() > 0
        prev = d1


# ----------------------------------------------------------------- Ruiz scaling (Sec. 4.1)
def _dense_rownorms(sys, Dx, Dy):
    K = dense_K(sys, delta=0.0)
    D = np.concatenate([Dx, Dy])
    return np.abs(D[:, None] * K * D[None, :]).max(1)


def test_ruiz_diagonal_closed_form():
    """K = diag(a) (no constraints): one iteration gives D = 1/sqrt(a) and
    unit rows; further iterations keep D (rows already at norm 1)."""
    rng = np.random.default_rng(2)
    a = 10.0 ** rng.uniform(-6, 6, 9)
    sys = make_sys(np.diag(a), np.zeros((0, 9)), np.ones(9), np.zeros(0))
    Dx, Dy = O.ruiz_scaling(sys, 1)
    np.testing.assert_array_equal(Dx, 1.0 / np.sqrt(a))
    np.testing.assert_allclose(_dense_rownorms(sys, Dx, Dy), 1.0, rtol=4e-16)
    np.testing.assert_allclose(O.ruiz_scaling(sys, 5)[0], Dx, rtol=4e-16)


def test_ruiz_leaves_an_equilibrated_matrix_alone():
    """Every row of K already has infinity norm exactly 1 (entries in [-1, 1]
    and a +-1 in each row): D stays the identity. (A 2-norm variant would
    move it.)"""
    rng = np.random.default_rng(3)
    n, m = 12, 4
    H = rng.uniform(-0.9, 0.9, (n, n))
    H = (H + H.T) / 2
    np.fill_diagonal(H, 1.0)
    J = np.zeros((m, n))
    c1 = rng.choice(n, m, replace=False)
    J[np.arange(m), c1] = -1.0
    J[np.arange(m), (c1 + 1 + rng.integers(0, n - 1, m)) % n] = 0.5     # another column of the row
    sys = make_sys(H, J, np.ones(n), np.ones(m))
    Dx, Dy = O.ruiz_scaling(sys, 7)
    assert (Dx == 1.0).all() and (Dy == 1.0).all()


@pytest.mark.parametrize("seed", range(8))
def test_ruiz_rows_converge_to_unit_norm(seed):
    """Rows of D K D approach unit infinity norm (Ruiz's convergence for
    symmetric matrices), checked on the dense matrix: within 1e-3 after 30
    iterations, from barriers spread over 12 decades."""
    sys = W.random_tiny_system(seed + 900, n_lo=10, n_hi=60, density=0.1)
    sys.H_vals = sys.H_vals * (10.0 ** np.random.default_rng(seed).uniform(-6, 6, sys.H_vals.size))
    Dx, Dy = O.ruiz_scaling(sys, 30)
    r = _dense_rownorms(sys, Dx, Dy)
    assert np.abs(r - 1).max() <= 1e-3


@pytest.mark.parametrize("seed", range(6))
def test_ruiz_scaled_solve_recovers_the_original_solution(seed):
    """With delta = 0 the scaled system D K D x^ = D b is the original one in
    other variables: the oracle's scaled solve, unscaled by D, equals a dense
    LU solve of K x = b (the gamma form of Sec. 4 is applied to the scaled
    system)."""
    sys = W.random_tiny_system(seed + 950, n_lo=10, n_hi=80, density=0.08)
    sys.delta = 0.0
    Dx, Dy = O.ruiz_scaling(sys, 10)
    sc = O.scale_system(sys, Dx, Dy)
    _, _, dxh, dyh, info = O.solve_system(sc, ir_maxit=2)
    got = np.concatenate([Dx * dxh, Dy * dyh])
    ref = np.linalg.solve(dense_K(sys, 0.0), np.concatenate([sys.r_x, sys.r_y]))
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


# ----------------------------------------------------------------- Krylov variants (Sec. 4)
@pytest.mark.parametrize("method", ["pcg", "minres"])
@pytest.mark.parametrize("seed", range(6))
def test_schur_variants_match_dense_lu(method, seed):
    """PCG with M = (J J^T)^-1 J H_gamma J^T (J J^T)^-1 and MINRES on eq.
    Schur1 reach the dense LU solution of K_delta."""
    sys = W.random_tiny_system(seed + 1200, n_lo=20, n_hi=90, density=0.08)
    sym = sym_of(sys)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    assert fac.ok
    dx, dy, it = O.schur_variant(fac, sys, method)
    ref = np.linalg.solve(dense_K(sys), np.concatenate([sys.r_x, sys.r_y]))
    assert np.linalg.norm(np.concatenate([dx, dy]) - ref) <= 1e-9 * np.linalg.norm(ref)
    assert 1 <= it <= sys.m + 2


@pytest.mark.parametrize("seed", range(4))
def test_pcg_with_square_j_converges_in_one_step(seed):
    """With J square (m = n) the preconditioner is exactly S^-1 (Sec. 4:
    M gives the exact solution when J is square), so PCG stops after one
    product."""
    rng = np.random.default_rng(seed)
    n = 15
    A = rng.standard_normal((n, n))
    H = A @ A.T + n * np.eye(n)
    J = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    sys = make_sys(H, J, rng.standard_normal(n), rng.standard_normal(n), gamma=10.0)
    fac = O.Factor(sym_of(sys), sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    dx, dy, it = O.schur_variant(fac, sys, "pcg")
    assert it == 1
    ref = np.linalg.solve(dense_K(sys), np.concatenate([sys.r_x, sys.r_y]))
    assert np.linalg.norm(np.concatenate([dx, dy]) - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("alpha,gamma", [(1.0, 1e2), (3.0, 1e4)])
def test_minres_on_identity_schur_complement_takes_one_step(alpha, gamma):
    """H~ = alpha I, J = [I 0]: S = I / (alpha + gamma), a multiple of the
    identity, so the first Lanczos step spans the solution."""
    n, m = 12, 5
    rng = np.random.default_rng(9)
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    sys = make_sys(alpha * np.eye(n), J, rng.standard_normal(n), rng.standard_normal(m), gamma=gamma)
    fac = O.Factor(sym_of(sys), sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    dx, dy, it = O.schur_variant(fac, sys, "minres")
    assert it == 1
    np.testing.assert_allclose(dy, sys.r_x[:m] - alpha * sys.r_y, rtol=1e-11, atol=1e-11)
