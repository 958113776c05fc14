"""CUDA path vs the CPU oracle (needs a B300). Every call goes through the
C ABI of libkkt.so. Tolerances: FP64 method on the workloads -- relative KKT
residual <= 1e-8 and solution relative difference <= 1e-6 (the stated
accuracy target); tiny well-conditioned systems -- 1e-9 on the solution."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2110_03636_b300 as K  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device=DEV)


def gpu_solve(sys, precision="fp64", delta=None, gamma=None, **opt):
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision=precision, **opt)
    code = s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta if delta is None else delta,
                    sys.gamma if gamma is None else gamma, check=False)
    if code != 0:
        return s, code, None, None
    dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y), check=False)
    torch.cuda.synchronize()
    return s, 0, dx.cpu().numpy(), dy.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiny_systems_match_oracle(seed, precision):
    sys = W.random_tiny_system(seed, n_lo=3, n_hi=120, density=0.08)
    _, _, odx, ody, oinfo = O.solve_system(sys)
    s, code, dx, dy = gpu_solve(sys, precision)
    assert code == 0
    info = s.info
    assert info.cg_status == 0
    # FP64 solves to 1e-12; the mixed form refines until RR <= 1e-9 (its default stop)
    rr_max, sol = (1e-10, 1e-9) if precision == "fp64" else (1e-9, 1e-7)
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= sol
    assert info.rr <= rr_max
    r = O.residual(O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx),
                   sys.H_vals, sys.J_vals, sys.delta, sys.r_x, sys.r_y, dx, dy)
    assert r["rr"] <= rr_max
    if precision == "fp64":
        assert abs(info.cg_iters - oinfo["iters"]) <= 1
    assert s.inertia_ok


@pytest.mark.parametrize("seed", range(6))
def test_factor_panels_match_oracle_cholesky(seed):
    """The FP64 supernodal factor holds the oracle's L entry by entry."""
    sys = W.random_tiny_system(seed + 50, n_lo=40, n_hi=160, density=0.06)
    delta, gamma = 1e-3, 30.0
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    s.factor(cu(sys.H_vals), cu(sys.J_vals), delta, gamma)
    panels = s.panels()
    g = s.symbolic()
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, delta, gamma)
    Lp, Li, Lx = fac.L_csc()
    start, rowptr, rows = g["sn_start"], g["sn_rowptr"], g["sn_rows"]
    off = 0
    worst = 0.0
    scale = np.abs(Lx).max()
    for sn in range(len(start) - 1):
        w = start[sn + 1] - start[sn]
        R = rows[rowptr[sn]:rowptr[sn + 1]]
        nr = len(R)
        ld = (nr + 3) // 4 * 4
        P = panels[off:off + w * ld].reshape(w, ld).T[:nr]
        pos = {r: i for i, r in enumerate(R)}
        for jj in range(w):
            j = start[sn] + jj
            col = np.zeros(nr)
            for q in range(Lp[j], Lp[j + 1]):
                col[pos[Li[q]]] = Lx[q]
            col[:jj] = P[:jj, jj]          # upper part of the diagonal block is not used
            worst = max(worst, np.abs(P[:, jj] - col).max())
        off += w * ld
    assert worst <= 1e-12 * scale


def panel_error_vs_oracle(s, sys, ordering="natural"):
    """max |panel entry - oracle L entry| over the stored lower trapezoids of
    every supernode (explicit zeros of relaxed supernodes compare with 0),
    and max |oracle L|."""
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, ordering=ordering)
    f = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    assert f.ok
    Lp, Li, Lx = f.L_csc()
    pan = s.panels()
    st, rp, rows, _ = sym.supernodes()
    off, worst = 0, 0.0
    for k in range(len(st) - 1):
        w, nr = st[k + 1] - st[k], rp[k + 1] - rp[k]
        ld = (nr + 3) // 4 * 4
        R = rows[rp[k]:rp[k + 1]]
        pos = {int(r): i for i, r in enumerate(R)}
        blk = pan[off:off + w * ld].reshape(w, ld)[:, :nr].T.copy()     # nr x w
        ref = np.zeros_like(blk)
        for c in range(w):
            col = st[k] + c
            q0, q1 = Lp[col], Lp[col + 1]
            ref[[pos[int(r)] for r in Li[q0:q1]], c] = Lx[q0:q1]
        worst = max(worst, float(np.abs(np.tril(blk - ref)).max()))
        off += w * ld
    return worst, float(np.abs(Lx).max())


def block_front_system(wa=600, seed=5):
    """n = wa + 400, natural order: block A (columns 0..wa-1) and block B
    (the next 100) are dense and both couple densely to block C (the last
    300), A and B do not couple. The etree gives fundamental supernodes A
    (wa columns, 300 rows below), B (100 columns, 300 below) and C; B + C is
    wider than the relaxation limit and A is not C's last child, so A stays
    a wa-column front: its update matrix is a K = wa product of 300 rows
    (ragged 128-row tiles). J rows stay inside one block."""
    from test_oracle import make_sys
    rng = np.random.default_rng(seed)
    n, m = wa + 400, 60
    blocks = [(0, wa), (wa, wa + 100), (wa + 100, n)]
    mask = np.zeros((n, n), bool)
    for lo, hi in blocks:
        mask[lo:hi, lo:hi] = True
    mask[0:wa + 100, wa + 100:n] = True
    mask = mask | mask.T
    H = np.where(mask, rng.uniform(-1, 1, (n, n)), 0.0) / np.sqrt(n)
    H = np.triu(H, 1)
    H = H + H.T
    H[np.arange(n), np.arange(n)] = np.abs(H).sum(1) + rng.uniform(0.5, 2.0, n)
    J = np.zeros((m, n))
    cols = rng.choice(n, m, replace=False)
    J[np.arange(m), cols] = 1.0
    for r, c in enumerate(cols):
        lo, hi = next(b for b in blocks if b[0] <= c < b[1])
        J[r, rng.integers(lo, hi)] += rng.standard_normal()
    return make_sys(H, J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e2)


@pytest.mark.parametrize("wa", [600, 1100])
def test_tensor_core_updates_match_oracle_on_a_wide_front(wa):
    """The FP32 factor with the tcgen05 split-TF32 updates (three products,
    tensor-memory accumulation drained to FP32 registers per 64 K) against
    the FP64 oracle's L, entry by entry, on a front with K = wa and 300
    update rows (wa = 1100 also takes the in-panel update beyond each
    128-column outer block on the tensor cores): within FP32 rounding of the
    largest entry, and no worse than 4x the FP32 FMA factor's own error.
    Both solve to the oracle's solution."""
    sys = block_front_system(wa)
    _, _, odx, ody, oinfo = O.solve_system(sys, ordering="natural")
    assert oinfo["status"] == 0
    errs = {}
    for tcs in (1, 0):
        s, code, dx, dy = gpu_solve(sys, "mixed", ordering="natural", tensor_cores=tcs)
        assert code == 0
        g = K.kkt_get_symbolic(s.h)
        st = g["sn_start"]
        assert wa in np.diff(st)                      # the wide front exists
        err, lmax = panel_error_vs_oracle(s, sys)
        errs[tcs] = err
        assert err <= 2e-5 * lmax, (tcs, err, lmax)
        assert s.info.rr <= 1e-9
        assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6
        s.close()
    assert errs[1] <= 4 * errs[0] + 1e-7 * lmax, errs


@pytest.mark.parametrize("name", ["grid2d_n20k", "grid2d_n2000"])
def test_tensor_core_factor_solves_grid_to_oracle(name):
    """Grid workloads with the tensor-core updates: the solution matches the
    FP64 oracle's to 1e-6 and RR <= 1e-9."""
    sys = W.make_config(name)
    _, _, odx, ody, _ = O.solve_system(sys, ordering="nd")
    s, code, dx, dy = gpu_solve(sys, "mixed", ordering="nd", tensor_cores=1)
    assert code == 0
    assert s.info.rr <= 1e-9
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("wide,hubs_last", [(40, False), (100, False), (40, True), (300, True)])
def test_wide_front_with_many_row_tiles(precision, wide, hubs_last):
    """Natural ordering of an arrowhead: `wide` hub variables couple to all
    1200 others. Hubs first: one dense supernode of all 1200 + wide columns,
    so every 32-column block step has many row tiles below it. Hubs last:
    1200 one-column fronts whose `wide` x `wide` update matrices (128-tile
    SYRK when wide >= 128) are all extend-added into the hub front. FP64
    panels equal the oracle's L; both precisions reach the oracle's solution."""
    from test_oracle import make_sys
    rng = np.random.default_rng(wide)
    n, m = wide + 1200, 60
    H = np.zeros((n, n))
    H[:wide, wide:] = rng.uniform(-1, 1, (wide, n - wide)) / np.sqrt(n)
    H = H + H.T
    H[np.arange(n), np.arange(n)] = np.abs(H).sum(1) + rng.uniform(0.5, 2.0, n)
    H[:wide, :wide] += rng.uniform(-0.1, 0.1, (wide, wide)) * (rng.random((wide, wide)) < 0.3)
    H[:wide, :wide] = (H[:wide, :wide] + H[:wide, :wide].T) / 2
    H[np.arange(wide), np.arange(wide)] += wide * 0.1
    if hubs_last:
        order = np.r_[wide:n, 0:wide]
        H = H[np.ix_(order, order)]
    J = np.zeros((m, n))
    J[np.arange(m), rng.choice(n, m, replace=False)] = 1.0
    J[np.arange(m), rng.integers(0, n, m)] += rng.standard_normal(m)
    sys = make_sys(H, J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e2)
    _, _, odx, ody, oinfo = O.solve_system(sys, ordering="natural")
    assert oinfo["status"] == 0
    s, code, dx, dy = gpu_solve(sys, precision, ordering="natural")
    assert code == 0
    assert s.info.rr <= (1e-10 if precision == "fp64" else 1e-9)
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= (1e-8 if precision == "fp64" else 1e-6)
    if precision == "fp64":
        sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, ordering="natural")
        f = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
        Lp, Li, Lx = f.L_csc()
        pan = s.panels()
        st, rp, rows, _ = sym.supernodes()
        off, worst = 0, 0.0
        for k in range(len(st) - 1):
            w, nr = st[k + 1] - st[k], rp[k + 1] - rp[k]
            ld = (nr + 3) // 4 * 4
            R = rows[rp[k]:rp[k + 1]]
            for c in range(w):
                col = st[k] + c
                q0, q1 = Lp[col], Lp[col + 1]
                ref = dict(zip(Li[q0:q1], Lx[q0:q1]))
                for r_i in range(c, nr):
                    v = pan[off + c * ld + r_i]
                    worst = max(worst, abs(v - ref.get(R[r_i], 0.0)))
            off += w * ld
        assert worst <= 1e-12 * np.abs(Lx).max()


def test_hsolve_matches_oracle():
    sys = W.make_config("grid2d_n2000")
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    b = np.random.default_rng(1).standard_normal(sys.n)
    x = s.hsolve(cu(b)).cpu().numpy()
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    ref = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma).hsolve(b)
    assert rel(x, ref) <= 1e-9


@pytest.mark.parametrize("ordering", ["amd", "nd"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_n2000_matches_oracle(precision, ordering):
    sys = W.make_config("grid2d_n2000")
    _, _, odx, ody, oinfo = O.solve_system(sys)
    s, code, dx, dy = gpu_solve(sys, precision, ordering=ordering)
    assert code == 0
    info = s.info
    assert info.rr <= 1e-8
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    assert O.residual(sym, sys.H_vals, sys.J_vals, sys.delta, sys.r_x, sys.r_y, dx, dy)["rr"] <= 1e-8
    if precision == "fp64":
        assert abs(info.cg_iters - oinfo["iters"]) <= 1
    assert s.inertia_ok


@pytest.mark.parametrize("ordering,precision", [("amd", "fp64"), ("nd", "fp64"), ("nd", "mixed")])
def test_grid_n20k_and_value_updates(ordering, precision):
    """Four value refactorizations on one resident pattern (interior iterations)."""
    base = W.make_config("grid2d_n20k")
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                    ordering=ordering, precision=precision)
    sym = O.Symbolic(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx)
    sys = base
    for t in range(4):
        if t:
            sys = W.rescale_barrier(sys, seed=(0, t))
        s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
        dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y))
        dx, dy = dx.cpu().numpy(), dy.cpu().numpy()
        fac = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
        odx, ody, _ = fac.solve(sys.r_x, sys.r_y)
        assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6
        assert s.info.rr <= 1e-8


def test_gamma_invariance_on_gpu():
    sys = W.make_config("grid2d_n2000")
    sols = []
    for gamma in (1e2, 1e4, 1e6):
        s, code, dx, dy = gpu_solve(sys, gamma=gamma)
        assert code == 0 and s.info.rr <= 1e-8
        sols.append(np.concatenate([dx, dy]))
    assert rel(sols[0], sols[2]) <= 1e-6 and rel(sols[1], sols[2]) <= 1e-6


def test_closed_form_one_iteration():
    from test_oracle import make_sys
    n, m, alpha = 300, 120, 3.0
    rng = np.random.default_rng(2)
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    sys = make_sys(alpha * np.eye(n), J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e4)
    s, code, dx, dy = gpu_solve(sys)
    assert code == 0 and s.info.cg_iters == 1
    np.testing.assert_allclose(dx[:m], sys.r_y, atol=1e-10)
    np.testing.assert_allclose(dy, sys.r_x[:m] - alpha * sys.r_y, atol=1e-8)


def test_not_spd_reported_and_handle_reusable():
    """Thm 1: H~ negative on null(J) -> NOT_SPD; delta_1 = 0.6 restores SPD (Sec. 4.1)."""
    from test_oracle import make_sys
    n, m = 50, 10
    H = np.eye(n)
    H[30, 30] = -0.5
    J = np.zeros((m, n))
    J[np.arange(m), np.arange(m)] = 1.0
    rng = np.random.default_rng(4)
    sys = make_sys(H, J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e4)
    s, code, _, _ = gpu_solve(sys)
    assert code == 2 and not s.inertia_ok
    with pytest.raises(K.KKTError) as e:
        s.solve(cu(sys.r_x), cu(sys.r_y))
    assert e.value.code == 8
    s.factor(cu(sys.H_vals), cu(sys.J_vals), 0.6, 1e4)
    dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y))
    ref = np.linalg.solve(np.block([[H + 0.6 * np.eye(n), J.T], [J, np.zeros((m, m))]]),
                          np.concatenate([sys.r_x, sys.r_y]))
    assert rel(np.concatenate([dx.cpu().numpy(), dy.cpu().numpy()]), ref) <= 1e-9


def test_rank_deficient_J_uses_delta2_and_clears_inertia():
    from test_oracle import make_sys
    n, m = 60, 8
    rng = np.random.default_rng(3)
    J = np.zeros((m, n))
    J[np.arange(m - 1), np.arange(m - 1)] = 1.0
    J[:m - 1, 20:24] = rng.standard_normal((m - 1, 4))
    J[m - 1] = J[0]
    sys = make_sys(2.0 * np.eye(n), J, rng.standard_normal(n), rng.standard_normal(m), gamma=1e2)
    s, code, dx, dy = gpu_solve(sys, delta2=1e-6, ir_maxit=0)
    assert code == 0
    assert s.info.delta2_used == 1 and not s.inertia_ok
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    _, ody, oinfo = O.Factor(sym, sys.H_vals, sys.J_vals, 0.0, 1e2).solve(sys.r_x, sys.r_y, delta2=1e-6)
    assert oinfo["delta2"] == 1e-6
    assert rel(dy, ody) <= 1e-6


def test_edge_sizes():
    from test_oracle import make_sys
    # n = 1, m = 0
    sys = make_sys(np.array([[4.0]]), np.zeros((0, 1)), np.array([2.0]), np.zeros(0))
    s, code, dx, dy = gpu_solve(sys)
    assert code == 0 and abs(dx[0] - 0.5) < 1e-15 and s.info.cg_iters == 0
    # m = 0, larger n: plain SPD solve
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 40))
    A = A @ A.T + 40 * np.eye(40)
    sys = make_sys(A, np.zeros((0, 40)), rng.standard_normal(40), np.zeros(0))
    s, code, dx, dy = gpu_solve(sys)
    assert code == 0 and rel(dx, np.linalg.solve(A, sys.r_x)) <= 1e-12
    # zero right-hand side
    sys = W.random_tiny_system(9)
    sys.r_x[:] = 0
    sys.r_y[:] = 0
    s, code, dx, dy = gpu_solve(sys)
    assert code == 0 and not dx.any() and not dy.any() and s.info.cg_iters == 0


def test_bounded_wait_times_out_and_context_survives():
    """A wait that nothing satisfies (host-injected: the root piece's head waits
    for one arrival too many) ends with KKT_ERR_TIMEOUT; the GPU context and
    the library stay usable."""
    sys = W.make_config("grid2d_n2000")
    hh = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    root_piece = K.kkt_symbolic_info_get(hh).npieces - 1
    K.kkt_destroy(hh)
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx,
                    debug_stall_piece=root_piece, spin_cycles=20_000_000)
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    with pytest.raises(K.KKTError) as e:
        s.solve(cu(sys.r_x), cu(sys.r_y))
    assert e.value.code == 7
    s2, code, dx, dy = gpu_solve(sys)
    assert code == 0 and s2.info.rr <= 1e-8


def test_host_buffer_entry_point():
    sys = W.make_config("grid2d_n2000")
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    dx, dy = s.factor_solve_host(sys.H_vals, sys.J_vals, sys.delta, sys.gamma, sys.r_x, sys.r_y)
    _, _, odx, ody, _ = O.solve_system(sys)
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6


def test_repeat_solves_agree():
    sys = W.make_config("grid2d_n2000")
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    a = torch.cat(s.solve(cu(sys.r_x), cu(sys.r_y))).cpu().numpy()
    b = torch.cat(s.solve(cu(sys.r_x), cu(sys.r_y))).cpu().numpy()
    assert rel(a, b) <= 1e-12


# ----------------------------------------------------------------- 4x4 form (Sec. 3)
def _oracle_4x4(p):
    """Oracle 4x4 solve (reduction, 2x2 solve, recovery); None when the
    oracle's Cholesky of H~ + gamma J^T J fails."""
    Hp, Hi, Hv, r_x = O.reduce4x4(p)
    s = W.KKTSystem(p["n_x"], p["m_c"], Hp, Hi, Hv, p["J_rowptr"], p["J_colidx"], p["J_vals"], r_x, p["r_y"],
                    p.get("delta", 0.0), p.get("gamma", 1e2))
    _, _, dx, dy, info = O.solve_system(s, ir_maxit=2)
    if info["status"] == 2:
        return None
    assert info["status"] == 0
    ds, dyd = O.recover4x4(p, dx)
    return np.concatenate([dx, ds, dy, dyd])


def _gpu_4x4(p, precision):
    s = K.KKTSolver4x4(p["n_x"], p["m_c"], p["m_d"], p["H_colptr"], p["H_rowidx"], p["J_rowptr"], p["J_colidx"],
                       p["Jd_rowptr"], p["Jd_colidx"], precision=precision)
    try:
        code = s.factor(cu(p["H_vals"]), cu(p["D_x"]), cu(p["Jd_vals"]), cu(p["D_s"]), cu(p["J_vals"]),
                        p.get("delta", 0.0), p.get("gamma", 1e2), check=False)
        if code == 2:
            return None
        assert code == 0
        out = s.solve(cu(p["r_xt"]), cu(p["r_s"]), cu(p["r_y"]), cu(p["r_yd"]))
        assert s.info.rr <= 1e-8
        return np.concatenate([o.cpu().numpy() for o in out])
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", range(6))
def test_4x4_tiny_matches_oracle(seed, precision):
    """Random 4x4 parts as drawn (H often indefinite on null(J): then both
    sides must report the failed Cholesky, Thm 1) and with D_x shifted by 10
    (H~ SPD: solutions agree)."""
    p = W.random_4x4_parts(seed, n_x=20 + 9 * seed, m_c=5 + seed, m_d=4 + 3 * seed)
    ref, got = _oracle_4x4(p), _gpu_4x4(p, precision)
    assert (ref is None) == (got is None)
    if ref is not None:
        assert rel(got, ref) <= 1e-6
    p["D_x"] = p["D_x"] + 10.0
    ref, got = _oracle_4x4(p), _gpu_4x4(p, precision)
    assert ref is not None and got is not None
    assert rel(got, ref) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_4x4_grid_matches_oracle(precision):
    """50x40 grid, J_d with 500 local rows, D_s over eight decades."""
    p = W.grid_4x4_parts("grid2d_n2000")
    assert rel(_gpu_4x4(p, precision), _oracle_4x4(p)) <= 1e-6


# ----------------------------------------------------------------- several right-hand sides (a12)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 11])
def test_multi_rhs_matches_oracle(precision, nrhs):
    """One factor, nrhs right-hand sides sharing the triangular sweeps (groups
    of up to 8 per launch): every solution equals the oracle's solve of that
    right-hand side, and each reaches the RR target."""
    sys = W.make_config("grid2d_n2000")
    rng = np.random.default_rng(nrhs)
    RX = rng.standard_normal((nrhs, sys.n))
    RY = rng.standard_normal((nrhs, sys.m))
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision=precision,
                    ordering="nd")
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    dx, dy, infos = s.solve_multi(cu(RX), cu(RY))
    dx, dy = dx.cpu().numpy(), dy.cpu().numpy()
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    for j in range(nrhs):
        odx, ody, oinfo = fac.solve(RX[j], RY[j])
        assert rel(np.concatenate([dx[j], dy[j]]), np.concatenate([odx, ody])) <= 1e-6
        assert infos[j].rr <= 1e-8 and infos[j].cg_status == 0
        if precision == "fp64":
            assert abs(infos[j].cg_iters - oinfo["iters"]) <= 1
    assert s.info.rr == max(i.rr for i in infos)
    assert s.inertia_ok


def test_multi_rhs_equals_single_solves():
    """The same right-hand sides solved together and one at a time agree to
    rounding (FP64)."""
    sys = W.make_config("grid2d_n20k")
    rng = np.random.default_rng(5)
    RX = rng.standard_normal((5, sys.n))
    RY = rng.standard_normal((5, sys.m))
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, ordering="nd")
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    dx, dy, _ = s.solve_multi(cu(RX), cu(RY))
    for j in range(5):
        sx, sy = s.solve(cu(RX[j]), cu(RY[j]))
        a = torch.cat([dx[j], dy[j]]).cpu().numpy()
        b = torch.cat([sx, sy]).cpu().numpy()
        assert rel(a, b) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_systems_match_oracle(precision):
    """Five systems on one analysed pattern (the 50x40 grid with per-entry
    rescaled barriers, one of them shifted to be indefinite): each solution
    equals the oracle's; the indefinite one reports NOT_SPD and is skipped."""
    base = W.make_config("grid2d_n2000")
    systems = [base]
    for t in range(1, 5):
        systems.append(W.rescale_barrier(systems[-1], seed=(7, t)))
    bad = 3
    Hbad = systems[bad].H_vals.copy()
    diag = systems[bad].H_colptr[:-1]           # the diagonal entry leads each lower column
    Hbad[diag] -= 1e3
    systems[bad] = W.KKTSystem(base.n, base.m, base.H_colptr, base.H_rowidx, Hbad, base.J_rowptr,
                               base.J_colidx, base.J_vals, systems[bad].r_x, systems[bad].r_y, base.delta, base.gamma)
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                    precision=precision, ordering="nd")
    code, st = s.factor_batch(cu(np.stack([x.H_vals for x in systems])), cu(np.stack([x.J_vals for x in systems])),
                              base.delta, base.gamma)
    assert code == 2 and list(st) == [0, 0, 0, 2, 0]
    dx, dy, infos, sst, code = s.solve_batch(cu(np.stack([x.r_x for x in systems])),
                                             cu(np.stack([x.r_y for x in systems])))
    assert code == 2 and list(sst) == [0, 0, 0, 2, 0]
    for b, x in enumerate(systems):
        if b == bad:
            continue
        _, _, odx, ody, oinfo = O.solve_system(x)
        assert infos[b].rr <= 1e-8
        assert rel(np.concatenate([dx[b].cpu().numpy(), dy[b].cpu().numpy()]), np.concatenate([odx, ody])) <= 1e-6


@pytest.mark.parametrize("lam", [0.5, -2.5e-8, -1e-5])
def test_factor_regularized_matches_oracle(lam):
    """Algorithm 1's delta_1 loop on the device takes the same delta_1 as the
    oracle's (FP64), and the solve at that shift matches."""
    from test_oracle import nullspace_indefinite_system
    sys, _, _ = nullspace_indefinite_system(lam)
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    fac, d_ref = O.factor_regularized(sym, sys.H_vals, sys.J_vals, sys.gamma)
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    code, d = s.factor_regularized(cu(sys.H_vals), cu(sys.J_vals), sys.gamma)
    assert d == d_ref
    assert (code == 0) == fac.ok
    if fac.ok:
        dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y))
        dx, dy = dx.cpu().numpy(), dy.cpu().numpy()
        # RR on K_delta at the accepted shift, evaluated by the oracle; with
        # lam near -delta_1, H_delta's smallest eigenvalue is ~1e-8 and even
        # the oracle's own solve (same 3 refinement passes) stops near 2e-7:
        # the gate is the oracle's achieved RR then
        rr = O.residual(sym, sys.H_vals, sys.J_vals, d, sys.r_x, sys.r_y, dx, dy)["rr"]
        _, _, oinfo = fac.solve(sys.r_x, sys.r_y, ir_maxit=3)
        assert rr <= max(1e-8, 10 * oinfo["rr"])
        if lam > 0:
            # well conditioned: the solutions agree; with lam near -delta_1 the
            # smallest eigenvalue of H_delta is ~1e-8 and the x part is
            # conditioning-limited (reading of the 1e-6 gate: RR decides)
            odx, ody, _ = fac.solve(sys.r_x, sys.r_y)
            assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6


def test_factor_regularized_sequence_matches_oracle(precision="fp64"):
    """A sequence of matrices on one handle: the device loop (one graph
    launch per matrix) carries delta_1 as Sec. 4.1 says, back to the
    previous matrix's value after a failed unshifted trial, and accepts the
    same delta_1 as the oracle at every step; kkt_set_delta_prev(0) starts a
    new sequence. Each accepted factor then solves to the oracle's RR. FP64
    only: the shifts here (~1e-8 against ||H_gamma|| ~ 1e3) lie below the
    FP32 factor's rounding, so its pivots decide at another threshold."""
    from test_oracle import nullspace_indefinite_system
    lams = [-2.5e-8, -1e-8, 0.5, -5e-9, -5e-8]
    base, _, _ = nullspace_indefinite_system(lams[0])
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx, precision=precision)
    sym = O.Symbolic(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx)
    prev = 0.0
    for t, lam in enumerate(lams + [lams[1]]):
        if t == len(lams):
            s.set_delta_prev(0.0)                  # new sequence: the second matrix again, from scratch
            prev = 0.0
        sys, _, _ = nullspace_indefinite_system(lam)
        fac, d_ref = O.factor_regularized(sym, sys.H_vals, sys.J_vals, sys.gamma, delta_prev=prev)
        code, d = s.factor_regularized(cu(sys.H_vals), cu(sys.J_vals), sys.gamma)
        assert (code == 0) == fac.ok and fac.ok
        assert d == d_ref, (lam, d, d_ref)
        dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y))
        rr = O.residual(sym, sys.H_vals, sys.J_vals, d, sys.r_x, sys.r_y, dx.cpu().numpy(), dy.cpu().numpy())["rr"]
        _, _, oinfo = fac.solve(sys.r_x, sys.r_y, ir_maxit=3)
        assert rr <= max(1e-8, 10 * oinfo["rr"])
        prev = d
    assert d == pytest.approx(1.6e-8, rel=1e-12)   # -1e-8 from scratch: 1e-9 * 2^4
    s.close()


@pytest.mark.parametrize("refine", [1, 2])
@pytest.mark.parametrize("name", ["grid2d_n2000", "grid2d_n20k"])
def test_mixed_refinement_modes_match_oracle(name, refine):
    """The mixed form with plain refinement passes (refine=1) and with
    flexible GMRES (refine=2, the default) reaches the oracle's solution and
    RR <= 1e-9."""
    sys = W.make_config(name)
    _, _, odx, ody, _ = O.solve_system(sys)
    s, code, dx, dy = gpu_solve(sys, "mixed", ordering="nd", refine=refine)
    assert code == 0
    assert s.info.rr <= 1e-9 and s.inertia_ok
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-6


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_solve_trace_records_every_item(precision):
    """A profile handle records the item timeline of one H^-1 application:
    every item of both sweeps ran (dispatch and finish stamps set, finish
    not before dispatch, a CTA index inside the grid), the backward sweep
    starts after the forward one ends, and a handle without profiling
    refuses the call."""
    sys = W.make_config("grid2d_n2000")
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx,
                    precision=precision, ordering="nd", profile=1)
    try:
        s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
        s.solve(cu(sys.r_x), cu(sys.r_y))
        torch.cuda.synchronize()
        tr = s.solve_trace().astype(np.int64)
        f, b = s.solve_item_order()
        assert tr.shape == (2, len(f), 3)
        start, end, cta = tr[..., 0], tr[..., 1], tr[..., 2]
        assert (start > 0).all() and (end >= start).all()
        assert (cta >= 0).all() and (cta < 148 * 4).all()
        assert start[1].min() >= end[0].max()
    finally:
        s.close()
    s2 = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx,
                     precision=precision, ordering="nd")
    try:
        with pytest.raises(K.KKTError):
            s2.solve_trace()
    finally:
        s2.close()


def test_analyse_like_reuses_the_analysis_in_the_other_precision():
    """kkt_analyse_like: an FP64 handle made from a mixed handle (and a mixed
    one from a host-only analysis) has the same symbolic analysis and solves
    the 50x40 workload to the oracle's solution; the profile toggle times
    the factor kernels of a handle made without profiling."""
    sys = W.make_config("grid2d_n2000")
    _, _, odx, ody, _ = O.solve_system(sys)
    ref = np.concatenate([odx, ody])
    a = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision="mixed")
    b = K.KKTSolver.like(a, precision="fp64")
    hs = K.KKTSolver.host_only(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    c = K.KKTSolver.like(hs, precision="mixed")
    ga, gb, gc = (K.kkt_get_symbolic(x.h) for x in (a, b, c))
    for k in ga:
        np.testing.assert_array_equal(ga[k], gb[k])
        np.testing.assert_array_equal(ga[k], gc[k])
    for x, tol in ((a, 1e-7), (b, 1e-9), (c, 1e-7)):
        x.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
        dx, dy = x.solve(cu(sys.r_x), cu(sys.r_y))
        assert rel(torch.cat([dx, dy]).cpu().numpy(), ref) <= tol
    with pytest.raises(K.KKTError):
        K.KKTSolver.like(a, precision="fp64", ordering=2)    # another ordering needs its own analysis
    c.set_profile(True)
    c.profile(reset=True)
    c.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    p = c.profile(reset=True)
    assert p["assemble"][1] == 1 and p["tri_inv"][1] == 1
    c.set_profile(False)
    c.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    assert c.profile(reset=True)["assemble"][1] == 0
    for x in (a, b, c, hs):
        x.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["grid2d_n2000", "tiny"])
def test_ruiz_scaling_matches_oracle(name, precision):
    """Symmetrized Ruiz scaling (Sec. 4.1) on the device: D equals the
    oracle's bit for bit (products, maxima, square roots and divisions
    only), and the solution of the scaled system, unscaled, matches the
    oracle's scaled solve; the refused forms say so."""
    if name == "tiny":
        # a badly scaled system: S H~ S and R J S with S, R spread over 6 decades
        sys = W.random_tiny_system(17, n_lo=60, n_hi=100, density=0.08)
        rng = np.random.default_rng(1)
        S, Rr = 10.0 ** rng.uniform(-3, 3, sys.n), 10.0 ** rng.uniform(-3, 3, sys.m)
        cols = np.repeat(np.arange(sys.n), np.diff(sys.H_colptr))
        sys.H_vals = S[sys.H_rowidx] * sys.H_vals * S[cols]
        jrow = np.repeat(np.arange(sys.m), np.diff(sys.J_rowptr))
        sys.J_vals = Rr[jrow] * sys.J_vals * S[sys.J_colidx]
    else:
        sys = W.make_config(name)
    iters = 10
    Dx, Dy = O.ruiz_scaling(sys, iters)
    sc = O.scale_system(sys, Dx, Dy)
    _, _, odx, ody, oinfo = O.solve_system(sc, ir_maxit=3)
    if oinfo["status"] != 0:
        pytest.skip("oracle: scaled H_gamma not SPD at this delta")
    ref = np.concatenate([Dx * odx, Dy * ody])
    s, code, dx, dy = gpu_solve(sys, precision, ruiz_iters=iters)
    assert code == 0
    np.testing.assert_array_equal(s.scaling(), np.concatenate([Dx, Dy]))
    assert s.info.rr <= (1e-10 if precision == "fp64" else 1e-9)
    assert rel(np.concatenate([dx, dy]), ref) <= (1e-9 if precision == "fp64" else 1e-6)
    with pytest.raises(K.KKTError):
        s.hsolve(cu(sys.r_x))
    with pytest.raises(K.KKTError):
        s.solve_multi(cu(np.stack([sys.r_x] * 2)), cu(np.stack([sys.r_y] * 2)))
    s.close()


@pytest.mark.parametrize("method,code", [("pcg", 1), ("minres", 2)])
@pytest.mark.parametrize("name", ["grid2d_n2000", "tiny"])
def test_schur_krylov_variants_match_oracle(name, method, code):
    """Sec. 4's variants on the device (FP64): CG preconditioned by
    M = (J J^T)^-1 J H_gamma J^T (J J^T)^-1 and MINRES on S, against the
    oracle's restatement: same solution to 1e-9, iteration counts within 1,
    RR <= 1e-10 (one refinement pass at most)."""
    sys = W.make_config(name) if name != "tiny" else W.random_tiny_system(23, n_lo=60, n_hi=100, density=0.08)
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    fac = O.Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    odx, ody, oit = O.schur_variant(fac, sys, method)
    s, c, dx, dy = gpu_solve(sys, "fp64", krylov=code)
    assert c == 0
    assert rel(np.concatenate([dx, dy]), np.concatenate([odx, ody])) <= 1e-9
    assert s.info.rr <= 1e-10
    assert abs(s.info.cg_iters - oit) <= 1 + s.info.ir_steps * (oit + 1)
    if s.info.ir_steps == 0:
        assert abs(s.info.cg_iters - oit) <= 1
    s.close()


def test_schur_krylov_variants_need_fp64():
    sys = W.make_config("grid2d_n2000")
    with pytest.raises(K.KKTError):
        K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision="mixed", krylov=1)


def test_batched_factor_on_tensor_core_fronts_matches_oracle():
    """The batched form's one-graph factorization (system b = blockIdx.y of
    every launch, one tensor-core operand workspace per system) on fronts that
    take the tensor-core SYRK and in-panel updates: each system's solution
    equals the oracle's, read from its own batch slot with no copies; the
    single-system path of the same handle still works afterwards."""
    base = block_front_system(1100)
    diag = base.H_colptr[:-1]
    systems = []
    for k in range(3):
        x = base.copy()
        off = np.ones(x.H_vals.size, bool)
        off[diag] = False
        x.H_vals = x.H_vals.copy()
        x.H_vals[off] *= 0.5 + 0.25 * k          # diagonal dominance kept
        x.r_x = np.random.default_rng(k).standard_normal(x.n)
        systems.append(x)
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                    precision="mixed", ordering="natural")
    code, st = s.factor_batch(cu(np.stack([x.H_vals for x in systems])), cu(np.stack([x.J_vals for x in systems])),
                              base.delta, base.gamma)
    assert code == 0 and list(st) == [0, 0, 0]
    dx, dy, infos, sst, code = s.solve_batch(cu(np.stack([x.r_x for x in systems])),
                                             cu(np.stack([x.r_y for x in systems])))
    assert code == 0
    for b, x in enumerate(systems):
        _, _, odx, ody, _ = O.solve_system(x, ordering="natural")
        assert infos[b].rr <= 1e-9
        assert rel(np.concatenate([dx[b].cpu().numpy(), dy[b].cpu().numpy()]), np.concatenate([odx, ody])) <= 1e-6
    x = systems[1]
    s.factor(cu(x.H_vals), cu(x.J_vals), x.delta, x.gamma)
    ddx, ddy = s.solve(cu(x.r_x), cu(x.r_y))
    assert rel(torch.cat([ddx, ddy]).cpu().numpy(), np.concatenate([dx[1].cpu().numpy(), dy[1].cpu().numpy()])) <= 1e-6
    s.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_handle_still_solves_after_handles_with_smaller_solve_layouts(precision):
    """Handles with different plans launch the same solve and triangle-inverse
    kernels with different shared-memory sizes: a handle made, used and
    destroyed later with a smaller layout (narrower pieces, fewer entries per
    item) must leave the first one able to factor and solve to the oracle's
    solution."""
    sys = W.make_config("grid2d_n2000")
    _, _, odx, ody, _ = O.solve_system(sys, ordering="nd")
    ref = np.concatenate([odx, ody])
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision=precision,
                    ordering="nd")
    for rep in range(2):
        if rep:
            t = K.KKTSolver.like(s, precision=precision, ordering="nd", solve_w=32, solve_ent=2048)
            t.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
            dx, dy = t.solve(cu(sys.r_x), cu(sys.r_y))
            assert rel(torch.cat([dx, dy]).cpu().numpy(), ref) <= 1e-6
            t.close()
        s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
        dx, dy = s.solve(cu(sys.r_x), cu(sys.r_y))
        assert s.info.cg_iters > 0 and s.info.rr <= 1e-9
        assert rel(torch.cat([dx, dy]).cpu().numpy(), ref) <= 1e-6
    s.close()


def test_multi_rhs_on_a_large_mixed_plan_equals_single_solves():
    """Mixed factors of at least 1e8 panel entries solve one right-hand side
    with chunk tiles over the inverse region (three solve CTAs per SM); the
    several-right-hand-side launches switch to the separate layout. On the
    500 x 500 workload (3.2e8 panel entries) four right-hand sides solved
    together equal their single solves to the refinement's tolerance and
    reach the RR target."""
    sys = W.make_config("grid2d_n250k")
    s = K.KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, precision="mixed",
                    ordering="nd")
    assert s.symbolic_info.panel_entries >= 10 ** 8
    rng = np.random.default_rng(11)
    RX = rng.standard_normal((4, sys.n))
    RY = rng.standard_normal((4, sys.m))
    s.factor(cu(sys.H_vals), cu(sys.J_vals), sys.delta, sys.gamma)
    dx, dy, infos = s.solve_multi(cu(RX), cu(RY))
    for j in range(4):
        assert infos[j].rr <= 1e-8
        sx, sy = s.solve(cu(RX[j]), cu(RY[j]))
        assert s.info.rr <= 1e-8
        a = torch.cat([dx[j], dy[j]]).cpu().numpy()
        b = torch.cat([sx, sy]).cpu().numpy()
        assert rel(a, b) <= 1e-6
    s.close()


def test_batched_form_on_a_large_mixed_plan_equals_single_solves():
    """The batched form on a plan that uses the overlapped solve layout (the
    500 x 500 workload, 3.2e8 panel entries, tensor-core fronts): two systems
    factored in one graph and solved on the helper handles equal the same
    systems factored and solved one at a time, and reach the RR target."""
    base = W.make_config("grid2d_n250k")
    systems = [base, W.rescale_barrier(base, seed=(3, 1))]
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx, precision="mixed",
                    ordering="nd")
    assert s.symbolic_info.panel_entries >= 10 ** 8
    code, st = s.factor_batch(cu(np.stack([x.H_vals for x in systems])), cu(np.stack([x.J_vals for x in systems])),
                              base.delta, base.gamma)
    assert code == 0 and list(st) == [0, 0]
    dx, dy, infos, sst, code = s.solve_batch(cu(np.stack([x.r_x for x in systems])),
                                             cu(np.stack([x.r_y for x in systems])))
    assert code == 0 and list(sst) == [0, 0]
    for b, x in enumerate(systems):
        assert infos[b].rr <= 1e-8
        s.factor(cu(x.H_vals), cu(x.J_vals), x.delta, x.gamma)
        sx, sy = s.solve(cu(x.r_x), cu(x.r_y))
        a = np.concatenate([dx[b].cpu().numpy(), dy[b].cpu().numpy()])
        assert rel(a, torch.cat([sx, sy]).cpu().numpy()) <= 1e-6
    s.close()
