"""kkt_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the FP64 CPU oracle's residual
(oracle.residual: the vector b - K_delta [dx; dy] and its norms, Sec. 5.1)
element by element, and against the residual the solver itself reports
(kkt_solve + kkt_get_info, which uses the library's allocated workspace), on
two calls in a row with different systems, so that anything the first call
leaves in the shared scratch would show up in the second. A system without
constraints (m = 0, no J arrays) is checked the same way. This file is
collected last on purpose."""
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


def cu(a, dt=np.float64):
    return torch.as_tensor(np.ascontiguousarray(a, dt), device=DEV)


def _noalloc(sys, Hp, Hi, Hv, Jp, Ji, Jv, rx, ry, dx, dy):
    res_x = torch.full((sys.n,), float("nan"), dtype=torch.float64, device=DEV)
    res_y = torch.full((sys.m,), float("nan"), dtype=torch.float64, device=DEV) if sys.m else None
    norms = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    code = K.kkt_residual_noalloc(sys.n, sys.m, Hp, Hi, Hv, Jp, Ji, Jv, sys.delta, rx, ry, dx, dy,
                                  res_x, res_y, norms)
    assert code == 0, K.kkt_status_string(code)
    torch.cuda.synchronize()
    res = res_x.cpu().numpy() if res_y is None else torch.cat([res_x, res_y]).cpu().numpy()
    return res, norms.cpu().numpy()


def _check_against_oracle(sys, res, norms, dx, dy):
    sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, ordering="natural")
    ref = O.residual(sym, sys.H_vals, sys.J_vals, sys.delta, sys.r_x, sys.r_y, dx, dy, vector=True)
    ref_vec = np.concatenate([ref["res_x"], ref["res_y"]])
    # the residual sums a handful of terms per row; atomics reorder them, so
    # each entry agrees to a few ulps of the largest term of its row
    scale = np.linalg.norm(np.concatenate([sys.r_x, sys.r_y]), np.inf) + ref["knorm"] * np.abs(
        np.concatenate([dx, dy])).max()
    assert np.abs(res - ref_vec).max() <= 1e-13 * scale
    rr, be, resn, knorm = norms
    assert knorm == pytest.approx(ref["knorm"], rel=1e-14)
    # norms of a residual that is itself tiny are relative to its own size
    assert resn == pytest.approx(ref["res"], rel=1e-6, abs=1e-13 * scale)
    assert rr == pytest.approx(ref["rr"], rel=1e-6, abs=1e-13 * scale)
    assert be == pytest.approx(ref["be"], rel=1e-6, abs=1e-13 * scale)
    assert np.linalg.norm(res) == pytest.approx(resn, rel=1e-12)
    return ref


def test_noalloc_residual_matches_oracle_and_solver_on_two_calls():
    base = W.make_config("grid2d_n2000")
    systems = [base, W.rescale_barrier(base, seed=(0, 1))]
    systems[1].H_vals = systems[1].H_vals * 3.0      # a different ||K||_inf on the second call
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx)
    Hp, Hi = cu(base.H_colptr, np.int64), cu(base.H_rowidx, np.int32)
    Jp, Ji = cu(base.J_rowptr, np.int64), cu(base.J_colidx, np.int32)
    for sys in systems:
        Hv, Jv, rx, ry = cu(sys.H_vals), cu(sys.J_vals), cu(sys.r_x), cu(sys.r_y)
        s.factor(Hv, Jv, sys.delta, sys.gamma)
        dx, dy = s.solve(rx, ry)
        solver = s.info                                # residual of the existing entry point
        res, norms = _noalloc(sys, Hp, Hi, Hv, Jp, Ji, Jv, rx, ry, dx, dy)
        ref = _check_against_oracle(sys, res, norms, dx.cpu().numpy(), dy.cpu().numpy())
        assert ref["rr"] <= 1e-8 and solver.rr <= 1e-8
        assert abs(norms[0] - solver.rr) <= 1e-3 * solver.rr
        assert abs(norms[1] - solver.be) <= 1e-3 * solver.be
    s.close()


def test_noalloc_residual_without_constraints():
    """m = 0: K_delta is H~ + delta I alone; the J arrays, r_y, dy and res_y
    are absent. An arbitrary (not solved) dx gives a residual of order one,
    compared entry by entry with the oracle's, on two calls in a row."""
    base = W.make_config("grid2d_n2000")
    rng = np.random.default_rng(7)
    sys = base.copy()
    sys.m = 0
    sys.J_rowptr = np.zeros(1, np.int64)
    sys.J_colidx = np.zeros(0, np.int32)
    sys.J_vals = np.zeros(0)
    sys.r_y = np.zeros(0)
    Hp, Hi, Hv = cu(sys.H_colptr, np.int64), cu(sys.H_rowidx, np.int32), cu(sys.H_vals)
    rx = cu(sys.r_x)
    for _ in range(2):
        dxh = rng.standard_normal(sys.n)
        res, norms = _noalloc(sys, Hp, Hi, Hv, None, None, None, rx, None, cu(dxh), None)
        _check_against_oracle(sys, res, norms, dxh, np.zeros(0))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """The C ABI itself refuses n + m beyond the fixed scratch before
    launching anything (the buffers are never touched)."""
    import ctypes as C
    n = K.NOALLOC_MAX_ROWS
    buf = torch.zeros(8, dtype=torch.float64, device=DEV)
    p = C.c_void_p(buf.data_ptr())
    code = K._lib.kkt_residual_noalloc(n, 1, p, p, p, p, p, p, 0.0, p, p, p, p, p, p, p, None)
    assert code == 9
    assert "no-allocation" in K.kkt_status_string(code)


def test_noalloc_binding_checks_lengths_and_device():
    """The binding refuses short arrays before calling into the library."""
    base = W.make_config("grid2d_n2000")
    Hp, Hi, Hv = cu(base.H_colptr, np.int64), cu(base.H_rowidx, np.int32), cu(base.H_vals)
    Jp, Ji, Jv = cu(base.J_rowptr, np.int64), cu(base.J_colidx, np.int32), cu(base.J_vals)
    vx, vy = cu(base.r_x), cu(base.r_y)
    out_x = torch.empty(base.n, dtype=torch.float64, device=DEV)
    out_y = torch.empty(base.m, dtype=torch.float64, device=DEV)
    norms = torch.empty(4, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        K.kkt_residual_noalloc(base.n, base.m, Hp, Hi, Hv, Jp, Ji, Jv, 0.0, vx, vy, vx, vy,
                               out_x[:-1], out_y, norms)
    with pytest.raises(ValueError):
        K.kkt_residual_noalloc(base.n, base.m, Hp, Hi, Hv[:-1], Jp, Ji, Jv, 0.0, vx, vy, vx, vy,
                               out_x, out_y, norms)
    with pytest.raises(ValueError):
        K.kkt_residual_noalloc(base.n, base.m, Hp, Hi, Hv, Jp[:-1], Ji, Jv, 0.0, vx, vy, vx, vy,
                               out_x, out_y, norms[:3])
