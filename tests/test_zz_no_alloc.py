"""kkt_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the residual the solver itself reports
(kkt_solve + kkt_get_info, which uses the library's allocated workspace),
on two calls in a row with different systems, so that anything the first
call leaves in the shared scratch would show up in the second. This file is
collected last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2110_03636_b300 as K  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a, dt=np.float64):
    return torch.as_tensor(np.ascontiguousarray(a, dt), device=DEV)


def test_noalloc_residual_matches_solver_on_two_calls():
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
        ref = s.info                                   # residual of the existing entry point
        res_x = torch.empty(sys.n, dtype=torch.float64, device=DEV)
        res_y = torch.empty(sys.m, dtype=torch.float64, device=DEV)
        norms = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
        code = K.kkt_residual_noalloc(sys.n, sys.m, Hp, Hi, Hv, Jp, Ji, Jv, sys.delta, rx, ry, dx, dy,
                                      res_x, res_y, norms)
        assert code == 0, K.kkt_status_string(code)
        torch.cuda.synchronize()
        rr, be, resn, knorm = norms.cpu().numpy()
        assert rr <= 1e-8 and ref.rr <= 1e-8
        assert abs(rr - ref.rr) <= 1e-3 * ref.rr
        assert abs(be - ref.be) <= 1e-3 * ref.be
        # the residual vector itself: ||res|| consistent with RR, and small
        assert resn == pytest.approx(rr * np.linalg.norm(np.concatenate([sys.r_x, sys.r_y])), rel=1e-12)
        assert np.linalg.norm(torch.cat([res_x, res_y]).cpu().numpy()) == pytest.approx(resn, rel=1e-12)
    s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    n = K.NOALLOC_MAX_ROWS
    z64 = torch.zeros(n + 1, dtype=torch.int64, device=DEV)
    z32 = torch.zeros(1, dtype=torch.int32, device=DEV)
    f = torch.zeros(1, dtype=torch.float64, device=DEV)
    code = K.kkt_residual_noalloc(n, 1, z64, z32, f, z64[:2], z32, f, 0.0, f, f, f, f, f, f,
                                  torch.zeros(4, dtype=torch.float64, device=DEV))
    assert code == 9
    assert "no-allocation" in K.kkt_status_string(code)
