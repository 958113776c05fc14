"""Full-size workloads on the GPU, checked through properties that hold at
any size: the relative residual of the returned solution on K_delta (Sec. 5.1,
RR), computed here on the host in FP64 from its definition with scipy, the
inertia flag, and agreement between the two precisions. The 100^3 workload
runs in its default (mixed, flexible GMRES) form, about 100 GB of device
memory and a minute of host analysis; its FP64 and plain-pass forms (minutes
of FP64 factorization) run only with KKT_BIG=1."""
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
import paper_2110_03636_b300 as K

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def host_rr(x, dx, dy):
    """||b - K_delta [dx; dy]|| / ||b|| with K_delta = [H~ + delta I, J^T; J, 0]."""
    import scipy.sparse as sp
    H = sp.csc_matrix((x.H_vals, x.H_rowidx, x.H_colptr), shape=(x.n, x.n))
    J = sp.csr_matrix((x.J_vals, x.J_colidx, x.J_rowptr), shape=(x.m, x.n))
    Hx = H @ dx + H.T @ dx - H.diagonal() * dx + x.delta * dx
    rx = x.r_x - Hx - J.T @ dy
    ry = x.r_y - J @ dx
    return np.sqrt(np.dot(rx, rx) + np.dot(ry, ry)) / np.sqrt(np.dot(x.r_x, x.r_x) + np.dot(x.r_y, x.r_y))


@pytest.mark.slow
def test_grid2d_n250k_both_precisions():
    """500x500 grid, ND ordering, two value sets of the interior sequence:
    both precisions reach RR <= 1e-8 by the oracle's residual and agree with
    each other to 1e-6."""
    base = W.make_config("grid2d_n250k")
    sets = [base, W.rescale_barrier(base, seed=(0, 1))]
    sols = {}
    for prec in ("mixed", "fp64"):
        s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                        precision=prec, ordering="nd")
        for t, x in enumerate(sets):
            s.factor(cu(x.H_vals), cu(x.J_vals), x.delta, x.gamma)
            dx, dy = s.solve(cu(x.r_x), cu(x.r_y))
            dx, dy = dx.cpu().numpy(), dy.cpu().numpy()
            rr = host_rr(x, dx, dy)
            assert rr <= 1e-8, (prec, t, rr)
            assert abs(rr - s.info.rr) <= 0.1 * rr + 1e-15
            assert s.inertia_ok
            sols[(prec, t)] = np.concatenate([dx, dy])
        s.close()
    for t in range(2):
        a, b = sols[("mixed", t)], sols[("fp64", t)]
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


BIG = pytest.mark.skipif(os.environ.get("KKT_BIG") != "1", reason="100^3 FP64 / plain passes: set KKT_BIG=1")


@pytest.mark.slow
@pytest.mark.parametrize("precision,refine", [pytest.param("fp64", 0, marks=BIG), pytest.param("mixed", 1, marks=BIG),
                                              ("mixed", 2)])
def test_grid3d_n1m(precision, refine):
    """The 100^3 precision-form workload (n = 1e6, m = 5e5, gamma = 1e6,
    barrier 10^U(-8,8)). FP64 must reach RR <= 1e-8 (checked on the host from
    the definition). The mixed form's FP32 factor carries an error of order
    eps_32 kappa(H_gamma), far above 1 here, so its refinement cannot reach
    the target with plain passes: the test checks that it reports the RR it
    reached truthfully (refine=1). Flexible GMRES preconditioned by the mixed
    solve (refine=2, the default) must reach the target."""
    x = W.make_config("grid3d_n1m")
    s = K.KKTSolver(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx, precision=precision, ordering="nd",
                    refine=refine)
    info = s.symbolic_info
    print(precision, "nnzL", info.nnz_l, "flops", info.flops, "device GB", info.device_bytes / 1e9, flush=True)
    import time
    torch.cuda.synchronize()
    t0 = time.time()
    s.factor(cu(x.H_vals), cu(x.J_vals), x.delta, x.gamma)
    torch.cuda.synchronize()
    t1 = time.time()
    dx, dy = s.solve(cu(x.r_x), cu(x.r_y), check=False)
    torch.cuda.synchronize()
    t2 = time.time()
    i = s.info
    rr = host_rr(x, dx.cpu().numpy(), dy.cpu().numpy())
    print(precision, refine, "factor s", round(t1 - t0, 2), "solve s", round(t2 - t1, 2), "cg", i.cg_iters, "ir", i.ir_steps,
          "rr(device)", i.rr, "rr(host)", rr, flush=True)
    # residuals near 1e-13 differ in their own rounding: absolute slack
    assert abs(rr - i.rr) <= 0.1 * rr + 1e-12
    s.close()
    del s, dx, dy
    torch.cuda.empty_cache()
    if precision == "fp64" or refine == 2:
        assert rr <= 1e-8
