"""Autotuner of the plan parameters (supernode relaxation, solve tile shape,
tensor-core switch): the coordinate search on a synthetic objective (CPU),
the symbolic parity of every relaxation setting it can pick (CPU), and one
measured search on the device (GPU)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2110_03636_b300 import autotune as AT


def _fake(best, slow_rr=()):
    """Objective with a known coordinate-wise optimum: each parameter away
    from ``best`` costs a fixed amount; sets listed in slow_rr miss the
    residual target."""
    calls = []

    def obj(p):
        calls.append(dict(p))
        t = 1.0 + sum(0.1 * (i + 1) for i, k in enumerate(sorted(p)) if p[k] != best[k])
        rr = 1e-6 if any(p[k] == v for k, v in slow_rr) else 1e-10
        return t, rr
    return obj, calls


def test_search_finds_the_coordinate_optimum_and_evaluates_each_set_once():
    best = {"relax_small": 32, "relax_frac": (1, 20), "relax_wmax": 256, "solve_w": 64, "solve_ent": 8192,
            "tensor_cores": 1, "tc_panel_min": 512}
    obj, calls = _fake(best)
    got, t, evals = AT.coordinate_search(obj)
    assert got == best and t == pytest.approx(1.0)
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys))
    assert len(evals) == len(calls)


def test_search_skips_sets_that_miss_the_residual_target():
    best = {"relax_small": 8, "relax_frac": (1, 10), "relax_wmax": 256, "solve_w": 128, "solve_ent": 12288,
            "tensor_cores": 0, "tc_panel_min": 128}
    obj, _ = _fake(best, slow_rr=[("tensor_cores", 0)])     # the faster setting is not accurate enough
    got, _, evals = AT.coordinate_search(obj)
    assert got["tensor_cores"] == 1 and got["relax_small"] == 8
    assert all(p["tensor_cores"] == 1 or rr > 1e-8 for p, _, rr in evals if np.isfinite(rr))


def test_every_relaxation_setting_of_the_space_is_bit_exact_with_the_oracle():
    """The tuner may pick any relaxation of its space: each one along the
    coordinates from the defaults gives the oracle's supernodes on the
    batching workload's pattern (200 x 100 grid, nested dissection)."""
    import paper_2110_03636_b300 as K
    sys = W.make_config("grid2d_n20k")
    sets = {(AT.DEFAULT["relax_small"], AT.DEFAULT["relax_frac"], AT.DEFAULT["relax_wmax"])}
    for name in ("relax_small", "relax_frac", "relax_wmax"):
        for v in AT.SPACE[name]:
            p = dict(AT.DEFAULT, **{name: v})
            sets.add((p["relax_small"], p["relax_frac"], p["relax_wmax"]))
    for small, (num, den), wmax in sorted(sets):
        o = K.kkt_default_options(ordering=2, relax_small=small, relax_num=num, relax_den=den, relax_wmax=wmax)
        h = K.kkt_analyse_host(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, o)
        try:
            g = K.kkt_get_symbolic(h)
        finally:
            K.kkt_destroy(h)
        sym = O.Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, relax_small=small,
                         relax_num=num, relax_den=den, wmax=wmax, ordering="nd")
        st, rp, rows, par = sym.supernodes()
        np.testing.assert_array_equal(g["sn_start"], st)
        np.testing.assert_array_equal(g["sn_rows"], rows)
        np.testing.assert_array_equal(g["sn_parent"], par)


@pytest.mark.gpu
def test_measured_search_on_the_device_picks_an_accurate_set():
    """A measured search (one sweep) on the 50 x 40 workload: the chosen set
    solves to the oracle's solution."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2110_03636_b300 as K
    sys = W.make_config("grid2d_n2000")
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    sets = [(cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y), x.delta, x.gamma)
            for x in (sys, W.rescale_barrier(sys, seed=(0, 1)))]
    pattern = (sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    opts, t, t_def, evals = AT.tune(pattern, sets, sweeps=1)
    assert t <= t_def and len(evals) >= 6
    s = K.KKTSolver(*pattern, precision="mixed", ordering="nd", **opts)
    s.factor(sets[0][0], sets[0][1], sys.delta, sys.gamma)
    dx, dy = s.solve(sets[0][2], sets[0][3])
    _, _, odx, ody, _ = O.solve_system(sys)
    got, ref = torch.cat([dx, dy]).cpu().numpy(), np.concatenate([odx, ody])
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    s.close()
