"""The request server (continuous batching over resident patterns) on the
GPU: every result is the same alone and in the mix (to the tolerance of the
method: solutions within 1e-6 of each other, each at RR <= 1e-8 recomputed
by the FP64 oracle from the definition), admission keeps the slots within
the HBM budget, and requests of several patterns overlap on the device."""
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


def _requests():
    """Two serving patterns (40 x 40 and 70 x 70 grids), four value updates
    each (barrier rescaled by 10^U(-1,1), new right-hand sides)."""
    reqs = []
    for pid, side in enumerate((40, 70)):
        x = W.serving_pattern(side)
        for t in range(4):
            x = W.rescale_barrier(x, seed=(side, t))
            reqs.append((pid, x))
    return reqs


def _run(srv, pids, reqs, together):
    out = []
    dev = [(cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y),
            torch.empty(x.n, dtype=torch.float64, device=DEV), torch.empty(x.m, dtype=torch.float64, device=DEV))
           for _, x in reqs]
    ids = []
    for (p, x), (H, J, rx, ry, dx, dy) in zip(reqs, dev):
        rid = srv.submit(pids[p], H, J, x.delta, x.gamma, rx, ry, dx, dy)
        if together:
            ids.append(rid)
        else:
            out.append(srv.wait(rid))
    for rid in ids:
        out.append(srv.wait(rid))
    return out, [(d[4].cpu().numpy(), d[5].cpu().numpy()) for d in dev]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_results_are_the_same_alone_and_in_the_mix(precision):
    reqs = _requests()
    pats = {}
    for p, x in reqs:
        pats.setdefault(p, x)
    srv = K.KKTServer(0, max_inflight=4, precision=precision, ordering="nd", solve_sms=37)
    pids = {p: srv.add_pattern(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx) for p, x in pats.items()}
    alone_info, alone = _run(srv, pids, reqs, together=False)
    mix_info, mix = _run(srv, pids, reqs, together=True)
    st = srv.stats()
    srv.close()
    assert st.completed == 2 * len(reqs) and st.failed == 0
    assert st.peak_inflight >= 2                        # requests overlapped
    syms = {p: O.Symbolic(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx, ordering="natural")
            for p, x in pats.items()}
    for k, (p, x) in enumerate(reqs):
        assert alone_info[k].status == 0 and mix_info[k].status == 0
        a = np.concatenate(alone[k])
        b = np.concatenate(mix[k])
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
        for dx, dy in (alone[k], mix[k]):
            rr = O.residual(syms[p], x.H_vals, x.J_vals, x.delta, x.r_x, x.r_y, dx, dy)["rr"]
            assert rr <= 1e-8


def test_admission_keeps_slots_within_the_budget():
    """A budget of exactly one slot per pattern: requests of the same
    pattern queue for its slot instead of allocating another one, and the
    accounted bytes never exceed the budget."""
    reqs = _requests()
    pats = {}
    for p, x in reqs:
        pats.setdefault(p, x)
    probe = K.KKTServer(0, max_inflight=1, precision="mixed", ordering="nd")
    pids = {p: probe.add_pattern(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx) for p, x in pats.items()}
    one_each = probe.stats().bytes_used
    probe.close()
    budget = int(one_each)
    srv = K.KKTServer(budget, max_inflight=4, precision="mixed", ordering="nd", solve_sms=37)
    pids = {p: srv.add_pattern(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx) for p, x in pats.items()}
    infos, _ = _run(srv, pids, reqs, together=True)
    st = srv.stats()
    srv.close()
    assert all(i.status == 0 for i in infos)
    assert st.slots == len(pats)
    assert st.bytes_peak <= st.budget
    assert st.peak_inflight <= len(pats)
