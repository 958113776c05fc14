"""Autotuner for the per-pattern plan parameters: supernode relaxation
(relax_small, relax_num/relax_den, relax_wmax), the triangular-solve tile
shape (solve_w columns per piece, solve_ent L entries per work item), the
tensor-core switch and the narrowest front whose in-panel updates take the
tensor cores. The analysis is exact for every parameter set (the
supernode partition only changes which explicit zeros are stored, never the
factor), so the tuner may pick any of them; it keeps the fastest one whose
solves meet the residual target.

Search: coordinate descent from the library defaults. Each sweep tries, for
one parameter at a time, every listed alternative with the others held at
the incumbent, and moves the incumbent when the measured objective improves
by more than ``min_gain``; it stops after a sweep without a move or after
``sweeps`` sweeps. The objective is a callable (options -> (seconds, rr)),
so the search logic runs without a GPU; :func:`measure` is the device
objective (median factor + solve time over value sets on the resident
pattern).
"""
from __future__ import annotations

import time

import numpy as np

__all__ = ["SPACE", "DEFAULT", "coordinate_search", "measure", "tune"]

# the searched values of each parameter (the first is the library default)
SPACE = {
    "relax_small": (16, 8, 32),
    "relax_frac": ((1, 10), (1, 20), (1, 5)),
    "relax_wmax": (256, 128, 512),
    "solve_w": (128, 64, 192),
    "solve_ent": (0, 8192, 12288),          # 0: the library's size-dependent default
    "tensor_cores": (1, 0),
    "tc_panel_min": (128, 512, 1024),
}
DEFAULT = {k: v[0] for k, v in SPACE.items()}


def to_options(params: dict) -> dict:
    """Library option keywords of a parameter set."""
    o = dict(params)
    num, den = o.pop("relax_frac")
    o["relax_num"], o["relax_den"] = num, den
    return o


def coordinate_search(objective, space=SPACE, start=None, rr_target=1e-8, sweeps=2, min_gain=0.02, log=None):
    """Returns (best parameters, best seconds, evaluations list). A parameter
    set is admissible when objective(params) returns an rr <= rr_target;
    inadmissible or failing sets (exceptions) are skipped. Each distinct set
    is evaluated once."""
    cache = {}

    def key(p):
        return tuple(sorted((k, v if not isinstance(v, list) else tuple(v)) for k, v in p.items()))

    def ev(p):
        k = key(p)
        if k not in cache:
            try:
                sec, rr = objective(dict(p))
                ok = rr <= rr_target
            except Exception as e:          # noqa: BLE001 - a failing set is just not admissible
                sec, rr, ok = float("inf"), float("nan"), False
                if log:
                    log(f"  {p}: failed ({e})")
            cache[k] = (sec if ok else float("inf"), rr)
            if log:
                log(f"  {p}: {sec * 1e3:.3f} ms rr {rr:.2e}{'' if ok else ' (not admissible)'}")
        return cache[k][0]

    best = dict(start or {k: v[0] for k, v in space.items()})
    best_t = ev(best)
    for _ in range(sweeps):
        moved = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                cand = dict(best)
                cand[name] = v
                t = ev(cand)
                if t < best_t * (1 - min_gain):
                    best, best_t, moved = cand, t, True
        if not moved:
            break
    evals = [(dict(k), v[0], v[1]) for k, v in cache.items()]
    return best, best_t, evals


def measure(pattern, value_sets, precision="mixed", ordering="nd", reps=3, warmup=1):
    """Device objective over one pattern: options -> (median seconds of a
    factor + solve on the resident pattern over the value sets, worst RR).
    pattern = (n, m, H_colptr, H_rowidx, J_rowptr, J_colidx); value_sets =
    list of (H_vals, J_vals, r_x, r_y, delta, gamma) CUDA tensors."""
    import torch

    import paper_2110_03636_b300 as K

    def objective(params):
        s = K.KKTSolver(*pattern, precision=precision, ordering=ordering, **to_options(params))
        try:
            ts, rr = [], 0.0
            for t in range(warmup + reps * len(value_sets)):
                Hv, Jv, rx, ry, delta, gamma = value_sets[t % len(value_sets)]
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.factor(Hv, Jv, delta, gamma)
                s.solve(rx, ry)
                torch.cuda.synchronize()
                if t >= warmup:
                    ts.append(time.perf_counter() - t0)
                    rr = max(rr, s.info.rr)
            return float(np.median(ts)), rr
        finally:
            s.close()
    return objective


def tune(pattern, value_sets, precision="mixed", ordering="nd", rr_target=1e-8, sweeps=2, log=None):
    """Measured coordinate search on the device; returns (library option
    keywords of the best set, its seconds, the defaults' seconds, evaluations)."""
    obj = measure(pattern, value_sets, precision, ordering)
    best, best_t, evals = coordinate_search(obj, rr_target=rr_target, sweeps=sweeps, log=log)
    t_def = next(t for p, t, _ in evals if p == {k: (v if not isinstance(v, list) else tuple(v))
                                                  for k, v in DEFAULT.items()})
    return to_options(best), best_t, t_def, evals
