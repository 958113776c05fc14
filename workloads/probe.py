"""Small runs of the library on one workload, for the ncu captures
summarised under profiles/ (every capture there names its command here):

    python -m workloads.probe dense WA WC REPS   # dense-front system: fronts A (WA columns),
                                                 # B (100) and the root C (WC), natural order;
                                                 # REPS mixed factorizations + solves
    python -m workloads.probe grid NAME REPS     # a named grid workload (make_config), ND
                                                 # order; REPS mixed factorizations + solves

Every input is seeded; each run prints the factor time and the solve's
relative residual.
"""
import sys
import time

import numpy as np

from . import KKTSystem, lower_csc, make_config


def dense_fronts(wa, wc, m=60, seed=1):
    """n = wa + 100 + wc, natural order: blocks A (columns 0..wa-1) and B (the
    next 100) are dense and both couple densely to block C (the last wc); A
    and B do not couple. Their fronts are A (wa columns, wc rows below), B
    (100 columns, wc rows below) and C (the root, wc columns). H is
    diagonally dominant (SPD); J has m rows of two adjacent unit entries."""
    rng = np.random.default_rng(seed)
    n = wa + 100 + wc
    rows, cols, vals = [], [], []
    for lo, hi in ((0, wa), (wa, wa + 100)):
        for j in range(lo, hi):
            r = np.r_[np.arange(j + 1, hi), np.arange(wa + 100, n)]
            rows.append(r)
            cols.append(np.full(r.size, j))
            vals.append(rng.uniform(-1, 1, r.size) / np.sqrt(n))
    for j in range(wa + 100, n):
        r = np.arange(j + 1, n)
        rows.append(r)
        cols.append(np.full(r.size, j))
        vals.append(rng.uniform(-1, 1, r.size) / np.sqrt(n))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    diag = np.zeros(n)
    np.add.at(diag, rows, np.abs(vals))
    np.add.at(diag, cols, np.abs(vals))
    diag += rng.uniform(0.5, 2.0, n)
    Hp, Hi, Hv = lower_csc(n, rows, cols, vals, diag)
    c = np.sort(rng.choice(n - 1, m, replace=False))
    Jp = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    Ji = np.stack([c, c + 1], 1).ravel().astype(np.int32)
    Jv = np.ones(2 * m)
    return KKTSystem(n=n, m=m, H_colptr=Hp, H_rowidx=Hi, H_vals=Hv, J_rowptr=Jp, J_colidx=Ji, J_vals=Jv,
                     r_x=rng.standard_normal(n), r_y=rng.standard_normal(m), delta=1e-8, gamma=1e2)


def run(x, ordering, reps):
    import torch

    import paper_2110_03636_b300 as K
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")   # noqa: E731
    s = K.KKTSolver(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx, precision="mixed",
                    ordering=ordering)
    H, J, rx, ry = cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y)
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.factor(H, J, x.delta, x.gamma)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.solve(rx, ry, check=False)
        print(f"factor {1e3 * (t1 - t0):.2f} ms, rr {s.info.rr:.2e}", flush=True)
    s.close()


def main(argv):
    if argv[0] == "dense":
        run(dense_fronts(int(argv[1]), int(argv[2])), "natural", int(argv[3]))
    elif argv[0] == "grid":
        run(make_config(argv[1]), "nd", int(argv[2]))
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
