"""Seeded synthetic KKT inputs shaped like interior-method systems.

This module only draws inputs. It holds none of the method's arithmetic
(no reduction, no Cholesky, no CG). Both the CUDA path's tests/bench and the
CPU oracle read the arrays it returns.

A 2x2 KKT system (Sec. 3, eq. linsys2x2) is given by
  * ``H``: the (1,1) block H~ (n x n, symmetric) as the LOWER triangle in CSC
    form, diagonal included: ``H_colptr`` int64[n+1], ``H_rowidx`` int32, rows
    ascending inside each column, the diagonal first; ``H_vals`` float64.
  * ``J``: the constraint Jacobian (m x n) in CSR form: ``J_rowptr`` int64[m+1],
    ``J_colidx`` int32 ascending inside each row; ``J_vals`` float64.
  * ``r_x`` (n) and ``r_y`` (m) right-hand sides, float64.

The paper's matrices come from AC optimal power flow (Sec. 5, Table 2), which
are not available here. The stand-in is a weighted grid-graph Laplacian plus a
barrier diagonal whose entries spread over many decades (the D_x = X^-1 Z_x
term of Sec. 2), and a sparse, local, full-row-rank J.

Recipe (every draw comes from ``numpy.random.default_rng(seed)``, PCG64, in
exactly this order):
  1. edge weights w_e ~ U(0.5, 2): x-edges first (row-major over the grid,
     idx = x + a*y (+ a*b*z)), then y-edges, then z-edges;
  2. barrier: ``rng.permutation(n)``; its first round(f*n) entries get
     10**U(-e, e) added to the diagonal, exponents drawn in that order;
  3. J unit columns: first m entries of ``rng.permutation(n)``, sorted
     ascending (row i has 1.0 at c_i; distinct columns => full row rank);
  4. local counts k_i ~ UniformInt[k_lo, k_hi] (``rng.integers``, size m);
  5. local columns: for each row, k_i distinct positions of the window
     [max(0,c_i-w), min(n-1,c_i+w)] minus {c_i}, drawn by Floyd's
     sampling (R. W. Floyd, "A sample of brilliance", CACM 30(9), 1987),
     vectorised over rows, one ``rng.random(m)`` per step;
  6. local values N(0,1) (``rng.standard_normal``) in row-major order;
  7. r_x ~ N(0,1) (n), r_y ~ N(0,1) (m).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "KKTSystem", "make_system", "CONFIGS", "make_config", "rescale_barrier",
    "serving_pattern", "random_tiny_system", "random_4x4_parts", "lower_csc",
]


@dataclasses.dataclass
class KKTSystem:
    n: int
    m: int
    H_colptr: np.ndarray
    H_rowidx: np.ndarray
    H_vals: np.ndarray
    J_rowptr: np.ndarray
    J_colidx: np.ndarray
    J_vals: np.ndarray
    r_x: np.ndarray
    r_y: np.ndarray
    delta: float
    gamma: float
    # bookkeeping for value updates on a fixed pattern (interior iterations)
    barrier_idx: np.ndarray | None = None     # indices carrying a barrier term
    barrier_val: np.ndarray | None = None     # current barrier values
    lap_diag: np.ndarray | None = None        # Laplacian diagonal (no barrier)
    name: str = ""

    def copy(self) -> "KKTSystem":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return KKTSystem(**kw)


def _grid_edges(dims):
    """Edges of a structured grid, x-edges first, then y, then z.

    dims = (a,) / (a, b) / (a, b, c); index = x + a*y + a*b*z.
    Returns (u, v) arrays with u < v.
    """
    dims = tuple(int(d) for d in dims)
    idx = np.arange(int(np.prod(dims)), dtype=np.int64).reshape(dims[::-1])
    us, vs = [], []
    # axis order in idx is (z, y, x); x is the last axis.
    for ax in range(len(dims) - 1, -1, -1):
        sl_lo = [slice(None)] * len(dims)
        sl_hi = [slice(None)] * len(dims)
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        us.append(idx[tuple(sl_lo)].ravel())
        vs.append(idx[tuple(sl_hi)].ravel())
    return np.concatenate(us), np.concatenate(vs)


def lower_csc(n, rows, cols, vals, diag):
    """Lower CSC from strictly-lower (rows > cols) triples plus a full
    diagonal. Entries in a column: diagonal first, then rows ascending."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    r = np.concatenate([np.arange(n, dtype=np.int64), rows])
    c = np.concatenate([np.arange(n, dtype=np.int64), cols])
    x = np.concatenate([np.asarray(diag, np.float64), np.asarray(vals, np.float64)])
    order = np.lexsort((r, c))
    r, c, x = r[order], c[order], x[order]
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, c + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, r.astype(np.int32), x


def _csr(nrows, rows, cols, vals):
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, np.float64)[order]
    rowptr = np.zeros(nrows + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), vals


def local_jacobian(n, m, rng, k_lo, k_hi, window):
    """J (m x n) with one 1.0 per row at distinct sorted columns c_i plus
    k_i ~ UniformInt[k_lo, k_hi] N(0,1) entries at distinct columns of
    [c_i - window, c_i + window] (clipped to [0, n)) other than c_i."""
    c = np.sort(rng.permutation(n)[:m]).astype(np.int64)
    k = rng.integers(k_lo, k_hi + 1, size=m).astype(np.int64)
    lo = np.maximum(0, c - window)
    hi = np.minimum(n - 1, c + window)
    s = hi - lo            # window size without c_i itself
    if np.any(s < k):
        raise ValueError("window too small for the requested local count")
    # Floyd's algorithm, vectorised over rows: for step t = 0..k_i-1,
    # jj = s - k + t, draw pick in [0, jj]; if already chosen, take jj.
    chosen = np.full((m, k_hi), -1, np.int64)
    for t in range(k_hi):
        u = rng.random(m)
        active = t < k
        jj = s - k + t
        pick = np.minimum((u * (jj + 1)).astype(np.int64), jj)
        dup = np.zeros(m, bool)
        for q in range(t):
            dup |= chosen[:, q] == pick
        val = np.where(dup, jj, pick)
        chosen[:, t] = np.where(active, val, -1)
    colm = lo[:, None] + chosen
    colm = np.where(colm >= c[:, None], colm + 1, colm)
    mask = chosen >= 0
    vals_local = rng.standard_normal(int(k.sum()))
    row_ids = np.repeat(np.arange(m, dtype=np.int64), k_hi).reshape(m, k_hi)
    rows_all = np.concatenate([np.arange(m, dtype=np.int64), row_ids[mask]])
    cols_all = np.concatenate([c, colm[mask]])
    vals_all = np.concatenate([np.ones(m), vals_local])
    return _csr(m, rows_all, cols_all, vals_all)


def make_system(dims, m, *, seed, barrier_frac, barrier_exp, k_lo, k_hi, window,
                delta=1e-8, gamma=1e4, name=""):
    """Build one seeded KKT system on a grid (see the module recipe)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    u, v = _grid_edges(dims)
    w = rng.uniform(0.5, 2.0, size=u.size)
    lap_diag = np.zeros(n)
    np.add.at(lap_diag, u, w)
    np.add.at(lap_diag, v, w)
    perm = rng.permutation(n)
    nb = int(round(barrier_frac * n))
    bexp = rng.uniform(-barrier_exp, barrier_exp, size=nb)
    order = np.argsort(perm[:nb], kind="stable")
    bidx = perm[:nb][order].astype(np.int64)
    bval = (10.0 ** bexp)[order]
    diag = lap_diag.copy()
    diag[bidx] += bval
    J_rowptr, J_colidx, J_vals = local_jacobian(n, m, rng, k_lo, k_hi, window)
    r_x = rng.standard_normal(n)
    r_y = rng.standard_normal(m)
    colptr, rowidx, vals = lower_csc(n, np.maximum(u, v), np.minimum(u, v), -w, diag)
    return KKTSystem(n, m, colptr, rowidx, vals, J_rowptr, J_colidx, J_vals,
                     r_x, r_y, float(delta), float(gamma), bidx, bval, lap_diag, name)


def rescale_barrier(sys: KKTSystem, seed) -> KKTSystem:
    """Next interior iteration on the same pattern: every barrier entry is
    multiplied by its own 10**U(-1,1) (cumulative), new r_x, r_y ~ N(0,1).
    Draws: exponents (one per barrier entry, ascending index), r_x, r_y."""
    rng = np.random.default_rng(seed)
    out = sys.copy()
    f = 10.0 ** rng.uniform(-1.0, 1.0, size=sys.barrier_idx.size)
    out.barrier_val = sys.barrier_val * f
    newdiag = sys.lap_diag.copy()
    newdiag[sys.barrier_idx] += out.barrier_val
    out.H_vals = sys.H_vals.copy()
    out.H_vals[sys.H_colptr[:-1]] = newdiag     # diagonal is first in each column
    out.r_x = rng.standard_normal(sys.n)
    out.r_y = rng.standard_normal(sys.m)
    return out


def reweight(sys: KKTSystem, seed) -> KKTSystem:
    """Same pattern, fresh values: edge weights U(0.5,2) and barrier
    10**U(-6,6) on the same barrier indices, drawn from ``seed`` (the
    batching workload's per-system values). J and the rhs are kept."""
    rng = np.random.default_rng(seed)
    out = sys.copy()
    n = sys.n
    Hp, Hi = sys.H_colptr, sys.H_rowidx
    col = np.repeat(np.arange(n), np.diff(Hp))
    off = Hi != col
    w = rng.uniform(0.5, 2.0, size=int(off.sum()))
    lap = np.zeros(n)
    np.add.at(lap, Hi[off], w)
    np.add.at(lap, col[off], w)
    bval = 10.0 ** rng.uniform(-6, 6, size=sys.barrier_idx.size)
    out.H_vals = sys.H_vals.copy()
    out.H_vals[off] = -w
    diag = lap.copy()
    diag[sys.barrier_idx] += bval
    out.H_vals[Hp[:-1]] = diag
    out.lap_diag, out.barrier_val = lap, bval
    return out


# The workloads. "dims" is the grid, a points along x (fastest index).
CONFIGS = {
    # plain FP64 method, small: 50x40 2-D grid, n=2000, m=1000
    "grid2d_n2000": dict(dims=(50, 40), m=1000, barrier_frac=0.3, barrier_exp=6,
                         k_lo=3, k_hi=5, window=100, delta=1e-8, gamma=1e4),
    # plain FP64 method at scale: 500x500 2-D grid, n=250000, m=125000
    "grid2d_n250k": dict(dims=(500, 500), m=125000, barrier_frac=0.3, barrier_exp=6,
                         k_lo=3, k_hi=6, window=500, delta=1e-8, gamma=1e4),
    # precision form: 100^3 3-D grid, n=1e6, m=5e5
    "grid3d_n1m": dict(dims=(100, 100, 100), m=500000, barrier_frac=0.4, barrier_exp=8,
                       k_lo=4, k_hi=8, window=500, delta=1e-8, gamma=1e6),
    # batching form: 200x100 2-D grid, n=20000, m=10000
    "grid2d_n20k": dict(dims=(200, 100), m=10000, barrier_frac=0.3, barrier_exp=6,
                        k_lo=3, k_hi=5, window=100, delta=1e-8, gamma=1e4),
}


def make_config(name, seed=0, **over):
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    return make_system(cfg.pop("dims"), cfg.pop("m"), seed=seed, name=name, **cfg)


def serving_pattern(side, seed=0):
    """Serving workload pattern: side x side 2-D grid, m = n/2, J as the
    20k batching workload (k in [3,5], window 100), gamma = 1e6."""
    n = side * side
    return make_system((side, side), n // 2, seed=seed, barrier_frac=0.3, barrier_exp=6,
                       k_lo=3, k_hi=5, window=100, delta=1e-8, gamma=1e6,
                       name=f"serve_grid2d_{side}")


def random_tiny_system(seed, n_lo=4, n_hi=40, density=0.15, spd=True, gamma=1e2):
    """Small random KKT system for brute-force checks.

    H~ = random sparse symmetric with a diagonal shift (SPD when ``spd``),
    J = m x n (m <= n/2) with a unit entry per row at distinct columns plus
    0-3 random entries. delta = 0.
    """
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi + 1))
    m = int(rng.integers(1, max(2, n // 2) + 1))
    mask = np.tril(rng.random((n, n)) < density, -1)
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(rows.size)
    diag = np.abs(rng.standard_normal(n)) + (n * 0.5 if spd else -0.5)
    colptr, rowidx, hv = lower_csc(n, rows, cols, vals, diag)
    c = np.sort(rng.permutation(n)[:m])
    Jr, Jc, Jv = [], [], []
    for i in range(m):
        extra = rng.choice(n, size=min(int(rng.integers(0, 4)), n), replace=False)
        for cc in sorted(set([int(c[i])]) | set(int(e) for e in extra)):
            Jr.append(i)
            Jc.append(cc)
            Jv.append(1.0 if cc == c[i] else float(rng.standard_normal()))
    rowptr, colidx, jv = _csr(m, Jr, Jc, Jv)
    return KKTSystem(n, m, colptr, rowidx, hv, rowptr, colidx, jv,
                     rng.standard_normal(n), rng.standard_normal(m), 0.0, float(gamma),
                     name=f"tiny{seed}")


def random_4x4_parts(seed, n_x, m_c, m_d):
    """Random parts of a 4x4 system (eq. linsys4x4): H (lower CSC, n_x x n_x),
    D_x (n_x), D_s (m_d), J (m_c x n_x CSR, unit entry per row), J_d
    (m_d x n_x CSR) and right-hand sides r~_x, r_s, r_y, r_yd."""
    rng = np.random.default_rng(seed)
    mask = np.tril(rng.random((n_x, n_x)) < 0.2, -1)
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(rows.size)
    diag = np.abs(rng.standard_normal(n_x)) + 1.0
    Hc, Hr, Hv = lower_csc(n_x, rows, cols, vals, diag)

    def rand_csr(mr, with_unit):
        R, Cc, V = [], [], []
        units = np.sort(rng.permutation(n_x)[:mr])
        for i in range(mr):
            extra = rng.choice(n_x, size=int(rng.integers(1, 4)), replace=False)
            s = set(int(e) for e in extra)
            if with_unit:
                s.add(int(units[i]))
            for cc in sorted(s):
                R.append(i)
                Cc.append(cc)
                V.append(1.0 if (with_unit and cc == units[i]) else float(rng.standard_normal()))
        return _csr(mr, R, Cc, V)

    Jp, Jc, Jv = rand_csr(m_c, True)
    Jdp, Jdc, Jdv = rand_csr(m_d, False)
    return dict(n_x=n_x, m_c=m_c, m_d=m_d, H_colptr=Hc, H_rowidx=Hr, H_vals=Hv,
                D_x=10.0 ** rng.uniform(-2, 2, n_x), D_s=10.0 ** rng.uniform(-2, 2, m_d),
                J_rowptr=Jp, J_colidx=Jc, J_vals=Jv,
                Jd_rowptr=Jdp, Jd_colidx=Jdc, Jd_vals=Jdv,
                r_xt=rng.standard_normal(n_x), r_s=rng.standard_normal(m_d),
                r_y=rng.standard_normal(m_c), r_yd=rng.standard_normal(m_d))


def grid_4x4_parts(name, m_d_frac=0.25, seed=7):
    """A 4x4 system (eq. linsys4x4) on a grid workload: H = the workload's
    H~ (Laplacian + barrier), D_x = 10^U(-2,2), J = the workload's J, and
    J_d with round(m_d_frac * n) rows of 2-4 N(0,1) entries at distinct
    columns within +-w of a uniform centre (w = the workload's window),
    D_s = 10^U(-4,4) (slack barriers spread over eight decades); right-hand
    sides N(0,1). Draw order: D_x, then per J_d row (centre, count, columns,
    values), then D_s, then r~_x, r_s, r_yd; r_y is the workload's."""
    base = make_config(name)
    rng = np.random.default_rng(seed)
    n = base.n
    w = CONFIGS[name]["window"]
    D_x = 10.0 ** rng.uniform(-2, 2, n)
    md = int(round(m_d_frac * n))
    R, Cc, V = [], [], []
    for r in range(md):
        c = int(rng.integers(0, n))
        k = int(rng.integers(2, 5))
        lo, hi = max(0, c - w), min(n, c + w + 1)
        cols = np.sort(lo + rng.choice(hi - lo, size=min(k, hi - lo), replace=False))
        vals = rng.standard_normal(cols.size)
        R += [r] * cols.size
        Cc += cols.tolist()
        V += vals.tolist()
    Jdp, Jdc, Jdv = _csr(md, R, Cc, V)
    D_s = 10.0 ** rng.uniform(-4, 4, md)
    return dict(n_x=n, m_c=base.m, m_d=md, H_colptr=base.H_colptr, H_rowidx=base.H_rowidx, H_vals=base.H_vals,
                D_x=D_x, D_s=D_s, J_rowptr=base.J_rowptr, J_colidx=base.J_colidx, J_vals=base.J_vals,
                Jd_rowptr=Jdp, Jd_colidx=Jdc, Jd_vals=Jdv,
                r_xt=rng.standard_normal(n), r_s=rng.standard_normal(md), r_y=base.r_y,
                r_yd=rng.standard_normal(md), delta=base.delta, gamma=base.gamma)
