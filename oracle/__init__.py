"""CPU oracle for the hybrid direct-iterative KKT method -- TEST INFRASTRUCTURE.

Plain, slow, single-threaded FP64 restatement of what the CUDA path computes
(symbolic analysis S1-S5, assembly of H_gamma = H~ + delta I + gamma J^T J,
Cholesky, CG on the Schur complement S = J H_gamma^-1 J^T, residuals).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA product path.

The C part (``kkt_oracle.c``) is compiled with plain gcc by ``build()``;
``reduce4x4``/``recover4x4`` (the 4x4 <-> 2x2 reduction of Sec. 3) are
numpy/scipy.

Parity status: S2 (the AMD order) and S2' (nested dissection) are pinned by
the special cases in the tests (zero fill on trees, identity on cliques,
hand-worked graphs, separator properties, valid permutation, brute-force
fill) and otherwise only by agreement with the library's independent
implementation ("parity unpinned" beyond those).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kkt_oracle.c")
_LIB = os.path.join(_HERE, "libkkt_oracle.so")
_lib = None

# S5 relaxation parameters used unless a caller overrides them
RELAX_SMALL, RELAX_NUM, RELAX_DEN, RELAX_WMAX = 16, 1, 10, 256


def build(force=False):
    """Compile the oracle with gcc (no BLAS, no OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        L.orc_analyse.restype = P
        L.orc_analyse.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i64p, i32p,
                                  C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                  C.POINTER(C.c_int32)]
        L.orc_analyse_perm.restype = P
        L.orc_analyse_perm.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i64p, i32p, C.c_int32, C.c_int32,
                                       C.c_int32, C.c_int32, C.c_int32, C.c_int32, i32p, C.POINTER(C.c_int32)]
        L.orc_sym_info.argtypes = [P, i64p]
        L.orc_sym_flops.restype = C.c_double
        L.orc_sym_flops.argtypes = [P]
        for nm in ("orc_sym_amd", "orc_sym_perm", "orc_sym_parent"):
            getattr(L, nm).argtypes = [P, i32p]
        L.orc_sym_colcount.argtypes = [P, i64p]
        L.orc_sym_lpattern.argtypes = [P, i64p, i32p]
        L.orc_sym_supernodes.argtypes = [P, i32p, i64p, i32p, i32p]
        L.orc_sym_free.argtypes = [P]
        L.orc_factor.restype = P
        L.orc_factor.argtypes = [P, f64p, f64p, C.c_double, C.c_double, C.POINTER(C.c_int32)]
        L.orc_factor_sample.restype = P
        L.orc_factor_sample.argtypes = [P, f64p, f64p, C.c_double, C.c_double, C.c_int64, f64p, f64p]
        L.orc_fail_col.restype = C.c_int64
        L.orc_fail_col.argtypes = [P]
        L.orc_get_L.argtypes = [P, i64p, i32p, f64p]
        L.orc_hsolve.argtypes = [P, f64p, f64p]
        L.orc_solve.restype = C.c_int32
        L.orc_solve.argtypes = [P, f64p, f64p, C.c_double, C.c_double, f64p, f64p, C.c_double,
                                C.c_double, C.c_int32, C.c_int32, C.c_double, f64p, f64p, f64p]
        L.orc_residual.argtypes = [P, f64p, f64p, C.c_double, f64p, f64p, f64p, f64p, f64p]
        L.orc_residual_vec.argtypes = [P, f64p, f64p, C.c_double, f64p, f64p, f64p, f64p, f64p, f64p]
        L.orc_num_free.argtypes = [P]
        _lib = L
    return _lib


def _c(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a if a.size else np.zeros(1, dt)


class Symbolic:
    """S1-S5 of the pinned symbolic analysis for one (H~, J) pattern."""

    def __init__(self, n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, *, relax_small=RELAX_SMALL,
                 relax_num=RELAX_NUM, relax_den=RELAX_DEN, wmax=RELAX_WMAX, ordering="amd", user_order=None,
                 nd_leaf=64):
        L = _load()
        self.n, self.m = int(n), int(m)
        st = C.c_int32(0)
        code = {"amd": 0, "natural": 1, "nd": 2, "user": 3}[ordering if user_order is None else "user"]
        uo = _c(user_order if user_order is not None else np.zeros(1), np.int32)
        self._h = L.orc_analyse_perm(self.n, self.m, _c(H_colptr, np.int64), _c(H_rowidx, np.int32),
                                     _c(J_rowptr, np.int64), _c(J_colidx, np.int32),
                                     relax_small, relax_num, relax_den, wmax, code, int(nd_leaf), uo,
                                     C.byref(st))
        if st.value != 0 or not self._h:
            self._h = None
            raise ValueError(f"oracle analyse: invalid input (status {st.value})")
        info = np.zeros(5, np.int64)
        L.orc_sym_info(self._h, info)
        self.nsuper = int(info[1])
        self.nnzL = int(info[2])
        self.n_snrows = int(info[3])
        self.panel_entries = int(info[4])
        self.flops = float(L.orc_sym_flops(self._h))

    def _get(self, fn, size, dt):
        a = np.zeros(size, dt)
        getattr(_load(), fn)(self._h, a)
        return a

    @property
    def amd_order(self):
        return self._get("orc_sym_amd", self.n, np.int32)

    @property
    def perm(self):
        return self._get("orc_sym_perm", self.n, np.int32)

    @property
    def parent(self):
        return self._get("orc_sym_parent", self.n, np.int32)

    @property
    def colcount(self):
        return self._get("orc_sym_colcount", self.n, np.int64)

    def l_pattern(self):
        """Strictly-lower pattern of L by columns (final labels)."""
        Lp = np.zeros(self.n + 1, np.int64)
        Li = np.zeros(max(1, self.nnzL - self.n), np.int32)
        _load().orc_sym_lpattern(self._h, Lp, Li)
        return Lp, Li[: self.nnzL - self.n]

    def supernodes(self):
        """(start[nsuper+1], rowptr[nsuper+1], rows, parent[nsuper])."""
        start = np.zeros(self.nsuper + 1, np.int32)
        rowptr = np.zeros(self.nsuper + 1, np.int64)
        rows = np.zeros(max(1, self.n_snrows), np.int32)
        par = np.zeros(max(1, self.nsuper), np.int32)
        _load().orc_sym_supernodes(self._h, start, rowptr, rows, par)
        return start, rowptr, rows[: self.n_snrows], par[: self.nsuper]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_sym_free(self._h)
            self._h = None


class Factor:
    """Cholesky of P(H~ + delta I + gamma J^T J)P^T on a Symbolic pattern."""

    def __init__(self, sym: Symbolic, H_vals, J_vals, delta, gamma):
        L = _load()
        self.sym = sym
        self.H_vals = _c(H_vals, np.float64)
        self.J_vals = _c(J_vals, np.float64)
        self.delta, self.gamma = float(delta), float(gamma)
        st = C.c_int32(0)
        self._h = L.orc_factor(sym._h, self.H_vals, self.J_vals, self.delta, self.gamma, C.byref(st))
        self.status = int(st.value)           # 0 ok, 2 not SPD
        self.fail_col = int(L.orc_fail_col(self._h))

    @property
    def ok(self):
        return self.status == 0

    def L_csc(self):
        """L in CSC, final labels, diagonal first in each column."""
        n, nnz = self.sym.n, self.sym.nnzL
        Lp = np.zeros(n + 1, np.int64)
        Li = np.zeros(nnz, np.int32)
        Lx = np.zeros(nnz, np.float64)
        _load().orc_get_L(self._h, Lp, Li, Lx)
        return Lp, Li, Lx

    def hsolve(self, b):
        """H_delta^-1 b in the original labels."""
        x = np.zeros(self.sym.n)
        _load().orc_hsolve(self._h, _c(b, np.float64), x)
        return x

    def solve(self, r_x, r_y, *, delta2=1e-9, rtol=1e-12, maxit=1000, ir_maxit=0, ir_rtol=1e-8):
        """Returns (dx, dy, info); info = dict(iters, rr, be, ir, delta2,
        cg_status, inertia_ok, status)."""
        n, m = self.sym.n, self.sym.m
        dx = np.zeros(n)
        dy = np.zeros(max(m, 1))
        info = np.zeros(8)
        ret = _load().orc_solve(self._h, self.H_vals, self.J_vals, self.delta, self.gamma,
                                _c(r_x, np.float64), _c(r_y, np.float64),
                                delta2, rtol, maxit, ir_maxit, ir_rtol, dx, dy, info)
        return dx, dy[:m], dict(iters=int(info[0]), rr=float(info[1]), be=float(info[2]),
                                ir=int(info[3]), delta2=float(info[4]), cg_status=int(info[5]),
                                inertia_ok=bool(info[6]), status=int(ret))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_num_free(self._h)
            self._h = None


class FactorSample(Factor):
    """Assembly + the first ``kmax`` rows of the oracle's factorization, timed
    in C (for a bounded CPU-baseline sample). ``times`` = (assembly s, rows s),
    ``work`` = inner-loop updates done; the full factorization performs
    sum_j (c_j - 1)(c_j - 2)/2 of them (c_j = column counts)."""

    def __init__(self, sym: Symbolic, H_vals, J_vals, delta, gamma, kmax):
        L = _load()
        self.sym = sym
        self.H_vals = _c(H_vals, np.float64)
        self.J_vals = _c(J_vals, np.float64)
        self.delta, self.gamma = float(delta), float(gamma)
        t = np.zeros(2)
        w = np.zeros(1)
        self._h = L.orc_factor_sample(sym._h, self.H_vals, self.J_vals, self.delta, self.gamma, int(kmax), t, w)
        self.times = (float(t[0]), float(t[1]))
        self.work = float(w[0])
        self.status = 0
        self.fail_col = -1


def factor_regularized(sym: Symbolic, H_vals, J_vals, gamma, delta_min=1e-9, delta_max=1e-6, delta_prev=0.0):
    """Algorithm 1's delta_1 loop (its lines from "delta_1 <- 0" to the end of
    the while loop) with the sequence rule of Sec. 4.1: try the Cholesky with
    delta_1 = 0; while it fails and delta_1 <= delta_max / 2, set delta_1 on
    the first retry back to the previous matrix's accepted value
    ``delta_prev`` (delta_min when that was 0) and double it afterwards (the
    garbled update is read as "double delta_1"). Returns (Factor of the last
    trial, delta_1); the caller carries delta_1 to the next matrix when the
    factorization succeeded."""
    d1 = 0.0
    fac = Factor(sym, H_vals, J_vals, d1, gamma)
    while not fac.ok and d1 <= delta_max / 2:
        if d1 == 0.0:
            d1 = delta_prev if delta_prev > 0 else delta_min
        else:
            d1 = 2.0 * d1
        fac = Factor(sym, H_vals, J_vals, d1, gamma)
    return fac, d1


def residual(sym: Symbolic, H_vals, J_vals, delta, r_x, r_y, dx, dy, *, vector=False):
    """RR, BE, ||res||_2, ||K_delta||_inf of [dx;dy] for K_delta = [H~+delta I, J^T; J, 0]
    (BE and RR as defined in Sec. 5.1, ||K||_2 estimated by ||K||_inf).
    With ``vector=True`` the dict also holds ``res`` = b - K_delta [dx; dy]
    as ``res_x`` (n) and ``res_y`` (m)."""
    out = np.zeros(4)
    n, m = sym.n, sym.m
    rv = np.zeros(n + max(m, 1))
    _load().orc_residual_vec(sym._h, _c(H_vals, np.float64), _c(J_vals, np.float64), float(delta),
                             _c(r_x, np.float64), _c(r_y, np.float64),
                             _c(dx, np.float64), _c(dy, np.float64), out, rv)
    d = dict(rr=float(out[0]), be=float(out[1]), res=float(out[2]), knorm=float(out[3]))
    if vector:
        d["res_x"], d["res_y"] = rv[:n].copy(), rv[n:n + m].copy()
    return d


def solve_system(sys, *, ir_maxit=0, **kw):
    """Analyse + factor + solve one workloads.KKTSystem; returns (sym, fac, dx, dy, info)."""
    sym_kw = {k: v for k, v in kw.items() if k in ("relax_small", "relax_num", "relax_den", "wmax", "ordering")}
    sol_kw = {k: v for k, v in kw.items() if k in ("delta2", "rtol", "maxit", "ir_rtol")}
    sym = Symbolic(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx, **sym_kw)
    fac = Factor(sym, sys.H_vals, sys.J_vals, sys.delta, sys.gamma)
    if not fac.ok:
        return sym, fac, None, None, dict(status=2)
    dx, dy, info = fac.solve(sys.r_x, sys.r_y, ir_maxit=ir_maxit, **sol_kw)
    return sym, fac, dx, dy, info


# --------------------------------------------------------------------------
# 4x4 <-> 2x2 reduction (Sec. 3, eqs. linsys4x4 / linsys2x2), numpy + scipy
# --------------------------------------------------------------------------
def reduce4x4(p):
    """From the parts of a 4x4 system (dict from workloads.random_4x4_parts)
    form H~ = H + D_x + J_d^T D_s J_d (lower CSC, pattern = pat(H) U
    pat(J_d^T J_d) U diag) and r_x = r~_x + J_d^T (D_s r_yd + r_s)."""
    import scipy.sparse as sp
    n = p["n_x"]
    H = sp.csc_matrix((p["H_vals"], p["H_rowidx"], p["H_colptr"]), shape=(n, n))
    Hfull = H + sp.tril(H, -1).T
    Jd = sp.csr_matrix((p["Jd_vals"], p["Jd_colidx"], p["Jd_rowptr"]), shape=(p["m_d"], n))
    Ht = Hfull + sp.diags(p["D_x"]) + (Jd.T @ sp.diags(p["D_s"]) @ Jd)
    # structural pattern: H's entries, J_d^T J_d's entries and the diagonal
    pat = (abs(Hfull) + abs(Jd.T) @ abs(Jd) + sp.eye(n)).tocsc()
    low = sp.tril(pat).tocsc()
    low.sort_indices()
    Htd = Ht.toarray()
    rows = low.indices.astype(np.int32)
    cols = np.repeat(np.arange(n), np.diff(low.indptr))
    vals = Htd[rows, cols]
    r_x = p["r_xt"] + Jd.T @ (p["D_s"] * p["r_yd"] + p["r_s"])
    return low.indptr.astype(np.int64), rows, vals, np.asarray(r_x)


def recover4x4(p, dx):
    """Delta s = J_d dx - r_yd, Delta y_d = D_s Delta s - r_s (Sec. 3)."""
    import scipy.sparse as sp
    Jd = sp.csr_matrix((p["Jd_vals"], p["Jd_colidx"], p["Jd_rowptr"]), shape=(p["m_d"], p["n_x"]))
    ds = Jd @ dx - p["r_yd"]
    dyd = p["D_s"] * ds - p["r_s"]
    return ds, dyd


# --------------------------------------------------------------------------
# Symmetrized Ruiz scaling (Sec. 4.1: the system is scaled before gamma and
# delta_min are chosen; D. Ruiz, "A scaling algorithm to equilibrate both
# rows and columns norms in matrices", RAL-TR-2001-034), numpy
# --------------------------------------------------------------------------
def ruiz_scaling(sys, iters):
    """Diagonal D = diag(D_x, D_y) making the rows of D K D (K = [H~, J^T;
    J, 0], symmetric) close to unit infinity norm: D = I, then ``iters``
    times, with the row norms r_i = max_j (D_i |K_ij|) D_j of the current
    scaled matrix (all rows from the same D), D_i <- D_i / sqrt(r_i) for
    every row with r_i > 0. Returns (D_x, D_y)."""
    n, m = sys.n, sys.m
    Hp, Hi, Hv = sys.H_colptr, sys.H_rowidx, np.abs(sys.H_vals)
    cols = np.repeat(np.arange(n), np.diff(Hp))
    Jp, Jc, Jv = sys.J_rowptr, sys.J_colidx, np.abs(sys.J_vals)
    jrow = np.repeat(np.arange(m), np.diff(Jp))
    D = np.ones(n + m)
    for _ in range(iters):
        r = np.zeros(n + m)
        # H~ entry (i, j) of the lower triangle lies in rows i and j
        np.maximum.at(r, Hi, (D[Hi] * Hv) * D[cols])
        np.maximum.at(r, cols, (D[cols] * Hv) * D[Hi])
        # J entry (r, c) lies in row n + r and (as J^T) in row c
        np.maximum.at(r, n + jrow, (D[n + jrow] * Jv) * D[Jc])
        np.maximum.at(r, Jc, (D[Jc] * Jv) * D[n + jrow])
        pos = r > 0
        D = np.where(pos, D / np.sqrt(np.where(pos, r, 1.0)), D)
    return D[:n].copy(), D[n:].copy()


def scale_system(sys, Dx, Dy):
    """The scaled system D K D x^ = D b as a new KKTSystem (values and
    right-hand sides scaled; delta and gamma unchanged, so they act on the
    scaled system). The solution of the original is x = D x^."""
    s = sys.copy()
    cols = np.repeat(np.arange(sys.n), np.diff(sys.H_colptr))
    s.H_vals = (Dx[sys.H_rowidx] * sys.H_vals) * Dx[cols]
    jrow = np.repeat(np.arange(sys.m), np.diff(sys.J_rowptr))
    s.J_vals = (Dy[jrow] * sys.J_vals) * Dx[sys.J_colidx]
    s.r_x = Dx * sys.r_x
    s.r_y = Dy * sys.r_y
    return s


# --------------------------------------------------------------------------
# Krylov variants on the Schur complement (Sec. 4, the discussion after eqs.
# Schur1-Schur2: CG or MINRES on S y = J w - r_y, with or without the
# multiplicative preconditioner M = (J J^T)^-1 J H_gamma J^T (J J^T)^-1),
# numpy + the oracle's Cholesky for H_gamma^-1 + a sparse LU of J J^T
# --------------------------------------------------------------------------
def _csr(sys):
    import scipy.sparse as sp
    J = sp.csr_matrix((sys.J_vals, sys.J_colidx, sys.J_rowptr), shape=(sys.m, sys.n))
    H = sp.csc_matrix((sys.H_vals, sys.H_rowidx, sys.H_colptr), shape=(sys.n, sys.n))
    return J, (H + sp.tril(H, -1).T).tocsr()


def schur_variant(fac: Factor, sys, method="pcg", rtol=1e-12, maxit=1000):
    """Solves K_delta [dx; dy] = [r_x; r_y] through eq. Schur1 with
    ``method`` = "pcg" (CG preconditioned by M, M applied as written: two
    solves with J J^T around J H_gamma J^T) or "minres" (MINRES of Paige and
    Saunders on S, unpreconditioned), stopping on ||b_S - S y|| <= rtol ||b_S||
    as the recurrence reports it, then eq. Schur2 for dx. Returns
    (dx, dy, iterations)."""
    import scipy.sparse.linalg as spla
    J, Hf = _csr(sys)
    g, d = fac.gamma, fac.delta
    hinv = fac.hsolve
    rhx = sys.r_x + g * (J.T @ sys.r_y)
    bS = J @ hinv(rhx) - sys.r_y
    S = lambda p: J @ hinv(J.T @ p)
    nb = np.linalg.norm(bS)
    y = np.zeros(sys.m)
    it = 0
    if nb == 0:
        pass
    elif method == "pcg":
        JJt = spla.splu((J @ J.T).tocsc())
        Hg = lambda v: Hf @ v + d * v + g * (J.T @ (J @ v))
        M = lambda r: JJt.solve(J @ Hg(J.T @ JJt.solve(r)))
        r = bS.copy()
        z = M(r)
        p = z.copy()
        rho = r @ z
        while it < maxit:
            q = S(p)
            a = rho / (p @ q)
            y += a * p
            r -= a * q
            it += 1
            if np.linalg.norm(r) <= rtol * nb:
                break
            z = M(r)
            rho2 = r @ z
            p = z + (rho2 / rho) * p
            rho = rho2
    elif method == "minres":
        # Lanczos on S with v_1 = b_S / ||b_S||, QR of the tridiagonal by Givens
        # rotations (c, s), search directions w updated by the last two
        v_old, v = np.zeros(sys.m), bS / nb
        beta, eta = nb, nb
        c_old = c = 1.0
        s_old = s = 0.0
        w_old2, w_old = np.zeros(sys.m), np.zeros(sys.m)
        while it < maxit:
            p = S(v)
            alpha = v @ p
            p = p - alpha * v - beta * v_old
            beta_new = np.linalg.norm(p)
            dlt = c * alpha - c_old * s * beta
            r1 = np.hypot(dlt, beta_new)
            r2 = s * alpha + c_old * c * beta
            r3 = s_old * beta
            c_new, s_new = dlt / r1, beta_new / r1
            w = (v - r3 * w_old2 - r2 * w_old) / r1
            y += c_new * eta * w
            eta = -s_new * eta
            it += 1
            if abs(eta) <= rtol * nb or beta_new == 0:
                break
            v_old, v = v, p / beta_new
            w_old2, w_old = w_old, w
            c_old, c, s_old, s = c, c_new, s, s_new
            beta = beta_new
    else:
        raise ValueError(method)
    dx = hinv(rhx - J.T @ y)
    return dx, y, it
