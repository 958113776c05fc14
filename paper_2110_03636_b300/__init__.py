"""B300-native hybrid direct-iterative KKT solver (Python binding).

Thin ctypes binding over the C ABI in ``include/kkt.h`` (``libkkt.so``):
the functions here have the C names and only marshal arguments -- device
buffers are torch CUDA tensors (``.data_ptr()``) on the current stream, host
buffers are numpy arrays. Every step of the method runs in the library's
CUDA kernels; there is no CPU fallback: importing this package without a
built ``libkkt.so`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkkt.so")

KKT_FP64, KKT_MIXED = 0, 1
STATUS = {0: "ok", 1: "invalid", 2: "not_spd", 3: "cg_breakdown", 4: "cg_maxit",
          5: "oom", 6: "cuda", 7: "timeout", 8: "state", 9: "too_large"}
NOALLOC_MAX_ROWS = 1 << 20


class KKTError(RuntimeError):
    def __init__(self, fn, code):
        self.code = int(code)
        super().__init__(f"{fn}: {STATUS.get(self.code, self.code)} ({_lib.kkt_status_string(self.code).decode()})")


class kkt_options(C.Structure):
    _fields_ = [("gamma", C.c_double), ("delta2", C.c_double), ("cg_rtol", C.c_double),
                ("cg_maxit", C.c_int32), ("ir_maxit", C.c_int32), ("ir_rtol", C.c_double),
                ("precision", C.c_int32), ("ordering", C.c_int32), ("relax_small", C.c_int32),
                ("relax_num", C.c_int32), ("relax_den", C.c_int32), ("relax_wmax", C.c_int32),
                ("solve_w", C.c_int32), ("device", C.c_int32), ("debug_stall_piece", C.c_int32),
                ("spin_cycles", C.c_int64), ("profile", C.c_int32), ("nd_leaf", C.c_int32),
                ("tensor_cores", C.c_int32), ("solve_ctas", C.c_int32), ("solve_ent", C.c_int32),
                ("refine", C.c_int32), ("ruiz_iters", C.c_int32),
                ("krylov", C.c_int32), ("solve_sms", C.c_int32), ("tc_panel_min", C.c_int32)]


class kkt_info(C.Structure):
    _fields_ = [("cg_iters", C.c_int32), ("ir_steps", C.c_int32), ("cg_status", C.c_int32),
                ("delta2_used", C.c_int32), ("rr", C.c_double), ("be", C.c_double)]


class kkt_symbolic_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("nsuper", C.c_int64), ("nnz_l", C.c_int64),
                ("panel_entries", C.c_int64), ("update_entries", C.c_int64), ("sn_rows_total", C.c_int64),
                ("npieces", C.c_int64), ("nchunks", C.c_int64), ("nlevels", C.c_int32), ("pad", C.c_int32),
                ("flops", C.c_double), ("device_bytes", C.c_double), ("fwd_depth", C.c_int64),
                ("bwd_depth", C.c_int64), ("nsub", C.c_int64), ("nitems", C.c_int64), ("tc_flops", C.c_double)]


class kkt_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("pattern", C.c_int32), ("slot", C.c_int32), ("cg_iters", C.c_int32),
                ("ir_steps", C.c_int32), ("retried", C.c_int32), ("rr", C.c_double), ("be", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double)]


class kkt_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("bytes_used", C.c_int64), ("bytes_peak", C.c_int64), ("budget", C.c_int64),
                ("patterns", C.c_int32), ("slots", C.c_int32), ("inflight", C.c_int32),
                ("peak_inflight", C.c_int32), ("waiting", C.c_int32), ("pad", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libkkt.so is not built ({LIB_PATH}); run python paper_2110_03636_b300/build.py")
    L = C.CDLL(LIB_PATH)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.kkt_default_options.argtypes = [C.POINTER(kkt_options)]
    L.kkt_default_options.restype = None
    L.kkt_analyse.argtypes = [I64, I64, P, P, P, P, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_analyse_host.argtypes = [I64, I64, P, P, P, P, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_factor.argtypes = [P, P, P, D, D, P]
    L.kkt_solve.argtypes = [P, P, P, P, P, P]
    L.kkt_solve_multi.argtypes = [P, I32, P, P, P, P, P, P]
    L.kkt_factor_regularized.argtypes = [P, P, P, D, D, D, P, P]
    L.kkt_set_delta_prev.argtypes = [P, D]
    L.kkt_set_profile.argtypes = [P, I32]
    L.kkt_server_create.argtypes = [I64, I32, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_server_add_pattern.argtypes = [P, I64, I64, P, P, P, P, C.POINTER(I32)]
    L.kkt_server_submit.argtypes = [P, I32, P, P, D, D, P, P, P, P, C.POINTER(I64)]
    L.kkt_server_wait.argtypes = [P, I64, C.POINTER(kkt_request_info)]
    L.kkt_server_get_stats.argtypes = [P, C.POINTER(kkt_server_stats)]
    L.kkt_server_destroy.argtypes = [P]
    for nm in ("kkt_server_create", "kkt_server_add_pattern", "kkt_server_submit", "kkt_server_wait",
               "kkt_server_get_stats", "kkt_server_destroy"):
        getattr(L, nm).restype = I32
    L.kkt_get_scaling.argtypes = [P, P]
    L.kkt_analyse_like.argtypes = [P, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_factor_batch.argtypes = [P, I32, P, P, D, D, P, P]
    L.kkt_solve_batch.argtypes = [P, I32, P, P, P, P, P, P, P]
    L.kkt_factor_solve_host.argtypes = [P, P, P, D, D, P, P, P, P, P]
    L.kkt_hsolve.argtypes = [P, P, P, P]
    L.kkt_get_info.argtypes = [P, C.POINTER(kkt_info)]
    L.kkt_inertia.argtypes = [P, C.POINTER(I32)]
    L.kkt_symbolic_info_get.argtypes = [P, C.POINTER(kkt_symbolic_info)]
    L.kkt_get_symbolic.argtypes = [P] + [P] * 8
    L.kkt_get_factor_panels.argtypes = [P, P]
    L.kkt_get_profile.argtypes = [P, P, P, I32]
    L.kkt_get_solve_counters.argtypes = [P, P, I32]
    L.kkt_get_solve_trace.argtypes = [P, P, I64]
    L.kkt_get_solve_item_order.argtypes = [P, P, P, I64]
    L.kkt_residual_noalloc.argtypes = [I64, I64, P, P, P, P, P, P, D, P, P, P, P, P, P, P, P]
    L.kkt_destroy.argtypes = [P]
    L.kkt_analyse_4x4.argtypes = [I64, I64, I64, P, P, P, P, P, P, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_analyse_4x4_host.argtypes = [I64, I64, I64, P, P, P, P, P, P, C.POINTER(kkt_options), C.POINTER(P)]
    L.kkt_4x4_inner.argtypes = [P]
    L.kkt_4x4_inner.restype = P
    L.kkt_get_4x4_pattern.argtypes = [P, P, P, P]
    L.kkt_factor_4x4.argtypes = [P, P, P, P, P, P, D, D, P]
    L.kkt_solve_4x4.argtypes = [P, P, P, P, P, P, P, P, P, P]
    L.kkt_destroy_4x4.argtypes = [P]
    L.kkt_status_string.argtypes = [I32]
    L.kkt_status_string.restype = C.c_char_p
    for nm in ("kkt_analyse", "kkt_analyse_host", "kkt_factor", "kkt_solve", "kkt_solve_multi", "kkt_factor_batch", "kkt_solve_batch", "kkt_factor_regularized", "kkt_set_delta_prev", "kkt_set_profile", "kkt_get_scaling", "kkt_analyse_like", "kkt_factor_solve_host", "kkt_hsolve", "kkt_get_info",
               "kkt_inertia", "kkt_symbolic_info_get", "kkt_get_symbolic", "kkt_get_factor_panels", "kkt_get_profile", "kkt_get_solve_counters", "kkt_residual_noalloc",
               "kkt_get_solve_trace", "kkt_get_solve_item_order", "kkt_destroy", "kkt_analyse_4x4", "kkt_analyse_4x4_host", "kkt_get_4x4_pattern", "kkt_factor_4x4",
               "kkt_solve_4x4", "kkt_destroy_4x4"):
        getattr(L, nm).restype = I32
    return L


_lib = _load()
EXPORTED = ("kkt_default_options", "kkt_analyse", "kkt_analyse_host", "kkt_factor", "kkt_solve", "kkt_solve_multi", "kkt_factor_batch", "kkt_solve_batch", "kkt_factor_regularized", "kkt_set_delta_prev", "kkt_set_profile", "kkt_get_scaling", "kkt_analyse_like", "kkt_server_create", "kkt_server_add_pattern",
            "kkt_server_submit", "kkt_server_wait", "kkt_server_get_stats", "kkt_server_destroy", "kkt_factor_solve_host",
            "kkt_hsolve", "kkt_get_info", "kkt_inertia", "kkt_symbolic_info_get", "kkt_get_symbolic",
            "kkt_get_factor_panels", "kkt_get_profile", "kkt_get_solve_counters", "kkt_residual_noalloc",
            "kkt_get_solve_trace", "kkt_get_solve_item_order", "kkt_destroy", "kkt_status_string", "kkt_analyse_4x4", "kkt_analyse_4x4_host", "kkt_4x4_inner",
            "kkt_get_4x4_pattern", "kkt_factor_4x4", "kkt_solve_4x4", "kkt_destroy_4x4")
KERNEL_KINDS = ("assemble", "potrf", "trsm", "panel_update", "syrk", "extend_add", "tc_split", "cg_persistent",
                "residual", "tri_inv", "syrk_tc", "block")


def _check(fn, code):
    if code != 0:
        raise KKTError(fn, code)


def _np(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, (a.ctypes.data if a.size else None)


def _dev(t, n):
    """Device pointer of a contiguous float64 CUDA tensor with n elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return t.data_ptr() if n else None


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def kkt_default_options(**over) -> kkt_options:
    o = kkt_options()
    _lib.kkt_default_options(C.byref(o))
    for k, v in over.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": KKT_FP64, "mixed": KKT_MIXED}[v]
        if k == "ordering" and isinstance(v, str):
            v = {"amd": 0, "natural": 1, "nd": 2}[v]
        setattr(o, k, v)
    return o


def kkt_analyse(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, opt: kkt_options | None = None):
    keep = [_np(H_colptr, np.int64), _np(H_rowidx, np.int32), _np(J_rowptr, np.int64), _np(J_colidx, np.int32)]
    h = C.c_void_p()
    _check("kkt_analyse", _lib.kkt_analyse(int(n), int(m), keep[0][1], keep[1][1], keep[2][1], keep[3][1],
                                           C.byref(opt) if opt is not None else None, C.byref(h)))
    return h


def kkt_analyse_host(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, opt: kkt_options | None = None):
    """Host-only symbolic analysis (no GPU needed); returns a handle for the
    symbolic getters."""
    keep = [_np(H_colptr, np.int64), _np(H_rowidx, np.int32), _np(J_rowptr, np.int64), _np(J_colidx, np.int32)]
    h = C.c_void_p()
    _check("kkt_analyse_host", _lib.kkt_analyse_host(int(n), int(m), keep[0][1], keep[1][1], keep[2][1],
                                                     keep[3][1], C.byref(opt) if opt is not None else None,
                                                     C.byref(h)))
    return h


def kkt_factor(h, H_vals, J_vals, delta, gamma, n_h, n_j, stream=None):
    return _lib.kkt_factor(h, _dev(H_vals, n_h), _dev(J_vals, n_j), float(delta), float(gamma), _stream(stream))


def kkt_solve(h, r_x, r_y, dx, dy, n, m, stream=None):
    return _lib.kkt_solve(h, _dev(r_x, n), _dev(r_y, m), _dev(dx, n), _dev(dy, m), _stream(stream))


def kkt_solve_multi(h, nrhs, r_x, r_y, dx, dy, n, m, stream=None):
    """nrhs right-hand sides, RHS after RHS: r_x, dx CUDA float64 (nrhs*n),
    r_y, dy (nrhs*m). Returns (status, [kkt_info per RHS])."""
    infos = (kkt_info * max(int(nrhs), 1))()
    code = _lib.kkt_solve_multi(h, int(nrhs), _dev(r_x, nrhs * n), _dev(r_y, nrhs * m), _dev(dx, nrhs * n),
                                _dev(dy, nrhs * m), C.cast(infos, C.c_void_p), _stream(stream))
    return code, [infos[j] for j in range(int(nrhs))]


def kkt_hsolve(h, b, x, n, stream=None):
    return _lib.kkt_hsolve(h, _dev(b, n), _dev(x, n), _stream(stream))


def kkt_factor_solve_host(h, H_vals, J_vals, delta, gamma, r_x, r_y, dx, dy, stream=None):
    """All value/vector arguments are host numpy float64 arrays (dx, dy written)."""
    for a in (H_vals, J_vals, r_x, r_y, dx, dy):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError("expected contiguous float64 numpy arrays")
    ptr = lambda a: a.ctypes.data if a.size else None
    return _lib.kkt_factor_solve_host(h, ptr(H_vals), ptr(J_vals), float(delta), float(gamma), ptr(r_x),
                                      ptr(r_y), ptr(dx), ptr(dy), _stream(stream))


def kkt_get_info(h) -> kkt_info:
    i = kkt_info()
    _check("kkt_get_info", _lib.kkt_get_info(h, C.byref(i)))
    return i


def kkt_inertia(h) -> bool:
    v = C.c_int32()
    _check("kkt_inertia", _lib.kkt_inertia(h, C.byref(v)))
    return bool(v.value)


def kkt_symbolic_info_get(h) -> kkt_symbolic_info:
    s = kkt_symbolic_info()
    _check("kkt_symbolic_info_get", _lib.kkt_symbolic_info_get(h, C.byref(s)))
    return s


def kkt_get_symbolic(h):
    s = kkt_symbolic_info_get(h)
    n, ns = s.n, s.nsuper
    out = dict(amd=np.zeros(n, np.int32), perm=np.zeros(n, np.int32), parent=np.zeros(n, np.int32),
               colcount=np.zeros(n, np.int64), sn_start=np.zeros(ns + 1, np.int32),
               sn_rowptr=np.zeros(ns + 1, np.int64), sn_rows=np.zeros(max(1, s.sn_rows_total), np.int32),
               sn_parent=np.zeros(max(1, ns), np.int32))
    keys = ("amd", "perm", "parent", "colcount", "sn_start", "sn_rowptr", "sn_rows", "sn_parent")
    _check("kkt_get_symbolic", _lib.kkt_get_symbolic(h, *[out[k].ctypes.data for k in keys]))
    out["sn_rows"] = out["sn_rows"][: s.sn_rows_total]
    out["sn_parent"] = out["sn_parent"][:ns]
    return out


def kkt_get_factor_panels(h):
    s = kkt_symbolic_info_get(h)
    out = np.zeros(max(1, s.panel_entries))
    _check("kkt_get_factor_panels", _lib.kkt_get_factor_panels(h, out.ctypes.data))
    return out[: s.panel_entries]


def kkt_get_profile(h, reset=False):
    """{kernel kind: (ms, launches)} accumulated by a handle made with profile=1."""
    ms = np.zeros(12)
    n = np.zeros(12, np.int64)
    _check("kkt_get_profile", _lib.kkt_get_profile(h, ms.ctypes.data, n.ctypes.data, int(bool(reset))))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def kkt_residual_noalloc(n, m, H_colptr, H_rowidx, H_vals, J_rowptr, J_colidx, J_vals, delta, r_x, r_y, dx, dy,
                         res_x, res_y, norms, stream=None):
    """Residual of K_delta without device allocation (for callers that
    cannot allocate device memory). Every array argument is a CUDA tensor on
    the current device: int64/int32 patterns, float64 values; norms is
    float64[4] (RR, BE, ||res||, ||K||_inf). The J arrays, r_y, dy and res_y
    may be None when m == 0. Sizes are checked here (ValueError) because the
    kernels trust them; the pattern's contents (H_colptr[n] equal to the
    entry count, indices in range) are the caller's to guarantee. Returns the
    status code; the work is asynchronous."""
    import torch

    n, m = int(n), int(m)
    cur = torch.cuda.current_device()

    def ptr(name, t, dt, size):
        if t is None:
            if size > 0:
                raise ValueError(f"{name}: a tensor of {size} elements is required")
            return None
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name}: expected a contiguous CUDA tensor of {dt}")
        if t.device.index != cur:
            raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{cur}")
        if size >= 0 and t.numel() != size:
            raise ValueError(f"{name}: {t.numel()} elements, expected {size}")
        return t.data_ptr() if t.numel() else None
    i64, i32, f64 = torch.int64, torch.int32, torch.float64
    nh = -1 if H_rowidx is None else H_rowidx.numel()
    nj = (-1 if J_colidx is None else J_colidx.numel()) if m > 0 else 0
    if nj < 0:
        raise ValueError("J_colidx: required when m > 0")
    args = (ptr("H_colptr", H_colptr, i64, n + 1), ptr("H_rowidx", H_rowidx, i32, nh),
            ptr("H_vals", H_vals, f64, nh), ptr("J_rowptr", J_rowptr, i64, m + 1 if m > 0 else 0),
            ptr("J_colidx", J_colidx, i32, nj), ptr("J_vals", J_vals, f64, nj))
    return _lib.kkt_residual_noalloc(n, m, *args, float(delta),
                                     ptr("r_x", r_x, f64, n), ptr("r_y", r_y, f64, m), ptr("dx", dx, f64, n),
                                     ptr("dy", dy, f64, m), ptr("res_x", res_x, f64, n),
                                     ptr("res_y", res_y, f64, m), ptr("norms", norms, f64, 4), _stream(stream))


def kkt_get_solve_counters(h, reset=False):
    """Cycle counters of the persistent solve kernel (profile=1 handles)."""
    out = np.zeros(32, np.uint64)
    _check("kkt_get_solve_counters", _lib.kkt_get_solve_counters(h, out.ctypes.data, int(bool(reset))))
    keys = ("dispatch", "dep_wait", "copy_wait", "items", "barriers", "n_items", "cta_launches",
            "subtree_cycles", "n_subtree", "head_cycles", "n_head", "chunk_cycles", "n_chunk",
            "subtree_level_cycles", "n_subtree_levels", "zero15",
            "fhd_issue", "fhd_dep", "fhd_load", "fch_issue", "fch_dep", "fch_load", "fch_matvec", "fch_publish",
            "bhd_issue", "bhd_dep", "bhd_load", "bhd_chunk0", "bhd_inverse", "bhd_publish", "fhd_inverse", "fhd_chunk0")
    return {k: int(out[i]) for i, k in enumerate(keys)}


def kkt_get_solve_trace(h):
    """Item timeline of the first H^-1 application of the last solve launch
    (profile=1 handles): uint64 array [2 sweeps, nitems, (start ns, end ns, CTA)]."""
    ni = kkt_symbolic_info_get(h).nitems
    out = np.zeros((2, ni, 3), np.uint64)
    _check("kkt_get_solve_trace", _lib.kkt_get_solve_trace(h, out.ctypes.data, out.size))
    return out


def kkt_get_solve_item_order(h):
    """Dispatch orders of the forward and backward sweeps (int32 item codes)."""
    ni = kkt_symbolic_info_get(h).nitems
    f, b = np.zeros(ni, np.int32), np.zeros(ni, np.int32)
    _check("kkt_get_solve_item_order", _lib.kkt_get_solve_item_order(h, f.ctypes.data, b.ctypes.data, ni))
    return f, b


def kkt_destroy(h):
    return _lib.kkt_destroy(h)


def kkt_analyse_4x4(n_x, m_c, m_d, H_colptr, H_rowidx, J_rowptr, J_colidx, Jd_rowptr, Jd_colidx,
                    opt: kkt_options | None = None, host=False):
    keep = [_np(H_colptr, np.int64), _np(H_rowidx, np.int32), _np(J_rowptr, np.int64), _np(J_colidx, np.int32),
            _np(Jd_rowptr, np.int64), _np(Jd_colidx, np.int32)]
    h = C.c_void_p()
    fn = "kkt_analyse_4x4_host" if host else "kkt_analyse_4x4"
    _check(fn, getattr(_lib, fn)(int(n_x), int(m_c), int(m_d), *[k[1] for k in keep],
                                 C.byref(opt) if opt is not None else None, C.byref(h)))
    return h


def kkt_4x4_inner(h4):
    return C.c_void_p(_lib.kkt_4x4_inner(h4))


def kkt_get_4x4_pattern(h4, n_x):
    nnz = C.c_int64()
    _check("kkt_get_4x4_pattern", _lib.kkt_get_4x4_pattern(h4, C.byref(nnz), None, None))
    ptr = np.zeros(n_x + 1, np.int64)
    row = np.zeros(max(1, nnz.value), np.int32)
    _check("kkt_get_4x4_pattern", _lib.kkt_get_4x4_pattern(h4, None, ptr.ctypes.data, row.ctypes.data))
    return ptr, row[: nnz.value]


def kkt_factor_4x4(h4, H_vals, D_x, Jd_vals, D_s, J_vals, delta, gamma, sizes, stream=None):
    nh, nx, njd, md, nj = sizes
    return _lib.kkt_factor_4x4(h4, _dev(H_vals, nh), _dev(D_x, nx), _dev(Jd_vals, njd), _dev(D_s, md),
                               _dev(J_vals, nj), float(delta), float(gamma), _stream(stream))


def kkt_solve_4x4(h4, r_xt, r_s, r_y, r_yd, dx, ds, dy, dyd, sizes, stream=None):
    nx, mc, md = sizes
    return _lib.kkt_solve_4x4(h4, _dev(r_xt, nx), _dev(r_s, md), _dev(r_y, mc), _dev(r_yd, md), _dev(dx, nx),
                              _dev(ds, md), _dev(dy, mc), _dev(dyd, md), _stream(stream))


def kkt_destroy_4x4(h4):
    return _lib.kkt_destroy_4x4(h4)


def kkt_status_string(code) -> str:
    return _lib.kkt_status_string(int(code)).decode()


class KKTSolver:
    """One analysed pattern: factor values, solve right-hand sides.

    >>> s = KKTSolver(sys.n, sys.m, sys.H_colptr, sys.H_rowidx, sys.J_rowptr, sys.J_colidx)
    >>> s.factor(H_vals_cuda, J_vals_cuda, delta, gamma); dx, dy = s.solve(r_x_cuda, r_y_cuda)
    """

    def __init__(self, n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, **options):
        self.n, self.m = int(n), int(m)
        self.nnz_h = int(np.asarray(H_colptr)[-1])
        self.nnz_j = int(np.asarray(J_rowptr)[-1]) if m else 0
        self.opt = kkt_default_options(**options)
        self.h = kkt_analyse(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, self.opt)

    @classmethod
    def host_only(cls, n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, **options):
        """The ordering, symbolic analysis and plan without device memory
        (kkt_analyse_host): a source for like()."""
        self = cls.__new__(cls)
        self.n, self.m = int(n), int(m)
        self.nnz_h = int(np.asarray(H_colptr)[-1])
        self.nnz_j = int(np.asarray(J_rowptr)[-1]) if m else 0
        self.opt = kkt_default_options(**options)
        self.h = kkt_analyse_host(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, self.opt)
        return self

    @classmethod
    def like(cls, other: "KKTSolver", **options):
        """A solver for other's pattern with other options (e.g. the other
        precision), reusing its ordering and symbolic analysis."""
        self = cls.__new__(cls)
        self.n, self.m, self.nnz_h, self.nnz_j = other.n, other.m, other.nnz_h, other.nnz_j
        self.opt = kkt_default_options(**options)
        h = C.c_void_p()
        _check("kkt_analyse_like", _lib.kkt_analyse_like(other.h, C.byref(self.opt), C.byref(h)))
        self.h = h
        return self

    def scaling(self):
        """The Ruiz scaling D (numpy float64[n + m]) of the last factorization."""
        D = np.zeros(self.n + self.m)
        _check("kkt_get_scaling", _lib.kkt_get_scaling(self.h, D.ctypes.data))
        return D

    def set_profile(self, on=True):
        """Per-kernel timing on (kernel by kernel, events) or off (graph)."""
        _check("kkt_set_profile", _lib.kkt_set_profile(self.h, int(bool(on))))

    def factor(self, H_vals, J_vals, delta, gamma=-1.0, stream=None, check=True):
        code = kkt_factor(self.h, H_vals, J_vals, delta, gamma, self.nnz_h, self.nnz_j, stream)
        if check:
            _check("kkt_factor", code)
        return code

    def solve(self, r_x, r_y, dx=None, dy=None, stream=None, check=True):
        import torch
        if dx is None:
            dx = torch.empty(self.n, dtype=torch.float64, device=r_x.device)
        if dy is None:
            dy = torch.empty(self.m, dtype=torch.float64, device=r_x.device)
        code = kkt_solve(self.h, r_x, r_y, dx, dy, self.n, self.m, stream)
        if check:
            _check("kkt_solve", code)
        return dx, dy

    def solve_multi(self, r_x, r_y, stream=None, check=True):
        """r_x: CUDA float64 (nrhs, n), r_y: (nrhs, m), contiguous; returns
        (dx, dy) of the same shapes and the per-RHS kkt_info list."""
        import torch
        k = int(r_x.shape[0])
        dx = torch.empty_like(r_x)
        dy = torch.empty((k, self.m), dtype=torch.float64, device=r_x.device)
        code, infos = kkt_solve_multi(self.h, k, r_x.reshape(-1), r_y.reshape(-1), dx.view(-1), dy.view(-1),
                                      self.n, self.m, stream)
        if check:
            _check("kkt_solve_multi", code)
        return dx, dy, infos

    def factor_regularized(self, H_vals, J_vals, gamma=-1.0, delta_min=1e-9, delta_max=1e-6, stream=None,
                           check=True):
        """Algorithm 1's delta_1 loop with the sequence rule of Sec. 4.1 (the
        first retry goes back to the delta_1 the handle accepted for the
        previous matrix); returns (status code, delta_1 used)."""
        d = C.c_double(0.0)
        code = _lib.kkt_factor_regularized(self.h, _dev(H_vals, self.nnz_h), _dev(J_vals, self.nnz_j), float(gamma),
                                           float(delta_min), float(delta_max), C.byref(d), _stream(stream))
        if check and code not in (0, 2):
            _check("kkt_factor_regularized", code)
        return code, d.value

    def set_delta_prev(self, delta_prev=0.0):
        """The delta_1 the next factor_regularized call goes back to after a
        failed unshifted trial (0 starts a new sequence)."""
        _check("kkt_set_delta_prev", _lib.kkt_set_delta_prev(self.h, float(delta_prev)))

    def factor_batch(self, H_vals, J_vals, delta, gamma=-1.0, stream=None):
        """H_vals: CUDA float64 (nsys, nnz(H~)), J_vals: (nsys, nnz(J)). Returns
        (status code, per-system status array)."""
        k = int(H_vals.shape[0])
        st = np.zeros(k, np.int32)
        code = _lib.kkt_factor_batch(self.h, k, _dev(H_vals.reshape(-1), k * self.nnz_h),
                                     _dev(J_vals.reshape(-1), k * self.nnz_j), float(delta), float(gamma),
                                     st.ctypes.data, _stream(stream))
        return code, st

    def solve_batch(self, r_x, r_y, stream=None):
        """r_x: CUDA float64 (nsys, n), r_y: (nsys, m). Returns (dx, dy, infos,
        per-system status, code)."""
        import torch
        k = int(r_x.shape[0])
        dx = torch.empty_like(r_x)
        dy = torch.empty((k, self.m), dtype=torch.float64, device=r_x.device)
        infos = (kkt_info * k)()
        st = np.zeros(k, np.int32)
        code = _lib.kkt_solve_batch(self.h, k, _dev(r_x.reshape(-1), k * self.n), _dev(r_y.reshape(-1), k * self.m),
                                    _dev(dx.view(-1), k * self.n), _dev(dy.view(-1), k * self.m),
                                    C.cast(infos, C.c_void_p), st.ctypes.data, _stream(stream))
        return dx, dy, [infos[j] for j in range(k)], st, code

    def hsolve(self, b, stream=None):
        import torch
        x = torch.empty_like(b)
        _check("kkt_hsolve", kkt_hsolve(self.h, b, x, self.n, stream))
        return x

    def factor_solve_host(self, H_vals, J_vals, delta, gamma, r_x, r_y, dx=None, dy=None, stream=None):
        dx = np.zeros(self.n) if dx is None else dx
        dy = np.zeros(self.m) if dy is None else dy
        _check("kkt_factor_solve_host", kkt_factor_solve_host(self.h, H_vals, J_vals, delta, gamma, r_x, r_y,
                                                               dx, dy, stream))
        return dx, dy

    @property
    def info(self):
        return kkt_get_info(self.h)

    @property
    def inertia_ok(self):
        return kkt_inertia(self.h)

    @property
    def symbolic_info(self):
        return kkt_symbolic_info_get(self.h)

    def symbolic(self):
        return kkt_get_symbolic(self.h)

    def panels(self):
        return kkt_get_factor_panels(self.h)

    def profile(self, reset=False):
        return kkt_get_profile(self.h, reset)

    def solve_counters(self, reset=False):
        return kkt_get_solve_counters(self.h, reset)

    def solve_trace(self):
        return kkt_get_solve_trace(self.h)

    def solve_item_order(self):
        return kkt_get_solve_item_order(self.h)

    def close(self):
        if getattr(self, "h", None):
            kkt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKTSolver4x4:
    """The 4x4 form (Sec. 3, eq. linsys4x4): H, D_x, D_s, J, J_d values per
    factorization; (r~_x, r_s, r_y, r_yd) -> (dx, ds, dy, dy_d) per solve.
    Reduction to the 2x2 form, the solve, and the recovery of ds and dy_d all
    run on the device."""

    def __init__(self, n_x, m_c, m_d, H_colptr, H_rowidx, J_rowptr, J_colidx, Jd_rowptr, Jd_colidx, **options):
        self.n, self.m, self.md = int(n_x), int(m_c), int(m_d)
        self.nnz_h = int(np.asarray(H_colptr)[-1])
        self.nnz_j = int(np.asarray(J_rowptr)[-1]) if m_c else 0
        self.nnz_jd = int(np.asarray(Jd_rowptr)[-1]) if m_d else 0
        self.opt = kkt_default_options(**options)
        self.h = kkt_analyse_4x4(n_x, m_c, m_d, H_colptr, H_rowidx, J_rowptr, J_colidx, Jd_rowptr, Jd_colidx,
                                 self.opt)

    def factor(self, H_vals, D_x, Jd_vals, D_s, J_vals, delta, gamma=-1.0, stream=None, check=True):
        code = kkt_factor_4x4(self.h, H_vals, D_x, Jd_vals, D_s, J_vals, delta, gamma,
                              (self.nnz_h, self.n, self.nnz_jd, self.md, self.nnz_j), stream)
        if check:
            _check("kkt_factor_4x4", code)
        return code

    def solve(self, r_xt, r_s, r_y, r_yd, stream=None, check=True):
        import torch
        f = lambda k: torch.empty(k, dtype=torch.float64, device=r_xt.device)
        dx, ds, dy, dyd = f(self.n), f(self.md), f(self.m), f(self.md)
        code = kkt_solve_4x4(self.h, r_xt, r_s, r_y, r_yd, dx, ds, dy, dyd, (self.n, self.m, self.md), stream)
        if check:
            _check("kkt_solve_4x4", code)
        return dx, ds, dy, dyd

    @property
    def inner(self):
        return kkt_4x4_inner(self.h)

    @property
    def info(self):
        return kkt_get_info(self.inner)

    @property
    def inertia_ok(self):
        return kkt_inertia(self.inner)

    def pattern(self):
        return kkt_get_4x4_pattern(self.h, self.n)

    def close(self):
        if getattr(self, "h", None):
            kkt_destroy_4x4(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKTServer:
    """Continuous-batching request server over resident patterns (the
    library's kkt_server_*): add patterns, submit value refactorizations +
    solves with device tensors, wait for their records.

    >>> srv = KKTServer(budget_bytes=0, max_inflight=4, precision="mixed", ordering="nd")
    >>> pid = srv.add_pattern(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx)
    >>> rid = srv.submit(pid, H_vals, J_vals, delta, gamma, r_x, r_y, dx, dy)
    >>> info = srv.wait(rid)
    """

    def __init__(self, budget_bytes=0, max_inflight=4, **options):
        self.opt = kkt_default_options(**options)
        h = C.c_void_p()
        _check("kkt_server_create", _lib.kkt_server_create(int(budget_bytes), int(max_inflight), C.byref(self.opt),
                                                           C.byref(h)))
        self.h = h
        self._sizes = []
        self._keep = {}

    def add_pattern(self, n, m, H_colptr, H_rowidx, J_rowptr, J_colidx):
        keep = [_np(H_colptr, np.int64), _np(H_rowidx, np.int32), _np(J_rowptr, np.int64), _np(J_colidx, np.int32)]
        pid = C.c_int32(0)
        _check("kkt_server_add_pattern", _lib.kkt_server_add_pattern(self.h, int(n), int(m), keep[0][1], keep[1][1],
                                                                     keep[2][1], keep[3][1], C.byref(pid)))
        self._sizes.append((int(n), int(m), int(np.asarray(H_colptr)[-1]), int(np.asarray(J_rowptr)[-1]) if m else 0))
        return pid.value

    def submit(self, pattern, H_vals, J_vals, delta, gamma, r_x, r_y, dx, dy):
        """All tensors on the device; they must stay alive and unchanged until
        wait() returns for this request (the server keeps references)."""
        n, m, nh, nj = self._sizes[pattern]
        rid = C.c_int64(0)
        _check("kkt_server_submit", _lib.kkt_server_submit(
            self.h, int(pattern), _dev(H_vals, nh), _dev(J_vals, nj), float(delta), float(gamma), _dev(r_x, n),
            _dev(r_y, m), _dev(dx, n), _dev(dy, m), C.byref(rid)))
        self._keep[rid.value] = (H_vals, J_vals, r_x, r_y, dx, dy)
        return rid.value

    def wait(self, rid):
        info = kkt_request_info()
        _check("kkt_server_wait", _lib.kkt_server_wait(self.h, int(rid), C.byref(info)))
        self._keep.pop(rid, None)
        return info

    def stats(self):
        st = kkt_server_stats()
        _check("kkt_server_get_stats", _lib.kkt_server_get_stats(self.h, C.byref(st)))
        return st

    def close(self):
        if getattr(self, "h", None):
            _lib.kkt_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
