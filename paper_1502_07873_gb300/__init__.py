"""Python binding of liboed (include/oed.h): the GB300 (sm_103a) CUDA path of the
Laplace-approximated expected information gain for seismic source inversion
(Long, Motamed & Tempone, arXiv:1502.07873).

This module only marshals arguments: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  The
functions carry the C names (``oed_forward``, ``oed_hessian``, ``oed_eig``,
``oed_eig_designs``, ``oed_nodes_mc``, ``oed_nodes_smolyak``, ``oed_eig_host``);
``Context`` owns an ``oed_ctx``.  If the shared library has not been built the
import of any entry point raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboed.so")

OED_OK, OED_EINVAL, OED_ENOMEM, OED_ENOTPD, OED_ECUDA, OED_ETIMEOUT, OED_PENDING, OED_ECANCELED = range(8)
OED_SERVER_NO_AUTOTUNE = 1
OED_FP32, OED_FP64 = 0, 1
OED_JAC_PAIRS, OED_JAC_DIFFERENCE, OED_JAC_SENSITIVITY = 0, 1, 2
OED_STF_GAUSS, OED_STF_RICKER = 0, 1
NTHETA = 7

SYMBOLS = ("oed_create", "oed_workspace_bytes", "oed_destroy", "oed_last_error",
           "oed_status_string", "oed_chunk_nodes", "oed_forward", "oed_hessian", "oed_eig",
           "oed_eig_designs", "oed_nodes_mc", "oed_nodes_smolyak", "oed_eig_host",
           "oed_last_step_time", "oed_autotune", "oed_get_tuning", "oed_set_tuning",
           "oed_resident_min_cluster", "oed_set_jacobian", "oed_get_jacobian",
           "oed_gauss_newton_noalloc", "oed_server_create", "oed_server_request_bytes",
           "oed_server_submit", "oed_server_poll", "oed_server_wait", "oed_server_stats",
           "oed_server_destroy", "oed_eig_subset", "oed_dlmc", "oed_hessian_ii", "oed_newton_step",
           "oed_hessian_map", "oed_wait_selftest", "oed_rebind", "oed_server_set_admission",
           "oed_server_set_log", "oed_server_cancel", "oed_server_checkpoint", "oed_server_metrics",
           "oed_server_pool", "oed_server_release")


class OedError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("nsteps", ctypes.c_int), ("nlayers", ctypes.c_int),
                ("z_top", ctypes.POINTER(ctypes.c_double)), ("vp", ctypes.POINTER(ctypes.c_double)),
                ("vs", ctypes.POINTER(ctypes.c_double)), ("rho", ctypes.POINTER(ctypes.c_double)),
                ("nrec", ctypes.c_int), ("rec_ix", ctypes.POINTER(ctypes.c_int)),
                ("precision", ctypes.c_int), ("stf", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("problem", Problem), ("n", ctypes.c_int), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double)), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double)), ("rel_step", ctypes.c_double),
                ("sigma", ctypes.c_double), ("jacobian", ctypes.c_int), ("n_done", ctypes.c_int),
                ("H_done", ctypes.POINTER(ctypes.c_double)), ("tag", ctypes.c_ulonglong)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("eig", ctypes.c_double), ("n_bad", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("footprint_bytes", ctypes.c_size_t),
                ("nodes_done", ctypes.c_int), ("workspace_reused", ctypes.c_int)]


_lib = None


def library():
    """Load liboed.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "oed_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(Problem), i]),
        "oed_workspace_bytes": (sz, [ctypes.POINTER(Problem), i]),
        "oed_destroy": (i, [vp]),
        "oed_last_error": (ctypes.c_char_p, [vp]),
        "oed_status_string": (ctypes.c_char_p, [i]),
        "oed_chunk_nodes": (i, [vp]),
        "oed_forward": (i, [vp, vp, i, vp, vp]),
        "oed_hessian": (i, [vp, vp, i, dp, dp, d, d, ip, i, vp, vp, vp, vp]),
        "oed_eig": (i, [vp, vp, i, vp, dp, dp, vp, vp, vp, vp, vp]),
        "oed_eig_designs": (i, [vp, vp, i, i, i, i, vp, i, vp, dp, dp, vp, vp, vp]),
        "oed_eig_subset": (i, [vp, vp, i, vp, dp, dp, i, vp, vp, vp, vp, vp]),
        "oed_dlmc": (i, [vp, vp, i, vp, i, i, d, vp, vp, vp]),
        "oed_hessian_ii": (i, [vp, vp, i, vp, d, vp, vp, vp, vp]),
        "oed_newton_step": (i, [vp, vp, i, dp, dp, i, vp, vp, vp]),
        "oed_hessian_map": (i, [vp, vp, i, vp, dp, dp, d, d, i, i, vp, vp, vp, vp]),
        "oed_nodes_mc": (i, [vp, i, dp, dp, vp, vp, vp]),
        "oed_nodes_smolyak": (i, [i, i, dp, dp, i, dp, dp, ip]),
        "oed_eig_host": (i, [vp, dp, dp, i, dp, dp, d, d, dp, dp, ip]),
        "oed_last_step_time": (i, [vp, ctypes.POINTER(ctypes.c_float), ip]),
        "oed_autotune": (i, [vp, i, vp]),
        "oed_get_tuning": (i, [vp, ip, ip, ip]),
        "oed_set_tuning": (i, [vp, i, i, i]),
        "oed_resident_min_cluster": (i, [vp]),
        "oed_set_jacobian": (i, [vp, i]),
        "oed_wait_selftest": (i, [vp, d, vp]),
        "oed_get_jacobian": (i, [vp]),
        "oed_gauss_newton_noalloc": (i, [vp, i, i, i, i, dp, dp, d, d, vp, vp]),
        "oed_server_create": (i, [ctypes.POINTER(vp), sz, i, i, i]),
        "oed_server_request_bytes": (sz, [ctypes.POINTER(Request), i]),
        "oed_server_submit": (i, [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_ulonglong)]),
        "oed_server_poll": (i, [vp, ctypes.c_ulonglong, ctypes.POINTER(Result)]),
        "oed_server_wait": (i, [vp, ctypes.c_ulonglong, d, ctypes.POINTER(Result)]),
        "oed_server_stats": (i, [vp, ctypes.POINTER(sz), ip, ip]),
        "oed_server_destroy": (i, [vp]),
        "oed_rebind": (i, [vp, ctypes.POINTER(Problem)]),
        "oed_server_set_admission": (i, [vp, d]),
        "oed_server_set_log": (i, [vp, ctypes.c_char_p]),
        "oed_server_cancel": (i, [vp, ctypes.c_ulonglong]),
        "oed_server_checkpoint": (i, [vp, ctypes.c_ulonglong, dp, i, ip]),
        "oed_server_metrics": (i, [vp, ctypes.c_ulonglong, ctypes.c_char_p, sz]),
        "oed_server_pool": (i, [vp, ip, ctypes.POINTER(sz)]),
        "oed_server_release": (i, [vp, ctypes.c_ulonglong]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _status_name(code: int) -> str:
    names = {0: "OED_OK", 1: "OED_EINVAL", 2: "OED_ENOMEM", 3: "OED_ENOTPD", 4: "OED_ECUDA",
             5: "OED_ETIMEOUT", 6: "OED_PENDING", 7: "OED_ECANCELED"}
    return names.get(code, f"status {code}")


def _darr(vals):
    a = (ctypes.c_double * len(vals))(*[float(v) for v in vals])
    return a


def _ptr(t) -> Optional[int]:
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _arg(t, name: str, dtype: str, numel: int = 0, rows: Optional[int] = None):
    """Device pointer of a tensor argument, after checking what the C call will read or
    write through it (a wrong dtype or a short tensor would be accessed past its end on
    the device): its dtype ("f64", "i32" or "u8"), at least `numel` elements, `rows` rows
    of 7 when given (a parameter array), then that it is a contiguous CUDA tensor."""
    if t is None:
        return None
    import torch
    want = {"f64": torch.float64, "i32": torch.int32, "u8": torch.uint8}[dtype]
    if t.dtype != want:
        raise ValueError(f"{name}: expected {want}, got {t.dtype}")
    if rows is not None and (t.dim() != 2 or t.shape[0] != rows or t.shape[1] != NTHETA):
        raise ValueError(f"{name}: expected shape [{rows}][7], got {list(t.shape)}")
    if t.numel() < numel:
        raise ValueError(f"{name}: needs at least {numel} elements, has {t.numel()}")
    return _ptr(t)


def _theta(theta, name: str = "theta"):
    """Node count of a parameter array theta[n][7] (FP64), checked."""
    if theta.dim() != 2 or theta.shape[1] != NTHETA:
        raise ValueError(f"{name}: expected shape [n][7], got {list(theta.shape)}")
    return int(theta.shape[0])


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check(ctx_handle, rc: int, what: str):
    if rc != OED_OK:
        msg = library().oed_last_error(ctx_handle) if ctx_handle else b""
        raise OedError(rc, f"{what}: {msg.decode() if msg else ''}")


def make_problem(nx, nz, h, dt, nsteps, layers, rec_ix, precision=OED_FP32, stf=None):
    """Build an oed_problem (keeps the host arrays alive on the returned object);
    stf: OED_STF_GAUSS (default) or OED_STF_RICKER."""
    p = Problem()
    p.nx, p.nz, p.h, p.dt, p.nsteps = int(nx), int(nz), float(h), float(dt), int(nsteps)
    p.nlayers = len(layers)
    p._z = _darr([l[0] for l in layers])
    p._vp = _darr([l[1] for l in layers])
    p._vs = _darr([l[2] for l in layers])
    p._rho = _darr([l[3] for l in layers])
    p.z_top, p.vp, p.vs, p.rho = p._z, p._vp, p._vs, p._rho
    p.nrec = len(rec_ix)
    p._rec = (ctypes.c_int * len(rec_ix))(*[int(r) for r in rec_ix])
    p.rec_ix = p._rec
    p.precision = int(precision)
    p.stf = OED_STF_GAUSS if stf is None else int(stf)
    return p


def problem_from_workload(w, precision=OED_FP32, rec_ix=None, nsteps=None, stf=None):
    return make_problem(w.nx, w.nz, w.h, w.dt, w.nsteps if nsteps is None else nsteps, w.layers,
                        w.rec_ix if rec_ix is None else rec_ix, precision, stf)


def oed_workspace_bytes(problem: Problem, max_solves: int) -> int:
    return int(library().oed_workspace_bytes(ctypes.byref(problem), int(max_solves)))


class Context:
    """An oed_ctx: device workspace for up to ``max_solves`` concurrent solves."""

    def __init__(self, problem: Problem, max_solves: int):
        L = library()
        self.problem = problem
        self.handle = ctypes.c_void_p()
        rc = L.oed_create(ctypes.byref(self.handle), ctypes.byref(problem), int(max_solves))
        if rc != OED_OK:
            raise OedError(rc, "oed_create failed")
        self.max_solves = int(max_solves)
        self.nrec = problem.nrec
        self.nlev = problem.nsteps + 1

    def close(self):
        if self.handle:
            library().oed_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def rebind(self, problem: Problem):
        """Re-target this context's workspace at another problem of the same grid shape and
        precision (oed_rebind).  The streams of earlier calls on this context must be
        synchronised first (the new problem's tables are written on the context's own stream)."""
        _check(self.handle, library().oed_rebind(self.handle, ctypes.byref(problem)), "oed_rebind")
        self.problem = problem
        self.nrec = problem.nrec
        self.nlev = problem.nsteps + 1

    def last_step_time(self):
        """(milliseconds, launches) of the stencil launches of the last time loop."""
        ms = ctypes.c_float()
        n = ctypes.c_int()
        _check(self.handle, library().oed_last_step_time(self.handle, ctypes.byref(ms), ctypes.byref(n)),
               "oed_last_step_time")
        return float(ms.value), int(n.value)

    def autotune(self, nsolve: Optional[int] = None, stream=None):
        """Pick the fastest stencil launch shape for nsolve solves (default: a full chunk)."""
        n = nsolve or 15 * self.chunk_nodes
        _check(self.handle, library().oed_autotune(self.handle, int(n), _stream(stream)), "oed_autotune")
        return self.tuning

    @property
    def tuning(self):
        """(cluster_size, rows_per_thread, warps_per_block); cluster_size 0 = streaming kernel."""
        c, zs, wz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        library().oed_get_tuning(self.handle, ctypes.byref(c), ctypes.byref(zs), ctypes.byref(wz))
        return int(c.value), int(zs.value), int(wz.value)

    def set_tuning(self, cluster_size: int = 0, rows_per_thread: int = 4, warps_per_block: int = 4):
        _check(self.handle, library().oed_set_tuning(self.handle, int(cluster_size), int(rows_per_thread),
                                                      int(warps_per_block)), "oed_set_tuning")

    @property
    def jacobian(self) -> int:
        return int(library().oed_get_jacobian(self.handle))

    @jacobian.setter
    def jacobian(self, mode: int):
        _check(self.handle, library().oed_set_jacobian(self.handle, int(mode)), "oed_set_jacobian")

    @property
    def resident_min_cluster(self) -> int:
        return int(library().oed_resident_min_cluster(self.handle))

    @property
    def chunk_nodes(self) -> int:
        return int(library().oed_chunk_nodes(self.handle))


def oed_forward(ctx: Context, theta, g, stream=None):
    """Seismograms g[n][nsteps+1][nrec][2] (FP64, device) of theta[n][7] (FP64, device)."""
    n = _theta(theta)
    _check(ctx.handle, library().oed_forward(ctx.handle, _arg(theta, "theta", "f64", rows=n), n,
                                             _arg(g, "g", "f64", n * ctx.nlev * ctx.nrec * 2), _stream(stream)),
           "oed_forward")
    return g


def oed_hessian(ctx: Context, theta, lo: Sequence[float], hi: Sequence[float], rel_step: float,
                sigma: float, H, win_levels: Optional[Sequence[int]] = None, H_rec=None,
                status=None, stream=None):
    """Gauss-Newton Hessians H[n][7][7] (device) from central-FD solves."""
    n = _theta(theta)
    nwin = 0 if win_levels is None else len(win_levels)
    wl = (ctypes.c_int * max(1, nwin))(*(win_levels or [0]))
    rc = library().oed_hessian(ctx.handle, _arg(theta, "theta", "f64", rows=n), n, _darr(lo), _darr(hi),
                               float(rel_step), float(sigma), wl if nwin else None, nwin,
                               _arg(H, "H", "f64", n * 49), _arg(H_rec, "H_rec", "f64", n * ctx.nrec * nwin * 28),
                               _arg(status, "status", "i32", n), _stream(stream))
    _check(ctx.handle, rc, "oed_hessian")
    return H


def oed_eig(ctx: Optional[Context], H, w, lo, hi, eig, dkl=None, status=None, n_bad=None,
            stream=None):
    """EIG = sum_i w_i D_KL-hat(H_i) into eig[1] (device)."""
    n = H.shape[0]
    h = ctx.handle if ctx is not None else None
    rc = library().oed_eig(h, _arg(H, "H", "f64", n * 49), n, _arg(w, "w", "f64", n), _darr(lo), _darr(hi),
                           _arg(eig, "eig", "f64", 1), _arg(dkl, "dkl", "f64", n), _arg(status, "status", "i32", n),
                           _arg(n_bad, "n_bad", "i32", 1), _stream(stream))
    _check(h, rc, "oed_eig")
    return eig


def oed_eig_subset(ctx: Optional[Context], H, w, lo, hi, free, eig, dkl=None, status=None,
                   n_bad=None, stream=None):
    """EIG of the problem whose unknown parameters are the indices in `free` (the others
    known): D_KL-hat from the sub-block of H_1, into eig[1] (device)."""
    mask = 0
    for j in free:
        mask |= 1 << int(j)
    n = H.shape[0]
    h = ctx.handle if ctx is not None else None
    rc = library().oed_eig_subset(h, _arg(H, "H", "f64", n * 49), n, _arg(w, "w", "f64", n), _darr(lo),
                                  _darr(hi), mask, _arg(eig, "eig", "f64", 1), _arg(dkl, "dkl", "f64", n),
                                  _arg(status, "status", "i32", n), _arg(n_bad, "n_bad", "i32", 1),
                                  _stream(stream))
    _check(h, rc, "oed_eig_subset")
    return eig


def oed_wait_selftest(ctx: Context, seconds: float = 0.05, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status code (OED_ETIMEOUT expected)."""
    return int(library().oed_wait_selftest(ctx.handle, float(seconds), _stream(stream)))


def oed_hessian_ii(ctx: Context, theta, y, sigma: float, H, grad=None, status=None, stream=None):
    """Adds H_II (Alg. 1 steps 6-10) at theta for data y to H; dL/dtheta into grad."""
    n = _theta(theta)
    _check(ctx.handle, library().oed_hessian_ii(ctx.handle, _arg(theta, "theta", "f64", rows=n), n,
                                                _arg(y, "y", "f64", n * ctx.nlev * ctx.nrec * 2), float(sigma),
                                                _arg(H, "H", "f64", n * 49), _arg(grad, "grad", "f64", n * 7),
                                                _arg(status, "status", "i32", n), _stream(stream)), "oed_hessian_ii")
    return H


def _mask(free):
    m = 0
    for j in free:
        m |= 1 << int(j)
    return m


def oed_newton_step(H, grad, theta, lo, hi, free=range(7), status=None, stream=None):
    """theta_F += -H_FF^-1 grad_F per node over the unknowns F, clamped to [lo, hi]."""
    n = _theta(theta)
    _check(None, library().oed_newton_step(_arg(H, "H", "f64", n * 49), _arg(grad, "grad", "f64", n * 7), n,
                                           _darr(lo), _darr(hi), _mask(free), _arg(theta, "theta", "f64", rows=n),
                                           _arg(status, "status", "i32", n), _stream(stream)), "oed_newton_step")
    return theta


def oed_hessian_map(ctx: Context, theta, y, lo, hi, rel_step: float, sigma: float, iters: int, H, grad,
                    free=range(7), status=None, stream=None):
    """Newton iterations over the unknowns F to the estimate of Thm 1; H = H_1 + H_II and
    grad at it."""
    n = _theta(theta)
    _check(ctx.handle, library().oed_hessian_map(ctx.handle, _arg(theta, "theta", "f64", rows=n), n,
                                                 _arg(y, "y", "f64", n * ctx.nlev * ctx.nrec * 2), _darr(lo),
                                                 _darr(hi), float(rel_step), float(sigma), _mask(free), int(iters),
                                                 _arg(H, "H", "f64", n * 49), _arg(grad, "grad", "f64", n * 7),
                                                 _arg(status, "status", "i32", n), _stream(stream)),
           "oed_hessian_map")
    return H


def oed_dlmc(g_outer, eps, g_inner, sigma, log_ev, eig=None, stream=None):
    """Double-loop Monte Carlo EIG: y_n = g_outer[n] + eps[n] against the inner samples
    g_inner (all device FP64, [N][D] / [M][D]); log_ev[N] and eig[1] (device)."""
    N = g_outer.shape[0]
    M = g_inner.shape[0]
    D = g_outer[0].numel()
    if g_inner[0].numel() != D or eps.shape[0] != N:
        raise ValueError("oed_dlmc: shapes")
    _check(None, library().oed_dlmc(_arg(g_outer, "g_outer", "f64", N * D), _arg(eps, "eps", "f64", N * D), N,
                                    _arg(g_inner, "g_inner", "f64", M * D), M, D, float(sigma),
                                    _arg(log_ev, "log_ev", "f64", N), _arg(eig, "eig", "f64", 1), _stream(stream)),
           "oed_dlmc")
    return eig


def oed_eig_designs(ctx: Optional[Context], H_rec, win: int, mask, w, lo, hi, eig, n_bad=None,
                    stream=None):
    """EIG of every receiver design in mask[ndesign][nrec] from H_rec[n][nrec][nwin][28]."""
    n, nrec, nwin = H_rec.shape[0], H_rec.shape[1], H_rec.shape[2]
    h = ctx.handle if ctx is not None else None
    nd = mask.shape[0]
    if mask.dim() != 2 or mask.shape[1] != nrec:
        raise ValueError(f"mask: expected shape [ndesign][{nrec}], got {list(mask.shape)}")
    rc = library().oed_eig_designs(h, _arg(H_rec, "H_rec", "f64", n * nrec * nwin * 28), n, nrec, nwin, int(win),
                                   _arg(mask, "mask", "u8", nd * nrec), nd, _arg(w, "w", "f64", n), _darr(lo),
                                   _darr(hi), _arg(eig, "eig", "f64", nd), _arg(n_bad, "n_bad", "i32", nd),
                                   _stream(stream))
    _check(h, rc, "oed_eig_designs")
    return eig


def oed_nodes_mc(u, lo, hi, theta, w, stream=None):
    M = _theta(u, "u")
    rc = library().oed_nodes_mc(_arg(u, "u", "f64", rows=M), M, _darr(lo), _darr(hi),
                                _arg(theta, "theta", "f64", rows=M), _arg(w, "w", "f64", M), _stream(stream))
    _check(None, rc, "oed_nodes_mc")
    return theta, w


def oed_nodes_smolyak(dim: int, level: int, lo=None, hi=None):
    """Host call: (nodes [count][dim], weights [count]) as numpy arrays."""
    import numpy as np
    L = library()
    cnt = ctypes.c_int()
    lo_a = _darr(lo) if lo is not None else None
    hi_a = _darr(hi) if hi is not None else None
    rc = L.oed_nodes_smolyak(dim, level, lo_a, hi_a, 0, None, None, ctypes.byref(cnt))
    _check(None, rc, "oed_nodes_smolyak")
    x = np.zeros((cnt.value, dim))
    w = np.zeros(cnt.value)
    rc = L.oed_nodes_smolyak(dim, level, lo_a, hi_a, cnt.value,
                             x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt))
    _check(None, rc, "oed_nodes_smolyak")
    return x, w


def oed_eig_host(ctx: Context, theta, w, lo, hi, rel_step: float, sigma: float, want_dkl=False):
    """Whole path with host arrays (numpy or pinned CPU tensors): returns (eig, dkl, n_bad)."""
    import numpy as np

    def hp(a):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("expected a contiguous CPU tensor")
            return ctypes.cast(a.data_ptr(), ctypes.POINTER(ctypes.c_double))
        return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    th_keep = theta if hasattr(theta, "data_ptr") else np.ascontiguousarray(theta, dtype=np.float64)
    w_keep = w if hasattr(w, "data_ptr") else np.ascontiguousarray(w, dtype=np.float64)
    n = th_keep.shape[0]
    eig = ctypes.c_double()
    bad = ctypes.c_int()
    dkl = np.zeros(n) if want_dkl else None
    rc = library().oed_eig_host(ctx.handle, hp(th_keep), hp(w_keep), n, _darr(lo), _darr(hi),
                                float(rel_step), float(sigma), ctypes.byref(eig),
                                dkl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_dkl else None,
                                ctypes.byref(bad))
    _check(ctx.handle, rc, "oed_eig_host")
    return eig.value, dkl, bad.value


def oed_gauss_newton_noalloc(g, lo, hi, rel_step: float, sigma: float, H, stream=None):
    """Allocation-free H_1[n][7][7] from seismograms g[n][15 or 7][nlev][nrec][2] (FP64,
    device).  For callers that cannot allocate device memory while they run; its scratch
    is a fixed 4 MiB array inside the library, shared by all calls on a device (calls that
    overlap on the GPU race).  Returns the status code (0 = OED_OK).  Shapes and dtypes
    are checked here: a wrong-sized or FP32 tensor would otherwise be read or written
    past its end on the device."""
    import torch
    if g.dim() != 5 or g.shape[4] != 2 or g.dtype != torch.float64:
        raise ValueError("g must be a float64 tensor of shape [n][15 or 7][nlev][nrec][2]")
    n, per_node, nlev, nrec = g.shape[0], g.shape[1], g.shape[2], g.shape[3]
    if H.dtype != torch.float64 or tuple(H.shape) != (n, 7, 7):
        raise ValueError("H must be a float64 tensor of shape [n][7][7]")
    if g.device != H.device or g.device.index != torch.cuda.current_device():
        raise ValueError("g and H must be on the current CUDA device")
    return int(library().oed_gauss_newton_noalloc(_ptr(g), n, per_node, nlev, nrec, _darr(lo),
                                                  _darr(hi), float(rel_step), float(sigma), _ptr(H),
                                                  _stream(stream)))


def make_request(problem: Problem, theta, w, lo, hi, rel_step: float, sigma: float,
                 jacobian: int = OED_JAC_PAIRS, H_done=None, tag: int = 0) -> Request:
    """Build an oed_request from host arrays (kept alive on the returned object).  H_done
    ([k][7][7], from Server.checkpoint of a request on the same nodes) resumes it: the
    first k nodes are not recomputed."""
    import numpy as np
    r = Request()
    r.problem = problem
    r._keep = [problem]
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 7)
    wt = np.ascontiguousarray(w, dtype=np.float64)
    r._th, r._w, r._lo, r._hi = th, wt, _darr(lo), _darr(hi)
    r.n = th.shape[0]
    r.theta = th.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.w = wt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.lo, r.hi = r._lo, r._hi
    r.rel_step, r.sigma, r.jacobian = float(rel_step), float(sigma), int(jacobian)
    if H_done is not None and len(H_done):
        hd = np.ascontiguousarray(H_done, dtype=np.float64).reshape(-1, 7, 7)
        if hd.shape[0] > r.n:
            raise ValueError("H_done has more nodes than the request")
        r._hd = hd
        r.n_done = hd.shape[0]
        r.H_done = hd.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.tag = int(tag)
    return r


class Server:
    """oed_server: continuous batching of EIG requests with admission by device footprint."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 4, chunk_nodes: int = 64,
                 autotune: bool = True):
        self.handle = ctypes.c_void_p()
        rc = library().oed_server_create(ctypes.byref(self.handle), int(hbm_budget_bytes),
                                         int(max_active), int(chunk_nodes),
                                         0 if autotune else OED_SERVER_NO_AUTOTUNE)
        if rc != OED_OK:
            raise OedError(rc, "oed_server_create failed")
        self.chunk_nodes = int(chunk_nodes)

    def request_bytes(self, req: Request) -> int:
        return int(library().oed_server_request_bytes(ctypes.byref(req), self.chunk_nodes))

    def submit(self, req: Request) -> int:
        rid = ctypes.c_ulonglong()
        rc = library().oed_server_submit(self.handle, ctypes.byref(req), ctypes.byref(rid))
        if rc != OED_OK:
            raise OedError(rc, "oed_server_submit")
        return int(rid.value)

    def poll(self, rid: int) -> Result:
        out = Result()
        _check(None, library().oed_server_poll(self.handle, rid, ctypes.byref(out)), "oed_server_poll")
        return out

    def wait(self, rid: int, timeout_s: float = 600.0) -> Result:
        out = Result()
        rc = library().oed_server_wait(self.handle, rid, float(timeout_s), ctypes.byref(out))
        if rc not in (OED_OK, OED_ETIMEOUT):
            raise OedError(rc, "oed_server_wait")
        return out

    def stats(self):
        b, a, q = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        library().oed_server_stats(self.handle, ctypes.byref(b), ctypes.byref(a), ctypes.byref(q))
        return int(b.value), int(a.value), int(q.value)

    def pool(self):
        """(idle pooled workspaces, their bytes)."""
        k, b = ctypes.c_int(), ctypes.c_size_t()
        library().oed_server_pool(self.handle, ctypes.byref(k), ctypes.byref(b))
        return int(k.value), int(b.value)

    def set_admission(self, max_wait_s: float):
        _check(None, library().oed_server_set_admission(self.handle, float(max_wait_s)),
               "oed_server_set_admission")

    def set_log(self, path: Optional[str]):
        _check(None, library().oed_server_set_log(self.handle, None if path is None else path.encode()),
               "oed_server_set_log")

    def cancel(self, rid: int):
        _check(None, library().oed_server_cancel(self.handle, rid), "oed_server_cancel")

    def checkpoint(self, rid: int):
        """Per-node Hessians finished so far, numpy [k][7][7]."""
        import numpy as np
        k = ctypes.c_int()
        _check(None, library().oed_server_checkpoint(self.handle, rid, None, 0, ctypes.byref(k)),
               "oed_server_checkpoint")
        H = np.zeros((max(1, k.value), 7, 7))
        _check(None, library().oed_server_checkpoint(self.handle, rid,
                                                     H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                     H.shape[0], ctypes.byref(k)), "oed_server_checkpoint")
        return H[:k.value]

    def release(self, rid: int) -> int:
        """Drop a finished request's record; returns the status code (OED_PENDING if it is
        still running)."""
        return int(library().oed_server_release(self.handle, rid))

    def metrics(self, rid: int) -> dict:
        """The finished request's JSON metrics line, parsed."""
        import json
        buf = ctypes.create_string_buffer(4096)
        _check(None, library().oed_server_metrics(self.handle, rid, buf, 4096), "oed_server_metrics")
        return json.loads(buf.value.decode())

    def close(self):
        if self.handle:
            library().oed_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
