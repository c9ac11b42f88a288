"""Python face of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It wraps ``oed_oracle.c`` (compiled with
gcc into ``liboedref.so`` next to this file) and adds the sparse-grid rule in
plain numpy.  It shares no code with the CUDA library.

Paper: Long, Motamed & Tempone, "Fast Bayesian optimal experimental design for
seismic source inversion", arXiv:1502.07873.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
from math import comb

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oed_oracle.c")
LIB = os.path.join(HERE, "liboedref.so")
NT = 7

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP over nodes only)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        L.ref_delta_1d.argtypes = [c_double, c_double, dp, dp]
        L.ref_delta_1d.restype = None
        L.ref_stf.argtypes = [c_double, c_double, c_double]
        L.ref_stf.restype = c_double
        L.ref_media.argtypes = [c_int, c_int, c_double, c_int, dp, dp, dp, dp, dp, dp, dp]
        L.ref_media.restype = None
        L.ref_source_patch.argtypes = [dp, c_int, c_int, c_double, ip, ip, dp, dp]
        L.ref_source_patch.restype = c_int
        L.ref_step.argtypes = [ctypes.c_void_p] + [dp] * 8
        L.ref_step.restype = None
        L.ref_forward.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip,
                                  dp, dp]
        L.ref_forward.restype = c_int
        L.ref_node_hessian.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int,
                                       ip, dp, dp, dp, c_double, c_double, c_int, ip, dp, dp]
        L.ref_node_hessian.restype = c_int
        L.ref_delta_1d_dxs.argtypes = [c_double, c_double, dp, dp]
        L.ref_delta_1d_dxs.restype = None
        L.ref_node_hessian_sens.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp,
                                            c_int, ip, dp, c_double, dp]
        L.ref_node_hessian_sens.restype = c_int
        L.ref_scaled_logdet.argtypes = [dp, dp, dp]
        L.ref_scaled_logdet.restype = c_int
        L.ref_dkl.argtypes = [c_double, c_int, c_double]
        L.ref_dkl.restype = c_double
        L.ref_eig.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip,
                              c_int, dp, dp, dp, dp, c_double, c_double, c_int, dp, dp, ip, dp]
        L.ref_eig.restype = c_int
        L.ref_scaled_logdet_sub.argtypes = [dp, c_int, dp]
        L.ref_scaled_logdet_sub.restype = c_int
        L.ref_dlmc.argtypes = [dp, dp, c_int, dp, c_int, c_int, c_double, dp, dp]
        L.ref_dlmc.restype = None
        L.ref_ricker.argtypes = [c_double, c_double, c_double]
        L.ref_ricker.restype = c_double
        L.ref_forward_stf.argtypes = [c_int] + L.ref_forward.argtypes
        L.ref_forward_stf.restype = c_int
        L.ref_node_hessian_stf.argtypes = [c_int] + L.ref_node_hessian.argtypes
        L.ref_node_hessian_stf.restype = c_int
        L.ref_delta_1d_dxs2.argtypes = [c_double, c_double, dp, dp]
        L.ref_delta_1d_dxs2.restype = None
        L.ref_stf_derivs.argtypes = [c_double, c_double, c_double, dp]
        L.ref_stf_derivs.restype = None
        L.ref_jacobian_sens.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip,
                                        dp, dp]
        L.ref_jacobian_sens.restype = c_int
        L.ref_forward_field.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip,
                                        dp, dp]
        L.ref_forward_field.restype = None
        L.ref_adjoint.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip, dp, dp]
        L.ref_adjoint.restype = None
        L.ref_hessian_ii.argtypes = [c_int, c_int, c_double, c_double, c_int, dp, dp, dp, c_int, ip,
                                     dp, dp, c_double, dp, dp]
        L.ref_hessian_ii.restype = c_int
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------- source
def delta_weights(alpha: float, h: float):
    """Six-point regularised delta and delta' weights at nodes k-2..k+3 (Sec. 3.3.2)."""
    d = np.zeros(6)
    dp = np.zeros(6)
    lib().ref_delta_1d(float(alpha), float(h), _pd(d), _pd(dp))
    return d, dp


def delta_weights_dxs(alpha: float, h: float):
    """d/dx_s of the delta and delta' weights (Alg. 1 step 2)."""
    d = np.zeros(6)
    dp = np.zeros(6)
    lib().ref_delta_1d_dxs(float(alpha), float(h), _pd(d), _pd(dp))
    return d, dp


def stf(t: float, ts: float, ws: float) -> float:
    """Gaussian source time function (Sec. 4.1) with omega_0 = omega_s."""
    return lib().ref_stf(float(t), float(ts), float(ws))


def ricker(t: float, ts: float, f: float) -> float:
    """Ricker wavelet (1 - 2a) exp(-a), a = (pi f (t - t_s))^2: the optional alternative time function."""
    return lib().ref_ricker(float(t), float(ts), float(f))


STF_GAUSS, STF_RICKER = 0, 1


def source_patch(theta, nx: int, nz: int, h: float):
    """(i0, j0, fx[6][6], fz[6][6], ok): spatial part of S(t) M grad(delta) (Eq. source)."""
    th = _d(theta)
    i0 = ctypes.c_int()
    j0 = ctypes.c_int()
    fx = np.zeros(36)
    fz = np.zeros(36)
    rc = lib().ref_source_patch(_pd(th), nx, nz, float(h), ctypes.byref(i0), ctypes.byref(j0),
                                _pd(fx), _pd(fz))
    return i0.value, j0.value, fx.reshape(6, 6), fz.reshape(6, 6), rc == 0


# ---------------------------------------------------------------- media / grid
class Grid:
    """Grid and node media of a workload (layered in depth)."""

    def __init__(self, nx, nz, h, dt, nsteps, layers, rec_ix):
        self.nx, self.nz, self.h, self.dt, self.nsteps = int(nx), int(nz), float(h), float(dt), int(nsteps)
        z_top = _d([l[0] for l in layers])
        vp = _d([l[1] for l in layers])
        vs = _d([l[2] for l in layers])
        rho = _d([l[3] for l in layers])
        n = self.nx * self.nz
        self.lam, self.mu, self.nu = np.zeros(n), np.zeros(n), np.zeros(n)
        lib().ref_media(self.nx, self.nz, self.h, len(layers), _pd(z_top), _pd(vp), _pd(vs),
                        _pd(rho), _pd(self.lam), _pd(self.mu), _pd(self.nu))
        self.rec_ix = _i(rec_ix)
        self.nrec = len(self.rec_ix)

    @classmethod
    def from_workload(cls, w):
        return cls(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, w.rec_ix)

    @classmethod
    def from_arrays(cls, nx, nz, h, dt, nsteps, lam, mu, nu, rec_ix):
        g = cls.__new__(cls)
        g.nx, g.nz, g.h, g.dt, g.nsteps = int(nx), int(nz), float(h), float(dt), int(nsteps)
        g.lam, g.mu, g.nu = _d(lam).ravel().copy(), _d(mu).ravel().copy(), _d(nu).ravel().copy()
        g.rec_ix = _i(rec_ix)
        g.nrec = len(g.rec_ix)
        return g

    def _args(self):
        return (self.nx, self.nz, self.h, self.dt, self.nsteps, _pd(self.lam), _pd(self.mu),
                _pd(self.nu), self.nrec, _pi(self.rec_ix))


class _RefGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("lam", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("nu", ctypes.c_void_p)]


def step(grid: Grid, ux, uz, uxm, uzm, fx=None, fz=None):
    """One leap-frog step of the FD scheme (Eq. Full_Disc) on [nz][nx] fields."""
    shape = (grid.nz, grid.nx)
    a = [_d(x).reshape(shape) for x in (ux, uz, uxm, uzm)]
    f = [_d(x).reshape(shape) if x is not None else np.zeros(shape) for x in (fx, fz)]
    uxn, uzn = np.zeros(shape), np.zeros(shape)
    G = _RefGrid(grid.nx, grid.nz, grid.h, grid.dt, grid.lam.ctypes.data, grid.mu.ctypes.data,
                 grid.nu.ctypes.data)
    lib().ref_step(ctypes.byref(G), *[_pd(x) for x in a], _pd(f[0]), _pd(f[1]), _pd(uxn), _pd(uzn))
    return uxn, uzn


def forward(grid: Grid, theta, stf=STF_GAUSS):
    """Seismograms g[m][r][c], m = 0..nsteps (Eq. forward_model); stf picks the time function."""
    g = np.zeros((grid.nsteps + 1, grid.nrec, 2))
    rc = lib().ref_forward_stf(int(stf), *grid._args(), _pd(_d(theta)), _pd(g))
    if rc != 0:
        raise ValueError("source patch leaves the grid interior")
    return g


def node_hessian(grid: Grid, theta, lo, hi, rel_step, sigma, win_levels=None, stf=STF_GAUSS):
    """(H[7][7], H_rec[nrec][nwin][7][7] or None): Gauss-Newton H_1 from central FD."""
    H = np.zeros(49)
    nwin = 0 if win_levels is None else len(win_levels)
    wl = _i(win_levels if win_levels is not None else [0])
    Hr = np.zeros(max(1, grid.nrec * nwin * 49))
    rc = lib().ref_node_hessian_stf(int(stf), *grid._args(), _pd(_d(theta)), _pd(_d(lo)), _pd(_d(hi)),
                                float(rel_step), float(sigma), nwin, _pi(wl), _pd(H),
                                _pd(Hr) if nwin else ctypes.POINTER(ctypes.c_double)())
    if rc != 0:
        raise ValueError("source patch leaves the grid interior")
    return H.reshape(7, 7), (Hr.reshape(grid.nrec, nwin, 7, 7) if nwin else None)


def node_hessian_sensitivity(grid: Grid, theta, sigma):
    """H_I (7x7) of Alg. 1 steps 1-5: sensitivity solves driven by df/dtheta_j."""
    H = np.zeros(49)
    rc = lib().ref_node_hessian_sens(*grid._args(), _pd(_d(theta)), float(sigma), _pd(H))
    if rc != 0:
        raise ValueError("source patch leaves the grid interior")
    return H.reshape(7, 7)


def scaled_logdet(H):
    """(logdet, Htilde, ok) with S = sqrt(diag H), Htilde = S^-1 H S^-1 (Sec. 3.3.3)."""
    Hd = _d(H).ravel()
    ld = ctypes.c_double()
    Ht = np.zeros(49)
    rc = lib().ref_scaled_logdet(_pd(Hd), ctypes.byref(ld), _pd(Ht))
    return ld.value, Ht.reshape(7, 7), rc == 0


def delta_weights_dxs2(alpha: float, h: float):
    """Second x_s-derivatives of the delta and delta' weights (Alg. 1 step 9)."""
    d = np.zeros(6)
    dp = np.zeros(6)
    lib().ref_delta_1d_dxs2(float(alpha), float(h), _pd(d), _pd(dp))
    return d, dp


def stf_derivs(t: float, ts: float, ws: float):
    """(S, S_ts, S_w, S_tsts, S_tsw, S_ww) at t."""
    out = np.zeros(6)
    lib().ref_stf_derivs(float(t), float(ts), float(ws), _pd(out))
    return out


def jacobian_sensitivity(grid: Grid, theta):
    """J[j][m][r][c] = dg/dtheta_j from sensitivity solves (Alg. 1 steps 1-3)."""
    J = np.zeros((7, grid.nsteps + 1, grid.nrec, 2))
    rc = lib().ref_jacobian_sens(*grid._args(), _pd(_d(theta)), _pd(J))
    if rc != 0:
        raise ValueError("source patch leaves the grid interior")
    return J


def forward_field(grid: Grid, f):
    """Seismograms of a full forcing sequence f[m][c][nz][nx], m < nsteps."""
    f = _d(f)
    assert f.shape == (grid.nsteps, 2, grid.nz, grid.nx)
    g = np.zeros((grid.nsteps + 1, grid.nrec, 2))
    lib().ref_forward_field(*grid._args(), _pd(f), _pd(g))
    return g


def adjoint(grid: Grid, w):
    """Dual solve (Eq. Dual_problems): dJ/df^m [m][c][nz][nx] for J = sum w . g."""
    w = _d(w)
    assert w.shape == (grid.nsteps + 1, grid.nrec, 2)
    gf = np.zeros((grid.nsteps, 2, grid.nz, grid.nx))
    lib().ref_adjoint(*grid._args(), _pd(w), _pd(gf))
    return gf


def hessian_ii(grid: Grid, theta, y, sigma):
    """(H_II [7][7], dL/dtheta [7]) at theta for data y (Alg. 1 steps 6-10)."""
    y = _d(y)
    assert y.shape == (grid.nsteps + 1, grid.nrec, 2)
    H2 = np.zeros(49)
    gr = np.zeros(7)
    rc = lib().ref_hessian_ii(*grid._args(), _pd(_d(theta)), _pd(y), float(sigma), _pd(H2), _pd(gr))
    if rc != 0:
        raise ValueError("source patch leaves the grid interior")
    return H2.reshape(7, 7), gr


def scaled_logdet_sub(H, free):
    """(logdet, ok) of the sub-block of H over the unknown parameters `free` (indices)."""
    mask = 0
    for j in free:
        mask |= 1 << int(j)
    ld = ctypes.c_double()
    rc = lib().ref_scaled_logdet_sub(_pd(_d(H).ravel()), int(mask), ctypes.byref(ld))
    return ld.value, rc == 0


def dlmc(g_outer, eps, g_inner, sigma):
    """Double-loop Monte Carlo EIG (Eq. expected_I by direct sampling, Sec. 4.4):
    returns (log_ev[N], eig).  g_outer, eps: [N][D]; g_inner: [M][D]."""
    go = _d(g_outer).reshape(len(g_outer), -1)
    e = _d(eps).reshape(go.shape)
    gi = _d(g_inner).reshape(len(g_inner), -1)
    assert gi.shape[1] == go.shape[1]
    N, D = go.shape
    le = np.zeros(N)
    eig = ctypes.c_double()
    lib().ref_dlmc(_pd(go), _pd(e), N, _pd(gi), gi.shape[0], D, float(sigma), _pd(le), ctypes.byref(eig))
    return le, eig.value


def dkl(logdet: float, n: int, log_prior_density: float) -> float:
    """D_KL-hat of Thm 4 (Eq. DKL_hat)."""
    return lib().ref_dkl(float(logdet), int(n), float(log_prior_density))


def eig(grid: Grid, theta, w, lo, hi, rel_step, sigma, nthreads=0, want_h=False):
    """EIG = sum_i w_i D_KL-hat(theta_i) (Eqs. intpoly / mcs).  Returns a dict."""
    th = _d(theta).reshape(-1, 7)
    n = th.shape[0]
    e = ctypes.c_double()
    D = np.zeros(max(n, 1))
    st = np.zeros(max(n, 1), dtype=np.int32)
    H = np.zeros(max(n, 1) * 49)
    used = lib().ref_eig(*grid._args(), n, _pd(th), _pd(_d(w)), _pd(_d(lo)), _pd(_d(hi)),
                         float(rel_step), float(sigma), int(nthreads), ctypes.byref(e), _pd(D),
                         _pi(st), _pd(H))
    out = {"eig": e.value, "dkl": D[:n], "status": st[:n], "threads": used}
    if want_h:
        out["H"] = H[: n * 49].reshape(n, 7, 7)
    return out


def noise_sigma(grid_all_surface: Grid, theta_mean, frac=0.01) -> float:
    """sigma = frac * peak |u| over every surface node, both components and all levels,
    at the prior-mean source (the noise level of the synthetic workloads)."""
    g = forward(grid_all_surface, theta_mean)
    return frac * float(np.max(np.abs(g)))


def log_uniform_density(lo, hi) -> float:
    return -float(np.sum(np.log(np.asarray(hi, float) - np.asarray(lo, float))))


# ---------------------------------------------------------------- quadrature
def mc_nodes(u, lo, hi):
    """Monte Carlo nodes theta = lo + (hi - lo) U with equal weights 1/M (Eq. mcs)."""
    u = np.asarray(u, float)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    return lo + (hi - lo) * u, np.full(u.shape[0], 1.0 / u.shape[0])


def smolyak(dim: int, level: int, lo=None, hi=None, merge_tol: float = 1e-11):
    """Smolyak sparse grid (Eq. intpoly) with 1-D Gauss-Legendre rules of m(l) = l + 1
    points, l >= 0, over the total-degree index set level - dim + 1 <= |l| <= level,
    combination coefficients (-1)^(level - |l|) C(dim - 1, level - |l|), coinciding
    nodes merged with summed weights.  Weights are for the uniform probability
    measure (they sum to 1).  Nodes are mapped affinely to [lo, hi] if given."""
    rules = {}
    for l in range(level + 1):
        x, w = np.polynomial.legendre.leggauss(l + 1)
        rules[l] = (x, w / 2.0)
    acc = {}
    for idx in itertools.product(range(level + 1), repeat=dim):
        s = sum(idx)
        if s > level or s < level - dim + 1:
            continue
        c = (-1) ** (level - s) * comb(dim - 1, level - s)
        if c == 0:
            continue
        xs = [rules[l][0] for l in idx]
        ws = [rules[l][1] for l in idx]
        for pts in itertools.product(*[range(len(x)) for x in xs]):
            node = tuple(xs[k][p] for k, p in enumerate(pts))
            wt = c * math.prod(ws[k][p] for k, p in enumerate(pts))
            key = tuple(int(round(v / merge_tol)) for v in node)
            if key in acc:
                acc[key][1] += wt
            else:
                acc[key] = [np.array(node), wt]
    nodes = np.array([v[0] for v in acc.values()])
    weights = np.array([v[1] for v in acc.values()])
    order = np.lexsort(nodes.T[::-1])
    nodes, weights = nodes[order], weights[order]
    if lo is not None:
        lo = np.asarray(lo, float)
        hi = np.asarray(hi, float)
        nodes = lo + (hi - lo) * (nodes + 1.0) / 2.0
    return nodes, weights
