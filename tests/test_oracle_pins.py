"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped index or a transposed operand) fails at least one of them:
exact moment conditions of the regularised delta, exactness of the FD operator
on quadratic fields, exact traction-free behaviour at the surface, the
absorbing-boundary rates, second-order convergence, linearity in the moment
tensor, additivity / scaling of H_1, a brute-force determinant, and the
linear-Gaussian closed form of the expected information gain.
"""
import itertools
import math
import os

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
VP, VS, RHO = 3000.0, 1732.0, 2500.0
MU = RHO * VS * VS
LAM = RHO * (VP * VP - 2 * VS * VS)
P2 = LAM + 2 * MU


# ------------------------------------------------------------------ delta (Sec. 3.3.2)
@pytest.mark.parametrize("alpha", [0.0, 0.13, 0.5, 0.77, 0.999])
@pytest.mark.parametrize("h", [1.0, 25.0])
def test_delta_moments_exact(oracle, alpha, h):
    """Discrete moments: h sum d_j (x_j - x_s)^q = [q = 0], h sum d'_j (x_j - x_s)^q = -[q = 1],
    q = 0..4 (the defining conditions of the fourth-order regularisation)."""
    d, dp = oracle.delta_weights(alpha, h)
    xj = (np.arange(-2, 4) - alpha) * h
    for q in range(5):
        m0 = h * np.sum(d * xj ** q)
        m1 = h * np.sum(dp * xj ** q)
        assert abs(m0 - (1.0 if q == 0 else 0.0)) < 1e-12 * max(1.0, h ** q)
        assert abs(m1 - (-1.0 if q == 1 else 0.0)) < 1e-12 * max(1.0, h ** q)


def test_delta_continuous_across_cells(oracle):
    """The weights of cell k at alpha -> 1 equal those of cell k+1 at alpha = 0 shifted by one
    node, and so do their first two alpha-derivatives (the discretisation is C^2 in x_s)."""
    eps = 1e-5

    def wts(a):
        d, dp = oracle.delta_weights(a, 1.0)
        return np.concatenate([d, [0.0]]), np.concatenate([dp, [0.0]])

    def shifted(a):
        d, dp = oracle.delta_weights(a, 1.0)
        return np.concatenate([[0.0], d]), np.concatenate([[0.0], dp])

    for k in range(2):
        left = wts(1.0)[k]
        right = shifted(0.0)[k]
        assert np.allclose(left, right, atol=1e-12)
        dl = (wts(1.0)[k] - wts(1.0 - eps)[k]) / eps
        dr = (shifted(eps)[k] - shifted(0.0)[k]) / eps
        assert np.allclose(dl, dr, atol=1e-3)
        d2l = (wts(1.0)[k] - 2 * wts(1.0 - eps)[k] + wts(1.0 - 2 * eps)[k]) / eps ** 2
        d2r = (shifted(2 * eps)[k] - 2 * shifted(eps)[k] + shifted(0.0)[k]) / eps ** 2
        assert np.allclose(d2l, d2r, atol=2e-1)


def test_source_time_function_moments(oracle):
    """S(t) with omega_0 = omega_s has unit area, mean t_s and variance 1/omega_s^2."""
    ts, ws = 1.3, 4.5
    t = np.linspace(ts - 12 / ws, ts + 12 / ws, 200001)
    s = np.array([oracle.stf(x, ts, ws) for x in t[::10]])
    tt = t[::10]
    dt = tt[1] - tt[0]
    area = np.sum(s) * dt
    mean = np.sum(s * tt) * dt
    var = np.sum(s * (tt - ts) ** 2) * dt
    assert abs(area - 1) < 1e-9
    assert abs(mean - ts) < 1e-9
    assert abs(var - 1 / ws ** 2) < 1e-9


def test_source_patch_moments(oracle):
    """First moments of the discrete force density equal minus the moment tensor:
    sum h^2 f_i (x_k - x_{s,k}) = -M_ik, and the total force vanishes (Eq. source)."""
    h = 10.0
    th = np.array([503.7, 311.2, 0.2, 5.0, 2.0e13, -3.0e13, 7.0e13])
    i0, j0, fx, fz, ok = oracle.source_patch(th, 101, 61, h)
    assert ok
    xi = (i0 + np.arange(6)) * h - th[0]
    zj = (j0 + np.arange(6)) * h - th[1]
    X, Z = np.meshgrid(xi, zj)   # [b][a]
    M = {"xx": th[4], "xz": th[5], "zz": th[6]}
    sc = 1e13
    assert abs(np.sum(fx) * h * h) / sc < 1e-10
    assert abs(np.sum(fz) * h * h) / sc < 1e-10
    assert abs(np.sum(fx * X) * h * h + M["xx"]) / sc < 1e-10
    assert abs(np.sum(fx * Z) * h * h + M["xz"]) / sc < 1e-10
    assert abs(np.sum(fz * X) * h * h + M["xz"]) / sc < 1e-10
    assert abs(np.sum(fz * Z) * h * h + M["zz"]) / sc < 1e-10


def test_source_patch_out_of_range_rejected(oracle):
    th = np.array([5.0, 300.0, 0.2, 5.0, 1e13, 1e13, 1e13])
    assert not oracle.source_patch(th, 101, 61, 10.0)[4]


# ------------------------------------------------------------------ operator A_h, B_h
def _grid(oracle, nx=13, nz=9, h=7.0, dt=1e-3):
    return oracle.Grid(nx, nz, h, dt, 1, W.HOMOGENEOUS, [0])


def _apply(oracle, G, ux, uz):
    """A_h u recovered from one step with u^{m-1} = u^m and no forcing."""
    uxn, uzn = oracle.step(G, ux, uz, ux, uz)
    return (uxn - ux) * RHO / G.dt ** 2, (uzn - uz) * RHO / G.dt ** 2


QUADRATICS = [  # (ux(x, z), uz(x, z), (A u)_x, (A u)_z) of the continuous operator
    (lambda x, z: x * x, lambda x, z: 0 * x, 2 * P2, 0.0),
    (lambda x, z: z * z, lambda x, z: 0 * x, 2 * MU, 0.0),
    (lambda x, z: 0 * x, lambda x, z: x * x, 0.0, 2 * MU),
    (lambda x, z: 0 * x, lambda x, z: z * z, 0.0, 2 * P2),
    (lambda x, z: x * z, lambda x, z: 0 * x, 0.0, LAM + MU),
    (lambda x, z: 0 * x, lambda x, z: x * z, LAM + MU, 0.0),
]


@pytest.mark.parametrize("k", range(len(QUADRATICS)))
def test_interior_operator_exact_on_quadratics(oracle, k):
    """A second-order operator reproduces div sigma exactly on quadratic fields; each field
    isolates one of the eight terms, with its sign and coefficient."""
    G = _grid(oracle)
    fx_, fz_, ax, az = QUADRATICS[k]
    x = np.arange(G.nx) * G.h + 3.0
    z = np.arange(G.nz) * G.h
    X, Z = np.meshgrid(x, z)
    Ax, Az = _apply(oracle, G, fx_(X, Z), fz_(X, Z))
    sl = (slice(1, G.nz - 1), slice(1, G.nx - 1))
    scale = abs(P2) * 4
    assert np.max(np.abs(Ax[sl] - ax)) < 1e-6 * scale
    assert np.max(np.abs(Az[sl] - az)) < 1e-6 * scale


TRACTION_FREE = [  # fields with sigma_xz = sigma_zz = 0 at z = 0 and their div sigma
    (lambda x, z: z * z, lambda x, z: 0 * x, 2 * MU, 0.0),
    (lambda x, z: 0 * x, lambda x, z: z * z, 0.0, 2 * P2),
    (lambda x, z: x * x, lambda x, z: -2 * LAM / P2 * x * z, 2 * P2 - 2 * LAM / P2 * (LAM + MU), 0.0),
    (lambda x, z: -2 * x * z, lambda x, z: x * x, 0.0, -2 * LAM),
]


@pytest.mark.parametrize("k", range(len(TRACTION_FREE)))
def test_free_surface_exact_on_traction_free_quadratics(oracle, k):
    """On the surface row the operator reproduces div sigma exactly for quadratic fields that
    satisfy the traction-free conditions (Eq. elastic_3rd)."""
    G = _grid(oracle)
    fx_, fz_, ax, az = TRACTION_FREE[k]
    x = np.arange(G.nx) * G.h - 20.0
    z = np.arange(G.nz) * G.h
    X, Z = np.meshgrid(x, z)
    Ax, Az = _apply(oracle, G, fx_(X, Z), fz_(X, Z))
    scale = abs(P2) * 4
    assert np.max(np.abs(Ax[0, 1:-1] - ax)) < 1e-6 * scale
    assert np.max(np.abs(Az[0, 1:-1] - az)) < 1e-6 * scale


def test_absorbing_rows_rates(oracle):
    """First-order Clayton-Engquist rows: d_t u = -c d_n u with c_p for the normal and c_s for
    the tangential component, outward normal -x, +x (sides) and +z (bottom)."""
    G = _grid(oracle)
    x = np.arange(G.nx) * G.h
    z = np.arange(G.nz) * G.h
    X, Z = np.meshgrid(x, z)
    zero = 0 * X
    for ux, uz in ((X, zero), (zero, X), (Z, zero), (zero, Z)):
        uxn, uzn = oracle.step(G, ux, uz, ux, uz)
        rx, rz = (uxn - ux) / G.dt, (uzn - uz) / G.dt
        gx = 1.0 if ux is X else 0.0
        gzx = 1.0 if uz is X else 0.0
        gxz = 1.0 if ux is Z else 0.0
        gz = 1.0 if uz is Z else 0.0
        # left column: outward -x, d_t u = +c d_x u; right column: d_t u = -c d_x u
        assert np.allclose(rx[:, 0], VP * gx, rtol=1e-9, atol=1e-6)
        assert np.allclose(rz[:, 0], VS * gzx, rtol=1e-9, atol=1e-6)
        assert np.allclose(rx[:, -1], -VP * gx, rtol=1e-9, atol=1e-6)
        assert np.allclose(rz[:, -1], -VS * gzx, rtol=1e-9, atol=1e-6)
        # bottom row (without corners): d_t u = -c d_z u
        assert np.allclose(rx[-1, 1:-1], -VS * gxz, rtol=1e-9, atol=1e-6)
        assert np.allclose(rz[-1, 1:-1], -VP * gz, rtol=1e-9, atol=1e-6)


def test_scheme_spectral_radius_at_most_one(oracle):
    """The one-step map of the full scheme (free surface, absorbing sides and bottom, two
    layers) has spectral radius <= 1: no growing mode."""
    layers = ((0.0, 2000.0, 1155.0, 2200.0), (150.0, 4500.0, 2598.0, 2700.0))
    nx, nz, h = 13, 9, 25.0
    G = oracle.Grid(nx, nz, h, 0.5 * h / 4500.0, 1, layers, [0])
    n = nx * nz
    A = np.zeros((4 * n, 4 * n))
    for k in range(4 * n):
        v = np.zeros(4 * n)
        v[k] = 1.0
        ux, uz, uxm, uzm = (v[i * n:(i + 1) * n].reshape(nz, nx) for i in range(4))
        a, b = oracle.step(G, ux, uz, uxm, uzm)
        A[:, k] = np.concatenate([a.ravel(), b.ravel(), ux.ravel(), uz.ravel()])
    rho = np.max(np.abs(np.linalg.eigvals(A)))
    assert rho <= 1.0 + 1e-9


def test_energy_decays_after_source(oracle):
    """With the source switched off the wavefield leaves through the absorbing boundaries."""
    w = W.plain_small()
    G = oracle.Grid(w.nx, w.nz, w.h, w.dt, 10 * w.nsteps, w.layers, list(range(0, w.nx, 4)))
    g = oracle.forward(G, [1000.0, 500.0, 0.2, 6.0, 5e13, 3e13, 4e13])
    env = np.abs(g).reshape(g.shape[0], -1).max(axis=1)
    peak = env.max()
    late = env[-w.nsteps:]
    assert np.all(np.isfinite(env))
    assert late.max() < 0.2 * peak
    assert late[-1] <= late[0] * 1.5


@pytest.mark.slow
def test_second_order_convergence(oracle):
    """Seismograms converge at second order under h -> h/2 (dt proportional to h), at an
    interior and a surface receiver, for a smooth source away from the boundaries."""
    th = np.array([3000.0, 1500.0, 0.6, 8.0, 5e13, 2e13, 3e13])

    def rate(rx, rz, T):
        res = []
        for h in (100.0, 50.0, 25.0, 12.5):
            nx, nz = int(6000 / h) + 1, int(3000 / h) + 1
            dt = 0.5 * h / 3000.0
            ix = int(round(rx / h)) + int(round(rz / h)) * nx
            G = oracle.Grid(nx, nz, h, dt, int(round(T / dt)), W.HOMOGENEOUS, [ix])
            res.append(oracle.forward(G, th)[:: int(round(100 / h))])
        n = min(len(r) for r in res)
        e = [np.abs(res[k][:n] - res[k + 1][:n]).max() for k in range(3)]
        return math.log2(e[1] / e[2])

    assert rate(3600.0, 2100.0, 1.1) > 1.8
    assert rate(3600.0, 0.0, 1.35) > 1.8


def test_mirror_symmetry(oracle):
    """A source on the mid-line with m_xz = 0: u_x is odd and u_z even about x_s."""
    nx, nz, h = 41, 21, 50.0
    xc = (nx - 1) // 2
    recs = [xc - 12, xc - 5, xc + 5, xc + 12]
    G = oracle.Grid(nx, nz, h, 0.5 * h / VP, 300, W.HOMOGENEOUS, recs)
    g = oracle.forward(G, [xc * h, 500.0, 0.2, 6.0, 4e13, 0.0, 7e13])
    sc = np.abs(g).max()
    assert np.allclose(g[:, 0, 0], -g[:, 3, 0], atol=1e-11 * sc)
    assert np.allclose(g[:, 1, 0], -g[:, 2, 0], atol=1e-11 * sc)
    assert np.allclose(g[:, 0, 1], g[:, 3, 1], atol=1e-11 * sc)
    assert np.allclose(g[:, 1, 1], g[:, 2, 1], atol=1e-11 * sc)


def test_linear_in_moment_tensor(oracle):
    """g is linear in (m_xx, m_xz, m_zz) (Eq. source)."""
    w = W.tiny()
    G = oracle.Grid.from_workload(w)
    base = [950.0, 470.0, 0.15, 5.5]
    m = [2e13, -5e13, 8e13]
    g = oracle.forward(G, base + m)
    parts = [oracle.forward(G, base + list(np.eye(3)[k])) for k in range(3)]
    comb_ = sum(m[k] * parts[k] for k in range(3))
    assert np.max(np.abs(g - comb_)) < 1e-12 * np.max(np.abs(g))


# ------------------------------------------------------------------ Jacobian and H_1
@pytest.fixture(scope="module")
def tiny_setup(oracle):
    w = W.tiny(nsteps=120, nrec=4)
    G = oracle.Grid.from_workload(w)
    th = np.array([1010.0, 520.0, 0.2, 6.0, 4e13, 2e13, 6e13])
    H, Hr = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step, 0.3,
                                win_levels=[31, 81, w.nlevels])
    return w, G, th, H, Hr


def test_hessian_symmetric_psd(tiny_setup, oracle):
    w, G, th, H, Hr = tiny_setup
    assert np.allclose(H, H.T, rtol=1e-14, atol=0)
    ld, Ht, ok = oracle.scaled_logdet(H)
    assert ok
    assert np.all(np.linalg.eigvalsh(Ht) > 0)
    assert np.allclose(np.diag(Ht), 1.0)


def test_hessian_moment_columns_equal_unit_solves(tiny_setup, oracle):
    """The FD Jacobian columns of m_xx, m_xz, m_zz equal the unit-moment seismograms (the
    map is linear in M), so H_1's moment block is their Gram matrix over sigma^2."""
    w, G, th, H, Hr = tiny_setup
    base = list(th[:4])
    cols = [oracle.forward(G, base + list(np.eye(3)[k])).ravel() for k in range(3)]
    gram = np.array([[cols[a] @ cols[b] for b in range(3)] for a in range(3)]) / 0.3 ** 2
    assert np.allclose(H[4:, 4:], gram, rtol=1e-8)


def test_hessian_additive_over_receivers_and_windows(tiny_setup, oracle):
    """H_1 is a sum over receivers and time levels (Appendix C): the per-receiver full-window
    blocks add up to H, and a run stopped at level L reproduces the window ending at L."""
    w, G, th, H, Hr = tiny_setup
    assert np.allclose(Hr[:, -1].sum(axis=0), H, rtol=1e-12)
    # receivers split into two runs
    G1 = oracle.Grid(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, w.rec_ix[:2])
    G2 = oracle.Grid(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, w.rec_ix[2:])
    H1, _ = oracle.node_hessian(G1, th, w.prior_lo, w.prior_hi, w.rel_step, 0.3)
    H2, _ = oracle.node_hessian(G2, th, w.prior_lo, w.prior_hi, w.rel_step, 0.3)
    assert np.allclose(H1 + H2, H, rtol=1e-12)
    # causality: a run of 80 steps equals the window of 81 levels
    Gs = oracle.Grid(w.nx, w.nz, w.h, w.dt, 80, w.layers, w.rec_ix)
    Hs, _ = oracle.node_hessian(Gs, th, w.prior_lo, w.prior_hi, w.rel_step, 0.3)
    assert np.allclose(Hs, Hr[:, 1].sum(axis=0), rtol=1e-12)
    # monotone in time (Loewner order)
    assert np.all(np.linalg.eigvalsh(Hr[:, 2].sum(0) - Hr[:, 1].sum(0)) > -1e-9 * np.abs(H).max())


def test_hessian_scaling_and_duplicate_receivers(tiny_setup, oracle):
    w, G, th, H, Hr = tiny_setup
    H2, _ = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step, 0.6)
    assert np.allclose(H2 * 4, H, rtol=1e-12)
    Gd = oracle.Grid(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, list(w.rec_ix) * 2)
    Hd, _ = oracle.node_hessian(Gd, th, w.prior_lo, w.prior_hi, w.rel_step, 0.3)
    assert np.allclose(Hd, 2 * H, rtol=1e-12)


def test_fd_step_richardson(tiny_setup, oracle):
    """Central differences are second order in the step: the change of H_1 between steps
    d, d/2 and d/2, d/4 shrinks by a factor near 4, and is tiny at rel_step = 1e-4."""
    w, G, th, H, Hr = tiny_setup
    H2, _ = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step / 2, 0.3)
    H4, _ = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step / 4, 0.3)
    d = np.sqrt(np.outer(np.diag(H), np.diag(H)))
    e1 = np.abs(H2 - H) / d
    e2 = np.abs(H4 - H2) / d
    k = np.unravel_index(np.argmax(e1), e1.shape)
    assert e1[k] < 1e-5
    assert 3.0 < e1[k] / e2[k] < 5.0


# ------------------------------------------------------------------ log-det, D_KL, EIG
def _det_bruteforce(A):
    """Leibniz expansion over all 7! permutations (no factorisation)."""
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        tot += (-1) ** inv * math.prod(A[i, perm[i]] for i in range(n))
    return tot


def test_scaled_logdet_vs_bruteforce(oracle):
    rng = np.random.default_rng(0)
    B = rng.standard_normal((7, 7))
    A = B @ B.T + 0.5 * np.eye(7)
    s = np.array([1e-3, 1e2, 1.0, 10.0, 1e-14, 3e-14, 1e-13])   # parameter units far apart
    H = A / np.outer(s, s)
    ld, Ht, ok = oracle.scaled_logdet(H)
    assert ok
    ref = math.log(_det_bruteforce(A)) - 2 * np.sum(np.log(s))
    assert abs(ld - ref) < 1e-9 * abs(ref)


def test_scaled_logdet_flags_not_pd(oracle):
    H = np.eye(7)
    H[2, 3] = H[3, 2] = 1.5
    assert not oracle.scaled_logdet(H)[2]
    H = np.eye(7)
    H[5, 5] = 0.0
    assert not oracle.scaled_logdet(H)[2]


def test_dkl_unit_invariance_and_sigma_shift(tiny_setup, oracle):
    """D_KL-hat with a uniform prior is unchanged when a parameter's unit changes (Sec. 3.3.3
    scaling), and doubling sigma lowers it by N_theta log 2."""
    w, G, th, H, Hr = tiny_setup
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    ld, _, _ = oracle.scaled_logdet(H)
    d0 = oracle.dkl(ld, 7, oracle.log_uniform_density(lo, hi))
    c = np.array([1e-3, 1.0, 1e3, 1.0, 1e-13, 1.0, 1.0])   # metres->km, s->ms, N m -> 1e13 N m
    Hc = H / np.outer(c, c)
    ldc, _, _ = oracle.scaled_logdet(Hc)
    d1 = oracle.dkl(ldc, 7, oracle.log_uniform_density(lo * c, hi * c))
    assert abs(d1 - d0) < 1e-9 * abs(d0)
    ld2, _, _ = oracle.scaled_logdet(H / 4)
    d2 = oracle.dkl(ld2, 7, oracle.log_uniform_density(lo, hi))
    assert abs((d0 - d2) - 7 * math.log(2)) < 1e-9


def test_linear_gaussian_closed_form(oracle):
    """For g(theta) = A theta with Gaussian prior N(0, P) and noise sigma^2 I the exact EIG is
    1/2 log det(I + P A^T A / sigma^2).  The Laplace estimate of Thm 4 (D_KL-hat averaged over
    the prior, with the Gaussian log-density as h) approaches it with error O(1/N)."""
    rng = np.random.default_rng(3)
    n = 7
    P = np.diag(rng.uniform(0.5, 2.0, n))
    Pinv = np.linalg.inv(P)
    gaps = []
    for N in (200, 800, 3200):
        A = rng.standard_normal((N, n))
        sigma = 1.0
        H = A.T @ A / sigma ** 2
        ld, _, ok = oracle.scaled_logdet(H)
        assert ok
        thetas = rng.multivariate_normal(np.zeros(n), P, size=400)
        logp = [-0.5 * (n * math.log(2 * math.pi) + math.log(np.linalg.det(P)) + t @ Pinv @ t)
                for t in thetas]
        lap = np.mean([oracle.dkl(ld, n, lp) for lp in logp])
        # the prior log-density averaged exactly: E[-h] = 1/2 log((2 pi e)^n det P)
        lap_exact_h = oracle.dkl(ld, n, -0.5 * (n * math.log(2 * math.pi * math.e) + math.log(np.linalg.det(P))))
        exact = 0.5 * np.linalg.slogdet(np.eye(n) + P @ A.T @ A / sigma ** 2)[1]
        assert abs(lap - lap_exact_h) < 0.1
        gaps.append(abs(lap_exact_h - exact))
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 0.02
    assert gaps[0] / gaps[2] > 8     # O(1/N): a factor 16 in N gives about 16


# ------------------------------------------------------------------ quadrature
def _golden_counts():
    rows = []
    with open(os.path.join(HERE, "golden", "smolyak_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, l, c = line.split()[:3]
                rows.append((int(d), int(l), int(c)))
    return rows


@pytest.mark.parametrize("dim,level,count", _golden_counts())
def test_smolyak_counts_match_paper(oracle, dim, level, count):
    x, w = oracle.smolyak(dim, level)
    assert len(x) == count
    assert abs(w.sum() - 1.0) < 1e-10


def test_smolyak_exact_on_total_degree_monomials(oracle):
    """Level-L Smolyak Gauss-Legendre integrates total-degree <= 2L+1 polynomials exactly
    (uniform measure on [-1, 1]^d: E[x^2] = 1/3, E[x^4] = 1/5, E[x^2 y^2] = 1/9)."""
    x, w = oracle.smolyak(7, 3)
    assert np.sum(w) == pytest.approx(1.0, abs=1e-12)
    assert np.sum(w * x[:, 0] ** 2) == pytest.approx(1 / 3, abs=1e-12)
    assert np.sum(w * x[:, 3] ** 4) == pytest.approx(1 / 5, abs=1e-12)
    assert np.sum(w * x[:, 1] ** 2 * x[:, 5] ** 2) == pytest.approx(1 / 9, abs=1e-12)
    assert np.sum(w * x[:, 2] ** 6) == pytest.approx(1 / 7, abs=1e-12)
    assert np.sum(w * x[:, 0] ** 3 * x[:, 4]) == pytest.approx(0.0, abs=1e-12)
    assert (w < 0).sum() == 99
    assert np.abs(w).sum() == pytest.approx(377.0, rel=1e-9)


def test_monte_carlo_nodes(oracle):
    w = W.plain_small()
    th, wt = oracle.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    assert th.shape == (16, 7) and np.allclose(wt, 1 / 16)
    assert np.all(th >= np.array(w.prior_lo)) and np.all(th <= np.array(w.prior_hi))


def _golden_cond():
    vals = {}
    with open(os.path.join(HERE, "golden", "scaled_hessian_cond.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_paper_model_conditioning_matches_sec_4_2(oracle):
    """The paper's worked example (Sec. 4.2): at the prior mean of its model problem,
    cond(H_1) = 3.88e30 and, after scaling by sqrt(diag H_1), 12.16.  The oracle reproduces
    both within 5% (central-FD and sensitivity Jacobians alike)."""
    gold = _golden_cond()
    w = W.paper_model()
    G = oracle.Grid.from_workload(w)
    mean = np.array(W.PAPER_PRIOR_MEAN)
    for H in (oracle.node_hessian(G, mean, w.prior_lo, w.prior_hi, w.rel_step, 0.01)[0],
              oracle.node_hessian_sensitivity(G, mean, 0.01)):
        S = np.sqrt(np.diag(H))
        assert abs(np.linalg.cond(H) / gold["cond_unscaled"] - 1) < 0.05
        assert abs(np.linalg.cond(H / np.outer(S, S)) / gold["cond_scaled"] - 1) < 0.05


def test_small_workload_scaled_hessian_conditioning(oracle):
    """Sec. 4.2: scaling by sqrt(diag H_1) brings cond from ~1e30 to O(10) (the paper prints
    3.88e30 and 12.16 for its own workload)."""
    w = W.plain_small()
    G = oracle.Grid.from_workload(w)
    th = (np.array(w.prior_lo) + np.array(w.prior_hi)) / 2
    H, _ = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step, 0.4)
    _, Ht, ok = oracle.scaled_logdet(H)
    assert ok
    assert np.linalg.cond(H) > 1e25
    assert 1.0 < np.linalg.cond(Ht) < 1e3


# ------------------------------------------------------------------ sensitivity solves (Alg. 1)
@pytest.mark.parametrize("alpha", [0.0, 0.21, 0.5, 0.88])
def test_delta_derivative_weights(oracle, alpha):
    """d/dx_s of the delta / delta' weights equals the central difference of the weights, and
    the derivative of the delta moments is the derivative of their exact values:
    d/dx_s sum h d_j (x_j - x_s)^q = 0 for every q gives sum h d'_j (x_j - x_s)^q = q [q = 1]."""
    h = 9.0
    dd, ddp = oracle.delta_weights_dxs(alpha, h)
    e = 1e-6
    dp_, dpp = oracle.delta_weights(alpha + e, h)
    dm_, dpm = oracle.delta_weights(alpha - e, h)
    assert np.allclose(dd, (dp_ - dm_) / (2 * e * h), rtol=1e-6, atol=1e-9 * np.abs(dd).max())
    assert np.allclose(ddp, (dpp - dpm) / (2 * e * h), rtol=1e-6, atol=1e-9 * np.abs(ddp).max())
    d, _ = oracle.delta_weights(alpha, h)
    xj = (np.arange(-2, 4) - alpha) * h
    for q in range(5):
        # d/dx_s [h sum d_j (x_j - x_s)^q] = h sum dd_j (x_j - x_s)^q - q h sum d_j (x_j - x_s)^(q-1) = 0
        lhs = h * np.sum(dd * xj ** q)
        rhs = q * h * np.sum(d * xj ** (q - 1)) if q > 0 else 0.0
        assert abs(lhs - rhs) < 1e-9 * max(1.0, h ** q)


def test_sensitivity_hessian_matches_fd_to_second_order(tiny_setup, oracle):
    """H_I from sensitivity solves (analytic df/dtheta, Alg. 1 steps 1-5) and the central-FD
    H_1 differ by O(d^2): small, and four times smaller at half the step."""
    w, G, th, H, Hr = tiny_setup
    Hs = oracle.node_hessian_sensitivity(G, th, 0.3)
    H2, _ = oracle.node_hessian(G, th, w.prior_lo, w.prior_hi, w.rel_step / 2, 0.3)
    d = np.sqrt(np.outer(np.diag(Hs), np.diag(Hs)))
    e1 = np.max(np.abs(H - Hs) / d)
    e2 = np.max(np.abs(H2 - Hs) / d)
    assert e1 < 1e-5
    assert 3.0 < e1 / e2 < 5.0
    assert np.allclose(Hs, Hs.T, rtol=1e-13, atol=0)


# ---------------------------------------------------- whole method vs definition
def test_laplace_eig_matches_the_definition_by_brute_force(oracle):
    """The Laplace EIG (Thm 4, Eq. DKL_hat, with H_1 from the central-FD Jacobian) against
    the expected information gain computed straight from its definition (Eq. expected_I)
    on a 41x21 grid with two free parameters, x_s (nonlinear) and m_xx (linear), the rest
    fixed, uniform prior on the box:
        I = E_{theta, eps}[ log p(y | theta) - log p(y) ],  y = g(theta) + eps,
        p(y) = (1 / |box|) int p(y | theta') dtheta'.
    The outer expectation is plain Monte Carlo (400 seeded draws of theta and eps); the
    inner evidence integral is a tensor trapezoid rule, 401 nodes in x_s (1 m apart, the
    posterior is about 4 m wide at sigma = 3) times 451 nodes in m_xx, using that g is
    linear in m_xx: g(x, m) = F(x) + m G(x), two solves per x node.  The noise variance
    of the outer average is reduced with a control variate of mean exactly zero:
    |P eps|^2 / (2 sigma^2) - d/2, P the projection onto the Jacobian's columns.
    Expected (concentration of measure, Sec. 4.4): agreement within a fraction of a
    percent when the posterior is narrow, a gap that grows as the noise widens it."""
    w = W.tiny(nsteps=120, nrec=4)
    G = oracle.Grid.from_workload(w)
    base = np.array([1010.0, 520.0, 0.2, 6.0, 4e13, 2e13, 6e13])
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    free = [0, 4]
    K, Jm_, N = 401, 451, 400

    def fwd(x, mxx, mxz, mzz):
        t = base.copy()
        t[0], t[4], t[5], t[6] = x, mxx, mxz, mzz
        return oracle.forward(G, t).ravel()

    xs, ms = np.linspace(lo[0], hi[0], K), np.linspace(lo[4], hi[4], Jm_)
    wx = np.full(K, (hi[0] - lo[0]) / (K - 1))
    wx[[0, -1]] *= 0.5
    wm = np.full(Jm_, (hi[4] - lo[4]) / (Jm_ - 1))
    wm[[0, -1]] *= 0.5
    Fk = np.array([fwd(x, 0.0, base[5], base[6]) for x in xs])
    Gk = np.array([fwd(x, 1.0, 0.0, 0.0) for x in xs])   # unit m_xx alone: no cancellation
    rng = np.random.default_rng(7)
    u = rng.random((N, 2))
    xn, mn = lo[0] + (hi[0] - lo[0]) * u[:, 0], lo[4] + (hi[4] - lo[4]) * u[:, 1]
    gn = np.array([fwd(xn[i], mn[i], base[5], base[6]) for i in range(N)])
    Z = rng.standard_normal(gn.shape)
    dx = 1e-4 * (hi[0] - lo[0])
    Jx = np.array([(fwd(xn[i] + dx, mn[i], base[5], base[6]) - fwd(xn[i] - dx, mn[i], base[5], base[6]))
                   / (2 * dx) for i in range(N)])
    Jmx = np.array([fwd(xn[i], 1.0, 0.0, 0.0) for i in range(N)])
    lp = oracle.log_uniform_density(lo[free], hi[free])
    D1 = np.empty(N)   # Laplace D_KL-hat of the two-parameter problem at sigma = 1
    for n in range(N):
        th = np.r_[xn[n], base[1:4], mn[n], base[5:]]
        H, _ = oracle.node_hessian(G, th, lo, hi, w.rel_step, 1.0)
        ld, _, ok = oracle.scaled_logdet(H)
        assert ok
        D1[n] = oracle.dkl(np.linalg.slogdet(H[np.ix_(free, free)])[1], 2, lp)
    vol = (hi[0] - lo[0]) * (hi[4] - lo[4])
    lw = np.log(wx)[:, None] + np.log(wm)[None, :]
    c = (Gk * Gk).sum(1)
    rel = {}
    for sigma in (1.0, 3.0, 10.0):
        E = sigma * Z
        Y = gn + E
        a = (Y * Y).sum(1)[:, None] + (Fk * Fk).sum(1)[None, :] - 2 * Y @ Fk.T   # |y - F_k|^2
        b = Y @ Gk.T - (Fk * Gk).sum(1)[None, :]                                # (y - F_k).G_k
        Dbf, cv = np.empty(N), np.empty(N)
        for n in range(N):
            q = a[n][:, None] - 2 * ms[None, :] * b[n][:, None] + (ms ** 2)[None, :] * c[:, None]
            z = -q / (2 * sigma ** 2) + lw
            zmax = z.max()
            log_py = zmax + math.log(np.exp(z - zmax).sum()) - math.log(vol)   # + const of p(y|.)
            Dbf[n] = -(E[n] @ E[n]) / (2 * sigma ** 2) - log_py
            Jn = np.stack([Jx[n], Jmx[n]], 1)
            Pe = Jn @ np.linalg.lstsq(Jn, E[n], rcond=None)[0]
            cv[n] = (Pe @ Pe) / (2 * sigma ** 2) - 1.0
        brute = Dbf + cv
        laplace = D1 - 2 * math.log(sigma)   # H_1 scales as sigma^-2
        gap = brute - laplace
        se = gap.std() / math.sqrt(N)
        # the control variate only removes noise: both averages agree within their errors
        assert abs(np.mean(cv)) < 4 * cv.std() / math.sqrt(N)
        assert abs(np.mean(Dbf) - np.mean(brute)) < 4 * Dbf.std() / math.sqrt(N)
        rel[sigma] = gap.mean() / brute.mean()
        assert se < 0.02 * abs(brute.mean())   # the comparison below is not lost in noise
    assert abs(rel[1.0]) < 0.005       # narrow posterior: a fraction of a percent
    assert abs(rel[3.0]) < 0.02
    assert abs(rel[10.0]) < 0.08       # the paper saw < 4% on its own problem
    assert rel[1.0] < rel[10.0]        # the gap grows as the posterior widens


def test_subset_logdet_matches_library_determinant(oracle):
    """Sec. 3.3.3's scaled log-det restricted to the unknown parameters of a subset (the known
    ones drop out, Sec. 4.3-4.4) against numpy's LU log-determinant of the sub-block."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        A = rng.standard_normal((7, 7)) * np.exp(rng.uniform(-12, 12, 7))[:, None]   # badly scaled
        H = A @ A.T
        k = int(rng.integers(1, 8))
        free = sorted(rng.choice(7, size=k, replace=False).tolist())
        ld, ok = oracle.scaled_logdet_sub(H, free)
        assert ok
        assert abs(ld - np.linalg.slogdet(H[np.ix_(free, free)])[1]) < 1e-8 * max(1.0, abs(ld))
    ld7, ok7 = oracle.scaled_logdet_sub(H, range(7))
    assert ok7 and abs(ld7 - oracle.scaled_logdet(H)[0]) < 1e-10 * abs(ld7)
    Hbad = np.eye(7)
    Hbad[1, 3] = Hbad[3, 1] = 1.5
    assert not oracle.scaled_logdet_sub(Hbad, [1, 3])[1]
    assert oracle.scaled_logdet_sub(Hbad, [1, 2])[1]


def test_dlmc_special_case_and_linear_gaussian_closed_form(oracle):
    """Double-loop Monte Carlo EIG (Eq. expected_I sampled directly, Sec. 4.4).
    (a) One inner sample equal to the outer one: the evidence is the likelihood itself and
        the estimate is exactly 0.
    (b) Linear map g = A theta, Gaussian prior N(0, P), noise sigma^2 I: the exact EIG is
        1/2 log det(I + P A^T A / sigma^2).  With independent inner samples the estimator's
        bias is positive and O(1/M) (Jensen: log of a mean underestimates the log evidence);
        at M = 4000 it sits within a few standard errors above the exact value, and a small M
        sits further above."""
    rng = np.random.default_rng(5)
    go = rng.standard_normal((6, 9))
    eps = 0.3 * rng.standard_normal((6, 9))
    for n in range(6):
        le, eig = oracle.dlmc(go[n:n + 1], eps[n:n + 1], go[n:n + 1], 0.3)
        assert abs(le[0] + (eps[n] @ eps[n]) / (2 * 0.09)) < 1e-12 and abs(eig) < 1e-12
    d, Ddat, sigma = 2, 12, 1.0
    A = 0.35 * rng.standard_normal((Ddat, d))
    P = np.diag([1.0, 0.6])
    exact = 0.5 * np.linalg.slogdet(np.eye(d) + P @ A.T @ A / sigma ** 2)[1]
    N = 3000

    def run(M, seed):
        r = np.random.default_rng(seed)
        th_o = r.multivariate_normal(np.zeros(d), P, size=N)
        th_i = r.multivariate_normal(np.zeros(d), P, size=M)
        e = sigma * r.standard_normal((N, Ddat))
        le, eig = oracle.dlmc(th_o @ A.T, e, th_i @ A.T, sigma)
        per = -(e * e).sum(1) / (2 * sigma ** 2) - le
        return eig, per.std() / math.sqrt(N)

    big, se = run(4000, 21)
    small, _ = run(8, 22)
    assert 0.3 < exact < 2.0
    assert -4 * se < big - exact < 4 * se + 0.02
    assert small - exact > big - exact + 2 * se


# ------------------------------------------------ H_II: dual solve (Alg. 1 steps 6-10)
@pytest.mark.parametrize("alpha", [0.0, 0.23, 0.5, 0.91])
def test_delta_second_derivative_weights(oracle, alpha):
    """d2/dx_s2 of the delta / delta' weights: central differences of the first derivatives,
    and the twice-differentiated moment conditions
    h sum d''_j (x_j - x_s)^q - 2 q h sum d'_j (x_j - x_s)^(q-1) + q (q-1) h sum d_j (x_j - x_s)^(q-2) = 0
    for delta (the moments are constants) and the same with q [q = 1] on the right for delta'
    replaced by 0 after two derivatives."""
    h = 7.0
    d2, dp2 = oracle.delta_weights_dxs2(alpha, h)
    e = 1e-6
    a1, b1 = oracle.delta_weights_dxs(alpha + e, h)
    a0, b0 = oracle.delta_weights_dxs(alpha - e, h)
    assert np.allclose(d2, (a1 - a0) / (2 * e * h), rtol=1e-6, atol=1e-9 * np.abs(d2).max())
    assert np.allclose(dp2, (b1 - b0) / (2 * e * h), rtol=1e-6, atol=1e-9 * np.abs(dp2).max())
    d, dp = oracle.delta_weights(alpha, h)
    d1, dp1 = oracle.delta_weights_dxs(alpha, h)
    xj = (np.arange(-2, 4) - alpha) * h
    for (w0, w1, w2) in ((d, d1, d2), (dp, dp1, dp2)):
        for q in range(5):
            t = h * np.sum(w2 * xj ** q)
            if q >= 1:
                t -= 2 * q * h * np.sum(w1 * xj ** (q - 1))
            if q >= 2:
                t += q * (q - 1) * h * np.sum(w0 * xj ** (q - 2))
            assert abs(t) < 1e-8 * max(1.0, h ** q) / h ** 2


def test_stf_derivatives_match_finite_differences(oracle):
    t, ts, ws = 0.37, 0.21, 6.3
    d = oracle.stf_derivs(t, ts, ws)
    e = 1e-5
    S = lambda a, b: oracle.stf(t, a, b)
    assert abs(d[0] - S(ts, ws)) < 1e-15
    assert abs(d[1] - (S(ts + e, ws) - S(ts - e, ws)) / (2 * e)) < 1e-7 * abs(d[1])
    assert abs(d[2] - (S(ts, ws + e) - S(ts, ws - e)) / (2 * e)) < 1e-7 * max(1, abs(d[2]))
    dd = lambda a, b: oracle.stf_derivs(t, a, b)
    assert abs(d[3] - (dd(ts + e, ws)[1] - dd(ts - e, ws)[1]) / (2 * e)) < 1e-6 * abs(d[3])
    assert abs(d[4] - (dd(ts, ws + e)[1] - dd(ts, ws - e)[1]) / (2 * e)) < 1e-6 * abs(d[4])
    assert abs(d[5] - (dd(ts, ws + e)[2] - dd(ts, ws - e)[2]) / (2 * e)) < 1e-6 * max(1, abs(d[5]))


@pytest.fixture(scope="module")
def adj_setup(oracle):
    w = W.tiny(nx=36, nz=19, h=50.0, nsteps=70, nrec=4,
               layers=((0.0, 2000.0, 1155.0, 2200.0), (400.0, 3000.0, 1732.0, 2500.0)))
    return w, oracle.Grid.from_workload(w)


def test_adjoint_is_the_transpose_of_the_scheme(adj_setup, oracle):
    """<w, G f> = <G^T w, f> for random forcing sequences and receiver weights (the dual
    problem, Eq. Dual_problems, is the exact transpose of the discrete scheme, free surface,
    layer interface and absorbing rows included)."""
    w, G = adj_setup
    rng = np.random.default_rng(8)
    for _ in range(2):
        f = rng.standard_normal((w.nsteps, 2, w.nz, w.nx))
        wt = rng.standard_normal((w.nsteps + 1, w.nrec, 2))
        lhs = float(np.sum(wt * oracle.forward_field(G, f)))
        rhs = float(np.sum(oracle.adjoint(G, wt) * f))
        assert abs(lhs - rhs) < 1e-11 * max(abs(lhs), 1.0)


def _theta_adj(w):
    return np.array([906.0, 431.0, 0.16, 6.4, 5e13, 3e13, 7e13])


def test_cost_gradient_from_dual_solve_equals_jacobian_transpose(adj_setup, oracle):
    """dL/dtheta = -J^T C^-1 r with J from the sensitivity solves (both exact derivatives of
    the discrete scheme, so they agree to rounding); zero residual gives zero H_II and
    gradient."""
    w, G = adj_setup
    th = _theta_adj(w)
    g = oracle.forward(G, th)
    rng = np.random.default_rng(2)
    sigma = 0.4
    y = g + sigma * rng.standard_normal(g.shape)
    H2, grad = oracle.hessian_ii(G, th, y, sigma)
    J = oracle.jacobian_sensitivity(G, th)
    wt = (y - g) / sigma ** 2
    ref = -np.array([np.sum(J[j] * wt) for j in range(7)])
    scale = np.sqrt(np.sum(J.reshape(7, -1) ** 2, 1)) * np.sqrt(np.sum(wt ** 2))
    assert np.all(np.abs(grad - ref) <= 1e-10 * scale)
    assert np.allclose(H2, H2.T, rtol=0, atol=0)
    H0, g0 = oracle.hessian_ii(G, th, g, sigma)
    assert np.all(H0 == 0.0) and np.all(g0 == 0.0)


def test_hessian_ii_equals_curvature_of_the_seismograms(adj_setup, oracle):
    """H_II = -sum w . d2 g / dtheta_a dtheta_b (Thm 2's H_2) against central differences of
    the sensitivity Jacobian: O(d^2), four times smaller at half the step, in every entry
    scaled by sqrt(|H_aa H_bb|) of the Gauss-Newton part."""
    w, G = adj_setup
    th = _theta_adj(w)
    g = oracle.forward(G, th)
    rng = np.random.default_rng(4)
    sigma = 0.4
    y = g + sigma * rng.standard_normal(g.shape)
    H2, _ = oracle.hessian_ii(G, th, y, sigma)
    wt = (y - g) / sigma ** 2
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)

    def fd(rel):
        out = np.zeros((7, 7))
        for b in range(7):
            d = rel * (hi[b] - lo[b])
            tp, tm = th.copy(), th.copy()
            tp[b] += d
            tm[b] -= d
            Jp, Jm = oracle.jacobian_sensitivity(G, tp), oracle.jacobian_sensitivity(G, tm)
            for a in range(7):
                out[a, b] = -np.sum((Jp[a] - Jm[a]) * wt) / (2 * d)
        return out

    H1 = oracle.node_hessian_sensitivity(G, th, sigma)
    sc = np.sqrt(np.outer(np.diag(H1), np.diag(H1)))
    e1 = np.max(np.abs(fd(2e-3) - H2) / sc)
    e2 = np.max(np.abs(fd(1e-3) - H2) / sc)
    assert e1 < 1e-4 and e2 < e1 / 3.0
    assert np.max(np.abs(H2) / sc) > 1e-3   # the check is not vacuous


# ------------------------------------------------------------------ Ricker time function
def test_ricker_closed_forms(oracle):
    """The optional Ricker wavelet: value 1 at t_s, zeros at |t - t_s| = 1/(pi f sqrt 2),
    zero mean, and equal to minus the second time derivative of the paper's Gaussian
    (omega_s = pi f sqrt 2) divided by its curvature 2 pi^2 f^2 and normalisation."""
    ts, f = 0.21, 7.5
    assert oracle.ricker(ts, ts, f) == 1.0
    z = 1.0 / (math.pi * f * math.sqrt(2.0))
    for s in (-1.0, 1.0):
        assert abs(oracle.ricker(ts + s * z, ts, f)) < 1e-15
        assert oracle.ricker(ts + s * 0.9 * z, ts, f) > 0 > oracle.ricker(ts + s * 1.1 * z, ts, f)
    t = np.linspace(ts - 2.0, ts + 2.0, 40001)
    r = np.array([oracle.ricker(x, ts, f) for x in t])
    assert abs(np.trapezoid(r, t)) < 1e-12
    ws = math.pi * f * math.sqrt(2.0)
    for x in (ts - 0.13, ts - 0.02, ts + 0.05, ts + 0.31):
        S_tt = oracle.stf_derivs(x, ts, ws)[3]
        ref = -S_tt * math.sqrt(2.0 * math.pi) / ws / (2.0 * math.pi ** 2 * f * f)
        assert abs(oracle.ricker(x, ts, f) - ref) < 1e-13


def test_forward_with_either_time_function_is_the_forward_of_its_forcing(oracle):
    """forward(theta, stf) equals the solve driven by the explicit forcing sequence
    S(t_m) f_patch (Eq. source, the time function of the chosen kind), bit for bit."""
    w = W.tiny(nx=40, nz=24, h=50.0, nsteps=60, nrec=3)
    G = oracle.Grid.from_workload(w)
    th = np.array([1010.0, 560.0, 0.12, 7.0, 5e13, 3e13, 7e13])
    i0, j0, px, pz, ok = oracle.source_patch(th, w.nx, w.nz, w.h)
    assert ok
    for kind, fn in ((oracle.STF_GAUSS, oracle.stf), (oracle.STF_RICKER, oracle.ricker)):
        f = np.zeros((w.nsteps, 2, w.nz, w.nx))
        for m in range(w.nsteps):
            s = fn(m * w.dt, th[2], th[3])
            f[m, 0, j0:j0 + 6, i0:i0 + 6] = s * px
            f[m, 1, j0:j0 + 6, i0:i0 + 6] = s * pz
        g = oracle.forward(G, th, stf=kind)
        assert np.max(np.abs(g)) > 0
        assert np.array_equal(g, oracle.forward_field(G, f))
    assert not np.allclose(oracle.forward(G, th, stf=oracle.STF_RICKER), oracle.forward(G, th))


# ------------------------------------------------------------------ media (Sec. 2.1)
def test_media_recover_the_wave_speeds_and_the_interface_rule(oracle):
    """The Lame parameters the oracle builds give back the layer's wave speeds through
    c_p = sqrt((lambda + 2 mu)/rho) and c_s = sqrt(mu/rho) (Sec. 2.1), and a node lying
    exactly on an interface takes the deeper layer (the reading both sides use)."""
    h = 25.0
    layers = ((0.0, 2000.0, 1155.0, 2200.0), (300.0, 3000.0, 1732.0, 2500.0), (612.5, 4500.0, 2598.0, 2700.0))
    G = oracle.Grid(9, 40, h, 1e-3, 1, layers, [0])
    lam, mu, nu = (a.reshape(40, 9) for a in (G.lam, G.mu, G.nu))
    for j in range(40):
        z = j * h
        expect = 0 if z < 300.0 else (1 if z < 612.5 else 2)
        _, vp, vs, rho = layers[expect]
        assert np.all(np.abs(np.sqrt((lam[j] + 2 * mu[j]) / nu[j]) - vp) < 1e-9 * vp)
        assert np.all(np.abs(np.sqrt(mu[j] / nu[j]) - vs) < 1e-9 * vs)
        assert np.all(nu[j] == rho)
    assert nu[12, 0] == 2500.0 and nu[11, 0] == 2200.0   # z = 300 m sits on the interface
    assert nu[24, 0] == 2500.0 and nu[25, 0] == 2700.0   # 612.5 m lies between nodes 24 and 25


def test_p_waves_travel_at_the_p_speed(oracle):
    """An explosive source (m_xx = m_zz, m_xz = 0) radiates P waves only; their onset at
    two surface receivers 800 m and 1000 m from the source is separated by the P travel
    time of the 200 m difference, 200 / c_p (grid dispersion is negligible at 30 nodes per
    wavelength), and the near onset precedes t_s + 800 / c_p by at most the pulse's
    half-width.  A slip in the Lame parameters or in the operator's (lambda + 2 mu) terms
    changes the speed by far more than the two-step tolerance."""
    h, vp, vs, rho = 10.0, 3000.0, 1732.0, 2500.0
    dt = 0.5 * h / vp
    nsteps = int(0.5 / dt)
    G = oracle.Grid(201, 121, h, dt, nsteps, ((0.0, vp, vs, rho),), [100, 160])
    ts, om = 0.1, 60.0
    g = oracle.forward(G, [1000.0, 800.0, ts, om, 1e13, 0.0, 1e13])
    t = np.arange(nsteps + 1) * dt
    onset = []
    for r in range(2):
        u = np.hypot(g[:, r, 0], g[:, r, 1])
        onset.append(t[np.argmax(u > 0.05 * u.max())])
    assert abs((onset[1] - onset[0]) - 200.0 / vp) <= 2 * dt
    assert ts + 800.0 / vp - 4.0 / om <= onset[0] <= ts + 800.0 / vp
    assert np.max(np.abs(g[:, 0, 0])) == 0.0   # the receiver above the source: u_x = 0 by symmetry


def test_s_waves_travel_at_the_s_speed(oracle):
    """A shear source (m_xz only) radiates no P wave straight up; the strongest motion at
    the receiver above it is the S pulse, peaking within a pulse half-width (1/omega_s) of
    t_s + 800 / c_s.  Checked for two shear speeds, so a slip in mu or in the mu terms of
    the operator moves the peak by more than the tolerance."""
    h, vp, rho = 10.0, 3000.0, 2500.0
    dt = 0.5 * h / vp
    nsteps = int(0.75 / dt)
    ts, om = 0.1, 60.0
    t = np.arange(nsteps + 1) * dt
    for vs in (1732.0, 1500.0):
        G = oracle.Grid(201, 121, h, dt, nsteps, ((0.0, vp, vs, rho),), [100])
        g = oracle.forward(G, [1000.0, 800.0, ts, om, 0.0, 1e13, 0.0])
        u = np.hypot(g[:, 0, 0], g[:, 0, 1])
        assert abs(t[np.argmax(u)] - (ts + 800.0 / vs)) < 1.0 / om, vs


def _rayleigh_speed(vp, vs):
    """Root of the Rayleigh equation (2 - x)^2 = 4 sqrt(1 - x) sqrt(1 - x vs^2/vp^2), x = (c/vs)^2."""
    k = (vs / vp) ** 2
    f = lambda x: (2 - x) ** 2 - 4 * math.sqrt(1 - x) * math.sqrt(1 - x * k)
    lo, hi = 0.5, 0.999
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return vs * math.sqrt(0.5 * (lo + hi))


def test_free_surface_carries_rayleigh_waves_at_the_rayleigh_speed(oracle):
    """A shallow explosive source under the free surface of a Poisson solid (lambda = mu)
    sends a Rayleigh pulse along it; the lag that best aligns u_z at surface receivers 600 m
    and 1000 m away (cross-correlation, parabolic refinement) gives its speed, which must
    be the root of the Rayleigh equation, c_R = 0.9194 c_s, within 1% at h = 10 m (0.35%
    measured, 0.02% at 5 m), and not c_s.  This pins the traction-free closure of the
    surface row against a textbook closed form."""
    h, vp, vs, rho = 10.0, 3000.0, 1732.0, 2500.0
    cR = _rayleigh_speed(vp, vs)
    assert abs(cR / vs - 0.9194) < 1e-3
    dt = 0.5 * h / vp
    nsteps = int(1.0 / dt)
    G = oracle.Grid(261, 81, h, dt, nsteps, ((0.0, vp, vs, rho),), [110, 150])
    g = oracle.forward(G, [500.0, 40.0, 0.1, 60.0, 1e13, 0.0, 1e13])
    a, b = g[:, 0, 1], g[:, 1, 1]
    c = np.correlate(b, a, mode="full")[len(a) - 1:]
    k = int(np.argmax(c))
    lag = (k + 0.5 * (c[k - 1] - c[k + 1]) / (c[k - 1] - 2 * c[k] + c[k + 1])) * dt
    speed = 400.0 / lag
    assert abs(speed / cR - 1) < 0.01, (speed, cR)
    assert abs(speed / vs - 1) > 0.05


def test_layer_interface_reflects_with_the_impedance_contrast(oracle):
    """A plane P pulse (a line force f_z along a whole row, 200 m deep) meets a welded
    interface at 600 m; at the surface the particle velocity of the reflected pulse over
    that of the direct one is the normal-incidence displacement reflection coefficient
    (Z1 - Z2) / (Z1 + Z2), Z = rho c_p (both pulses are doubled alike by the free surface),
    to 5% (1.1% measured with 25 nodes per wavelength); the reflection arrives after the
    1000 m two-way path to within one node spacing (the interface node belongs to the
    deeper layer)."""
    h = 20.0
    l1, l2 = (0.0, 3000.0, 1732.0, 2500.0), (600.0, 4500.0, 2598.0, 2700.0)
    nx, nz = 201, 61
    dt = 0.5 * h / l2[1]
    nsteps = int(0.55 / dt)
    G = oracle.Grid(nx, nz, h, dt, nsteps, (l1, l2), [100])
    om, ts = 40.0, 0.12
    f = np.zeros((nsteps, 2, nz, nx))
    for m in range(nsteps):
        f[m, 1, 10, :] = oracle.stf(m * dt, ts, om)
    uz = oracle.forward_field(G, f)[:, 0, 1]
    v = np.diff(uz) / dt
    t = (np.arange(nsteps) + 0.5) * dt
    w = 3.0 / om

    def pulse(t_expect):
        sel = (t > t_expect - w) & (t < t_expect + w)
        k = np.argmax(np.abs(v[sel]))
        return v[sel][k], t[sel][k]

    vd, td = pulse(ts + 200.0 / l1[1])
    vr, tr = pulse(ts + 1000.0 / l1[1])
    Z1, Z2 = l1[3] * l1[1], l2[3] * l2[1]
    R = (Z1 - Z2) / (Z1 + Z2)
    assert abs(vr / vd - R) < 0.05 * abs(R), (vr / vd, R)
    assert abs(td - (ts + 200.0 / l1[1])) < 2 * dt
    assert abs(tr - (ts + 1000.0 / l1[1])) < h / l1[1] + 2 * dt


def test_absorbing_bottom_passes_a_normally_incident_pulse(oracle):
    """The first-order absorbing bottom row is exact for normal incidence in the continuum;
    a plane P pulse (line force along a row) that reaches it returns to the surface with
    under 5% of the direct pulse's particle velocity (2.2% measured at 25 nodes per
    wavelength).  Taking c_s for the normal component there would reflect (c_p - c_s) /
    (c_p + c_s) = 27%."""
    h = 20.0
    layer = (0.0, 3000.0, 1732.0, 2500.0)
    nx, nz = 201, 31   # bottom row at 600 m
    dt = 0.5 * h / layer[1]
    nsteps = int(0.6 / dt)
    G = oracle.Grid(nx, nz, h, dt, nsteps, (layer,), [100])
    om, ts = 40.0, 0.12
    f = np.zeros((nsteps, 2, nz, nx))
    for m in range(nsteps):
        f[m, 1, 10, :] = oracle.stf(m * dt, ts, om)
    uz = oracle.forward_field(G, f)[:, 0, 1]
    v = np.diff(uz) / dt
    t = (np.arange(nsteps) + 0.5) * dt
    w = 3.0 / om
    direct = np.max(np.abs(v[(t > ts + 200 / 3000.0 - w) & (t < ts + 200 / 3000.0 + w)]))
    back = np.max(np.abs(v[(t > ts + 1000 / 3000.0 - w) & (t < ts + 1000 / 3000.0 + w)]))
    assert back < 0.05 * direct, back / direct
