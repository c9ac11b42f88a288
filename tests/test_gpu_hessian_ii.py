"""Parity of H_II from the dual solve (Alg. 1 steps 6-10) and of the Newton estimate of
Thm 1 with the FP64 oracle, through the C ABI.

Tolerances: FP64 stencil, H_II and the cost gradient to 1e-9 of the scale of the
Gauss-Newton part (|H_II - H_II,ref|_ab / sqrt(H1_aa H1_bb), |grad - ref|_a / sqrt(H1_aa)
times the residual norm); the FP32 stencil's residual carries its seismogram error
(1e-4 normwise) divided by sigma, so there the bar is 2e-3 of that scale."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
LAYERS2 = ((0.0, 2000.0, 1155.0, 2200.0), (400.0, 3000.0, 1732.0, 2500.0))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _case():
    w = W.tiny(nx=36, nz=19, h=50.0, nsteps=70, nrec=4, layers=LAYERS2)
    th = np.array([[906.0, 431.0, 0.16, 6.4, 5e13, 3e13, 7e13],
                   [1111.0, 150.0, 0.21, 5.1, 2e13, 9e13, 4e13],    # patch reaches the surface row
                   [802.0, 577.0, 0.11, 7.7, 8e13, 1e13, 1e13]])
    return w, th


@pytest.mark.parametrize("prec,tol", [(1, 1e-9), (0, 2e-3)])
def test_hessian_ii_and_gradient_match_oracle(P, oracle, prec, tol):
    w, th = _case()
    G = oracle.Grid.from_workload(w)
    rng = np.random.default_rng(12)
    sigma = 0.4
    n = th.shape[0]
    ys = np.array([oracle.forward(G, t) + sigma * rng.standard_normal((w.nlevels, w.nrec, 2)) for t in th])
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=2)   # two chunks
    H = torch.zeros((n, 7, 7), dtype=torch.float64, device=DEV)
    gr = torch.empty((n, 7), dtype=torch.float64, device=DEV)
    st = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    P.oed_hessian_ii(ctx, _t(th), _t(ys), sigma, H, grad=gr, status=st)
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [0] * n
    for k in range(n):
        H2, g2 = oracle.hessian_ii(G, th[k], ys[k], sigma)
        H1 = oracle.node_hessian_sensitivity(G, th[k], sigma)
        d = np.sqrt(np.diag(H1))
        assert np.max(np.abs(H[k].cpu().numpy() - H2) / np.outer(d, d)) <= tol, k
        rnorm = np.sqrt(np.sum((ys[k] - oracle.forward(G, th[k])) ** 2)) / sigma
        assert np.max(np.abs(gr[k].cpu().numpy() - g2) / (d * rnorm)) <= tol, k
        assert np.max(np.abs(H2) / np.outer(d, d)) > 1e-4   # not vacuous


def test_hessian_ii_is_added_and_vanishes_for_zero_residual(P):
    w, th = _case()
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=8)
    n = th.shape[0]
    g = torch.empty((n, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    H0 = torch.randn((n, 7, 7), dtype=torch.float64, device=DEV)
    H = H0.clone()
    gr = torch.empty((n, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian_ii(ctx, _t(th), g, 0.3, H, grad=gr)
    torch.cuda.synchronize()
    assert torch.equal(H, H0)
    assert torch.all(gr == 0)


def test_invalid_source_gives_nan_and_status(P):
    w, th = _case()
    th = th.copy()
    th[1, 1] = 20.0   # depth 20 m: the patch leaves the grid through the surface
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=8)
    y = torch.zeros((3, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    H = torch.zeros((3, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.empty(3, dtype=torch.int32, device=DEV)
    P.oed_hessian_ii(ctx, _t(th), y, 0.3, H, status=st)
    assert st.cpu().tolist() == [0, P.OED_EINVAL, 0]
    assert torch.isnan(H[1]).all() and not torch.isnan(H[0]).any()


def test_newton_estimate_and_thm3_hessian(P, oracle):
    """Newton iterations from theta* on data y = g(theta*) + eps reach a stationary point of
    the cost (Newton decrement grad^T H^-1 grad << 1) near theta* (Thm 1: O(N^-1/2)), and
    H = H_1 + H_II there matches the oracle's at the same point."""
    w, _ = _case()
    th = np.array([[906.0, 431.0, 0.16, 6.4, 5e13, 3e13, 7e13],
                   [1080.0, 540.0, 0.24, 5.3, 2.5e13, 8e13, 4e13]])   # inside the prior box
    G = oracle.Grid.from_workload(w)
    rng = np.random.default_rng(3)
    sigma = 0.4
    n = th.shape[0]
    ys = np.array([oracle.forward(G, t) + sigma * rng.standard_normal((w.nlevels, w.nrec, 2)) for t in th])
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=14)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    theta = _t(th)
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=DEV)
    gr = torch.empty((n, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian_map(ctx, theta, _t(ys), w.prior_lo, w.prior_hi, w.rel_step, sigma, 4, H, gr)
    torch.cuda.synchronize()
    thh, Hn, gn = theta.cpu().numpy(), H.cpu().numpy(), gr.cpu().numpy()
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    for k in range(n):
        dec = float(gn[k] @ np.linalg.solve(Hn[k], gn[k]))
        assert dec < 1e-8, (k, dec)
        H1 = oracle.node_hessian_sensitivity(G, thh[k], sigma)
        sd = np.sqrt(np.diag(np.linalg.inv(H1)))
        assert np.all(np.abs(thh[k] - th[k]) < 6 * sd + 1e-12 * (hi - lo)), k   # O(N^-1/2)
        H2, _ = oracle.hessian_ii(G, thh[k], ys[k], sigma)
        d = np.sqrt(np.diag(H1))
        assert np.max(np.abs(Hn[k] - (H1 + H2)) / np.outer(d, d)) <= 1e-8, k


def test_thm3_gain_against_the_definition(P, oracle):
    """Thm 3 (H_1 + H_II at the Newton estimate on the data) and Thm 4 (H_1 at theta*) against
    the EIG computed by brute force from its definition, on the problem of the oracle pin
    (41x21 grid, x_s and m_xx unknown, the rest known; the same outer samples (theta*, eps),
    the evidence integral by a tensor trapezoid rule, the zero-mean control variate
    |P eps|^2 / (2 sigma^2) - d/2 on the brute-force side).  With a narrow posterior
    (sigma = 1, 3) all three agree to a fraction of a percent (nodes whose H_1 + H_II is not
    positive definite are left out of Thm 3's mean, as the EIG kernels do); the numbers at
    sigma = 10 are printed (there H_1 + H_II is indefinite at ~9% of the estimates and the
    box truncates the posterior, where neither asymptotic form applies)."""
    import math
    w = W.tiny(nsteps=120, nrec=4)
    G = oracle.Grid.from_workload(w)
    base = np.array([1010.0, 520.0, 0.2, 6.0, 4e13, 2e13, 6e13])
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    free = [0, 4]
    K, Jm_, N = 401, 451, 256

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
    Gk = np.array([fwd(x, 1.0, 0.0, 0.0) for x in xs])
    rng = np.random.default_rng(7)
    u = rng.random((N, 2))
    xn, mn = lo[0] + (hi[0] - lo[0]) * u[:, 0], lo[4] + (hi[4] - lo[4]) * u[:, 1]
    thn = np.tile(base, (N, 1))
    thn[:, 0], thn[:, 4] = xn, mn
    gn = np.array([fwd(xn[i], mn[i], base[5], base[6]) for i in range(N)])
    dx = 1e-4 * (hi[0] - lo[0])
    Jx = np.array([(fwd(xn[i] + dx, mn[i], base[5], base[6]) - fwd(xn[i] - dx, mn[i], base[5], base[6]))
                   / (2 * dx) for i in range(N)])
    Jmx = np.array([fwd(xn[i], 1.0, 0.0, 0.0) for i in range(N)])
    Z = rng.standard_normal(gn.shape)
    vol = (hi[0] - lo[0]) * (hi[4] - lo[4])
    lw = np.log(wx)[:, None] + np.log(wm)[None, :]
    c = (Gk * Gk).sum(1)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=7 * 64)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    wts = _t(np.full(N, 1.0 / N))
    res = {}
    for sigma in (1.0, 3.0, 10.0):
        E = sigma * Z
        Y = gn + E
        a = (Y * Y).sum(1)[:, None] + (Fk * Fk).sum(1)[None, :] - 2 * Y @ Fk.T
        b = Y @ Gk.T - (Fk * Gk).sum(1)[None, :]
        brute = np.empty(N)
        for n in range(N):
            q = a[n][:, None] - 2 * ms[None, :] * b[n][:, None] + (ms ** 2)[None, :] * c[:, None]
            z = -q / (2 * sigma ** 2) + lw
            zmax = z.max()
            brute[n] = -(E[n] @ E[n]) / (2 * sigma ** 2) - (zmax + math.log(np.exp(z - zmax).sum()) - math.log(vol))
            Jn = np.stack([Jx[n], Jmx[n]], 1)
            Pe = Jn @ np.linalg.lstsq(Jn, E[n], rcond=None)[0]
            brute[n] += (Pe @ Pe) / (2 * sigma ** 2) - 1.0
        H = torch.empty((N, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, _t(thn), w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
        d4 = torch.empty(N, dtype=torch.float64, device=DEV)
        e4 = torch.empty(1, dtype=torch.float64, device=DEV)
        P.oed_eig_subset(ctx, H, wts, w.prior_lo, w.prior_hi, free, e4, dkl=d4)
        theta = _t(thn)
        gr = torch.empty((N, 7), dtype=torch.float64, device=DEV)
        ys = _t(Y.reshape(N, w.nlevels, w.nrec, 2))
        P.oed_hessian_map(ctx, theta, ys, w.prior_lo, w.prior_hi, w.rel_step, sigma, 4, H, gr, free=free)
        d3 = torch.empty(N, dtype=torch.float64, device=DEV)
        e3 = torch.empty(1, dtype=torch.float64, device=DEV)
        st3 = torch.empty(N, dtype=torch.int32, device=DEV)
        P.oed_eig_subset(ctx, H, wts, w.prior_lo, w.prior_hi, free, e3, dkl=d3, status=st3)
        torch.cuda.synchronize()
        ok = st3.cpu().numpy() == 0
        g3 = brute[ok] - d3.cpu().numpy()[ok]
        g4 = brute - d4.cpu().numpy()
        res[sigma] = dict(brute=brute.mean(), thm4=float(d4.cpu().numpy().mean()),
                          thm3=float(d3.cpu().numpy()[ok].mean()), gap4=g4.mean(), se4=g4.std() / math.sqrt(N),
                          gap3=g3.mean(), se3=g3.std() / math.sqrt(ok.sum()), not_pd=int((~ok).sum()))
    print(res)
    for sg in (1.0, 3.0):
        r = res[sg]
        assert r["not_pd"] <= N // 100   # an estimate at the box edge can leave H_1 + H_II indefinite
        for gap, se in ((r["gap4"], r["se4"]), (r["gap3"], r["se3"])):
            assert abs(gap) < max(4 * se, 0.005 * r["brute"]) and abs(gap) < 0.015 * r["brute"], (sg, r)


def test_hessian_ii_paper_model_one_node(P, oracle):
    """H_II and the gradient at the scale of the paper's model problem (101x76, two layers,
    T = 1.25 s, two receivers, sigma = 0.01) against the oracle at one node, FP64."""
    w = W.paper_study_model()
    G = oracle.Grid.from_workload(w)
    th = W.paper_study_thetas(np.random.default_rng(45).random((1, 3)))
    sigma = 0.01
    y = oracle.forward(G, th[0]) + sigma * np.random.default_rng(0).standard_normal((w.nlevels, w.nrec, 2))
    H2, g2 = oracle.hessian_ii(G, th[0], y, sigma)
    H1 = oracle.node_hessian_sensitivity(G, th[0], sigma)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=4)
    H = torch.zeros((1, 7, 7), dtype=torch.float64, device=DEV)
    gr = torch.empty((1, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian_ii(ctx, _t(th), _t(y[None]), sigma, H, grad=gr)
    torch.cuda.synchronize()
    d = np.sqrt(np.diag(H1))
    assert np.max(np.abs(H[0].cpu().numpy() - H2) / np.outer(d, d)) <= 1e-9
    rnorm = np.sqrt(np.sum((y - oracle.forward(G, th[0])) ** 2)) / sigma
    assert np.max(np.abs(gr[0].cpu().numpy() - g2) / (d * rnorm)) <= 1e-9
