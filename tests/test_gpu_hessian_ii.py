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
