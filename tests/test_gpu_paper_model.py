"""The paper's own model problem (Sec. 4.1) and experiments (Sec. 4.2, Sec. 4.5) on the GPU.

Two-layer box, h = 200 m, dt = 0.025 s, T = 8 s, C_eps = 1e-4 I; per-receiver partial
Hessians over the 91 candidate surface nodes from sensitivity solves (Alg. 1 steps 1-5),
FP32 stencil.  Checks: H_1 at the prior mean against the oracle and the conditioning the
paper prints (3.88e30 -> 12.16); the shape of Scenarios I-III: EIG grows with the number
of receivers on a fixed aperture (I) and at fixed spacing (II), and a five-receiver array
has an interior optimum spacing on a flat top, 1000 .. 1800 m, with the paper's 1000 m
within 0.3% of the best (III).
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def test_prior_mean_hessian_and_conditioning(P, oracle):
    w = W.paper_model()
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    mean = np.array([W.PAPER_PRIOR_MEAN])
    H = torch.empty((1, 7, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, torch.tensor(mean, device=DEV), w.prior_lo, w.prior_hi, w.rel_step, 0.01, H)
    Hg = H[0].cpu().numpy()
    Href = oracle.node_hessian_sensitivity(oracle.Grid.from_workload(w), mean[0], 0.01)
    d = np.sqrt(np.outer(np.diag(Href), np.diag(Href)))
    assert np.max(np.abs(Hg - Href) / d) < 1e-4
    S = np.sqrt(np.diag(Hg))
    assert 3.5e30 < np.linalg.cond(Hg) < 4.2e30          # paper: 3.88e30
    assert 11.5 < np.linalg.cond(Hg / np.outer(S, S)) < 12.8   # paper: 12.16


def test_scenarios_shape(P):
    w = W.paper_model()
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    n = 1024
    th = lo + (hi - lo) * np.random.default_rng(6).random((n, 7))
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * n)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=DEV)
    Hr = torch.empty((n, w.nrec, 1, 28), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, torch.tensor(th, device=DEV), w.prior_lo, w.prior_hi, w.rel_step, 0.01, H,
                  win_levels=[w.nlevels], H_rec=Hr)
    scen = W.paper_scenarios()
    masks = torch.tensor(np.stack([m for _, _, m in scen]), device=DEV)
    eig = torch.empty(len(scen), dtype=torch.float64, device=DEV)
    nb = torch.empty(len(scen), dtype=torch.int32, device=DEV)
    P.oed_eig_designs(ctx, Hr, 0, masks, torch.full((n,), 1.0 / n, dtype=torch.float64, device=DEV),
                      w.prior_lo, w.prior_hi, eig, n_bad=nb)
    e = eig.cpu().numpy()
    assert not nb.cpu().numpy().any()
    by = {}
    for k, (sc, v, _) in enumerate(scen):
        by.setdefault(sc, []).append((v, e[k]))
    s1 = [x for _, x in by["I"]]
    s2 = [x for _, x in by["II"]]
    s3 = by["III"]
    assert all(np.diff(s1) > 0) and all(np.diff(s2) > 0)
    # diminishing returns in Scenario I beyond ~17-20 receivers
    assert (s1[3] - s1[2]) / 8 > (s1[5] - s1[4]) / 40
    # Scenario III: an interior optimum on a flat top.  On this model the sparse grid of
    # 8583 nodes and 10^4 Monte Carlo nodes both put it at 1400 m, with the paper's 1000 m
    # within 0.15% of the maximum and every spacing in 1000 .. 1800 m within 0.2%; the
    # array of 200 m (too short) and 4000 m (too wide) spacing are clearly below
    best, top = max(s3, key=lambda t: t[1])
    assert 1000 <= best <= 1800, s3                      # paper: 1000 m
    at = dict(s3)
    assert at[1000] >= top * (1 - 3e-3), s3
    assert at[200] < top * (1 - 1e-2) and at[4000] < top * (1 - 1e-2), s3
    # the union of candidates at fixed spacing 1000 m: Scenario I (17 receivers, 1000 m)
    # and Scenario II (17 receivers) are the same design
    assert by["I"][3][1] == pytest.approx(by["II"][8][1], rel=1e-12)
