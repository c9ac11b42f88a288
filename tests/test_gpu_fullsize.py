"""Full-size workloads, sampled against the oracle (GPU, slow).

- Layered medium: 801x401 grid (h = 2.5 m), 3 layers, 4000 steps, 40 receivers, level-3
  Smolyak rule (589 nodes): the streaming kernel (the grid does not fit on chip) in the
  launch configuration of a full run; sampled nodes' D_KL-hat against the oracle; the
  node rule against the oracle's.
- Design sweep: 401x201 grid to T = 2 s (2400 steps), 40 candidate receivers, windows
  T = 0.5 / 1 / 2 s, per-receiver partial Hessians of 1024 MC nodes, EIG of 512 seeded
  subsets for every k = 1..10: sampled partial Hessians against the oracle, the sweep's
  arithmetic against the oracle's log-det on the same partial Hessians, and growth of
  EIG with receiver count and measurement time.
FP32 stencil with the difference-form Jacobian (the FP32 precision path).
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def test_layered_smolyak_sampled(P, oracle):
    w = W.layered()
    x, wt = P.oed_nodes_smolyak(7, w.smolyak_level, w.prior_lo, w.prior_hi)
    xo, wo = oracle.smolyak(7, w.smolyak_level, w.prior_lo, w.prior_hi)
    assert x.shape == (589, 7) and np.allclose(x, xo, rtol=1e-13) and np.allclose(wt, wo, atol=1e-11)
    sigma = 0.2
    sample = [0, 294, 588]   # first, middle (the prior mean) and last node
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * 64)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    assert ctx.resident_min_cluster == 0       # 801x401 does not fit on chip
    ctx.autotune(7 * 64)
    H = torch.empty((len(sample), 7, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(x[sample]), w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
    dkl = torch.empty(len(sample), dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(np.full(len(sample), 1.0)), w.prior_lo, w.prior_hi, eig, dkl=dkl)
    G = oracle.Grid.from_workload(w)
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    for k, i in enumerate(sample[:2]):
        Href, _ = oracle.node_hessian(G, x[i], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, ok = oracle.scaled_logdet(Href)
        d_ref = oracle.dkl(ld, 7, lp)
        assert abs(float(dkl[k].item()) - d_ref) <= 1e-4 * abs(d_ref), (i, float(dkl[k].item()), d_ref)


def test_design_sweep_sampled(P, oracle):
    w = W.design_sweep()
    wl = w.win_levels()
    assert wl == [601, 1201, 2401]
    th, wt = oracle.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    sigma = 0.3
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * 1024)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    ctx.autotune(7 * 1024)
    n = w.n_nodes
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=DEV)
    Hr = torch.empty((n, w.nrec, 3, 28), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=wl, H_rec=Hr)
    masks = W.design_subsets(w.nrec, 10, 512, seed=w.seed)
    eig = torch.empty((3, masks.shape[0]), dtype=torch.float64, device=DEV)
    nb = torch.empty((3, masks.shape[0]), dtype=torch.int32, device=DEV)
    m_t = _t(masks, torch.uint8)
    w_t = _t(wt)
    for win in range(3):
        P.oed_eig_designs(ctx, Hr, win, m_t, w_t, w.prior_lo, w.prior_hi, eig[win], n_bad=nb[win])
    torch.cuda.synchronize()
    e = eig.cpu().numpy().reshape(3, 10, 512)
    bad = nb.cpu().numpy().reshape(3, 10, 512)
    # EIG grows with receiver count (mean over subsets of size k) and with measurement time
    ok = bad == 0
    means = np.array([[e[t, k][ok[t, k]].mean() for k in range(10)] for t in range(3)])
    assert np.all(np.diff(means[:, 1:], axis=1) > 0), means
    assert np.all(np.diff(means[:, 1:], axis=0) > 0), means
    # nested designs: adding receivers never lowers the EIG of the same nodes
    full = np.ones(w.nrec, dtype=np.uint8)
    e_full = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig_designs(ctx, Hr, 2, _t(full[None], torch.uint8), w_t, w.prior_lo, w.prior_hi, e_full)
    assert float(e_full.item()) > e[2][ok[2]].max()
    # the sweep's arithmetic against the oracle's log-det on the same partial Hessians
    Hr_h = Hr.cpu().numpy()
    iu = np.triu_indices(7)
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    rng = np.random.default_rng(0)
    for d in rng.choice(masks.shape[0], 3, replace=False):
        sel = np.nonzero(masks[d])[0]
        tot, nbad, cnd = 0.0, 0, 0.0
        for i in range(n):
            M = np.zeros((7, 7))
            M[iu] = Hr_h[i, sel, 2].sum(axis=0)
            M = M + np.triu(M, 1).T
            ld, Ht, good = oracle.scaled_logdet(M)
            if good:
                tot += wt[i] * oracle.dkl(ld, 7, lp)
                cnd += abs(wt[i]) * np.linalg.cond(Ht)
            else:
                nbad += 1
        assert bad[2].ravel()[d] == nbad
        assert abs(e[2].ravel()[d] - tot) <= 1e-10 * abs(tot) + 1e-14 * cnd
    # sampled partial Hessians against the oracle (FP32 stencil, difference form)
    G = oracle.Grid.from_workload(w)
    for i in (0, 511):
        _, Hrr = oracle.node_hessian(G, th[i], w.prior_lo, w.prior_hi, w.rel_step, sigma, wl)
        tot_ref = Hrr[:, 2].sum(axis=0)
        d = np.sqrt(np.outer(np.diag(tot_ref), np.diag(tot_ref)))[iu]
        assert np.max(np.abs(Hr_h[i, :, 2].sum(axis=0) - tot_ref[iu]) / d) <= 1e-4
