"""The allocation-free entry point oed_gauss_newton_noalloc.

It serves callers that cannot allocate device memory while they run (work being
recorded into a CUDA graph, stream-ordered pipelines, applications with a fixed
memory budget): it computes H_1 from seismograms the caller already holds, with
its scratch in a fixed array inside the library.  Its output is checked against
oed_hessian on the same problem, for two calls in a row (the second call must not
see the first call's leftovers in the shared scratch array).  This file is
collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _scaled(H, Href):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Href)))
    return float(np.max(np.abs(H - Href) / (d[..., :, None] * d[..., None, :])))


def test_noalloc_matches_oed_hessian_on_two_calls():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P

    w = W.tiny(nx=61, nz=31, h=33.0, nsteps=90, nrec=4)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    d = w.rel_step * (hi - lo)
    sigma = 0.05
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=60)
    for call, (seed, mode) in enumerate(((1, P.OED_JAC_PAIRS), (2, P.OED_JAC_DIFFERENCE))):
        n = 3 + call
        rng = np.random.default_rng(seed)
        th = lo + (hi - lo) * rng.random((n, 7))
        # reference: the existing entry point
        ctx.jacobian = mode
        H_ref = torch.empty((n, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, torch.tensor(th, device=DEV), w.prior_lo, w.prior_hi, w.rel_step,
                      sigma, H_ref)
        # seismograms of every perturbed solve from the forward map
        pert = [[t] + [t + s * d[j] * np.eye(7)[j] for j in range(7) for s in (1.0, -1.0)]
                for t in th]
        pert = np.array(pert).reshape(n * 15, 7)
        gs = torch.empty((n * 15, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
        P.oed_forward(ctx, torch.tensor(pert, device=DEV), gs)
        gs = gs.reshape(n, 15, w.nlevels, w.nrec, 2)
        if mode == P.OED_JAC_DIFFERENCE:
            gs = (gs[:, 1::2] - gs[:, 2::2]).contiguous()   # g(theta + d e_j) - g(theta - d e_j)
        H = torch.full((n, 7, 7), float("nan"), dtype=torch.float64, device=DEV)
        rc = P.oed_gauss_newton_noalloc(gs, w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
        torch.cuda.synchronize()
        assert rc == P.OED_OK
        assert _scaled(H.cpu().numpy(), H_ref.cpu().numpy()) <= 1e-9, call
    # beyond the fixed scratch array: refused, nothing launched
    big = torch.zeros((600, 7, 9, 4, 2), dtype=torch.float64, device=DEV)
    Hb = torch.zeros((600, 7, 7), dtype=torch.float64, device=DEV)
    assert P.oed_gauss_newton_noalloc(big, w.prior_lo, w.prior_hi, w.rel_step, sigma, Hb) == P.OED_ENOMEM
    assert not Hb.any()
    ctx.close()


def _gn_numpy(g, lo, hi, rel_step, sigma):
    """sigma^-2 sum over (m, r, c) of J J^T with J from the FD form of g (numpy, FP64)."""
    d = rel_step * (np.asarray(hi) - np.asarray(lo))
    if g.shape[1] == 15:
        J = (g[:, 1::2] - g[:, 2::2]) / (2.0 * d)[None, :, None, None, None]
    else:
        J = g / (2.0 * d)[None, :, None, None, None]
    J = J.reshape(g.shape[0], 7, -1)
    return np.einsum("njk,nik->nji", J, J) / sigma ** 2


@pytest.mark.parametrize("per_node,nlev,nrec,n", [(15, 40, 100, 2), (7, 5, 3, 4), (7, 12, 256, 1),
                                                  (15, 1, 7, 3)])
def test_noalloc_launch_shapes_against_numpy(per_node, nlev, nrec, n):
    """The other launch shapes: more than 64 receivers (one lane per seismogram row, blocks
    of up to 512 threads and 118 KB of shared memory) and fewer than eight time levels
    (one sub-segment per level), on random FP64 seismograms, against numpy."""
    import __graft_entry__ as g_
    g_.build()
    import paper_1502_07873_gb300 as P

    rng = np.random.default_rng(1000 * nrec + nlev)
    lo, hi = np.array(W.PRIOR_LO), np.array(W.PRIOR_HI)
    g = rng.standard_normal((n, per_node, nlev, nrec, 2))
    sigma = 0.3
    for _ in range(2):   # two calls in a row through the shared scratch array
        H = torch.full((n, 7, 7), float("nan"), dtype=torch.float64, device=DEV)
        rc = P.oed_gauss_newton_noalloc(torch.tensor(g, device=DEV), lo, hi, 1e-4, sigma, H)
        torch.cuda.synchronize()
        assert rc == P.OED_OK
        Href = _gn_numpy(g, lo, hi, 1e-4, sigma)
        assert _scaled(H.cpu().numpy(), Href) <= 1e-11
        g = g[::-1].copy()


def test_noalloc_binding_refuses_bad_tensors():
    """Shape and dtype checks in the binding: nothing reaches the device."""
    import __graft_entry__ as g_
    g_.build()
    import paper_1502_07873_gb300 as P

    lo, hi = W.PRIOR_LO, W.PRIOR_HI
    g = torch.zeros((2, 7, 9, 4, 2), dtype=torch.float64, device=DEV)
    H = torch.zeros((2, 7, 7), dtype=torch.float64, device=DEV)
    for bad_g, bad_H in ((g.float(), H), (g[..., 0], H), (g, H.float()), (g, H[:1])):
        with pytest.raises(ValueError):
            P.oed_gauss_newton_noalloc(bad_g, lo, hi, 1e-4, 0.1, bad_H)
