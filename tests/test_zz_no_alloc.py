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
