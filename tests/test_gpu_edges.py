"""Argument limits and degenerate inputs through the C ABI: the largest receiver counts
accepted (4096 for forward solves, 256 for Hessians), what lies beyond them rejected with
OED_EINVAL, empty batches as no-ops, and a one-receiver, one-step problem."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def test_receiver_and_batch_limits(P, oracle):
    nx = 4100
    w = W.tiny(nx=nx, nz=12, h=25.0, nsteps=6, nrec=3)
    th = np.array([[nx * 25.0 / 2, 100.0, 0.0, 6.0, 5e13, 2e13, 8e13]])
    # 4096 receivers: accepted, and the samples agree with the oracle's
    rec = list(range(2, 2 + 4096))
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64, rec_ix=rec), max_solves=1)
    g = torch.empty((1, w.nlevels, 4096, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    torch.cuda.synchronize()
    G = oracle.Grid(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, rec)
    ref = oracle.forward(G, th[0])
    assert np.max(np.abs(g[0].cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    # 4097 receivers: rejected at creation
    with pytest.raises(P.OedError):
        P.Context(P.problem_from_workload(w, P.OED_FP64, rec_ix=list(range(4097))), max_solves=1)
    # a Hessian needs at most 256 receivers
    ctx257 = P.Context(P.problem_from_workload(w, P.OED_FP64, rec_ix=list(range(257))), max_solves=15)
    H = torch.empty((1, 7, 7), dtype=torch.float64, device=DEV)
    with pytest.raises(P.OedError):
        P.oed_hessian(ctx257, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H)
    # solves per context in 1..65535
    for bad in (0, 65536):
        with pytest.raises(P.OedError):
            P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=bad)


def test_empty_batches_are_no_ops(P):
    w = W.tiny(nx=41, nz=21, nsteps=10, nrec=3)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=15)
    th = torch.empty((0, 7), dtype=torch.float64, device=DEV)
    g = torch.empty((0, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    H = torch.empty((0, 7, 7), dtype=torch.float64, device=DEV)
    wts = torch.empty(0, dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, th, g)
    P.oed_hessian(ctx, th, w.prior_lo, w.prior_hi, w.rel_step, 0.1, H)
    eig = torch.full((1,), 7.0, dtype=torch.float64, device=DEV)
    nb = torch.full((1,), 9, dtype=torch.int32, device=DEV)
    P.oed_eig(ctx, H, wts, w.prior_lo, w.prior_hi, eig, n_bad=nb)
    torch.cuda.synchronize()
    assert float(eig.item()) == 0.0 and int(nb.item()) == 0


@pytest.mark.parametrize("prec", [1, 0])
def test_one_receiver_one_step(P, oracle, prec):
    """nsteps = 1 (two levels, the first zero) and a single receiver: H_1 has rank <= 2, so
    every node is reported not positive definite and the EIG sums nothing."""
    w = W.tiny(nx=41, nz=21, nsteps=1, nrec=1)
    th = np.array([[1000.0, 500.0, 0.0, 6.0, 5e13, 2e13, 8e13]])
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=15)
    g = torch.empty((1, 2, 1, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    G = oracle.Grid.from_workload(w)
    ref = oracle.forward(G, th[0])
    tol = 1e-10 if prec == 1 else 1e-5
    assert np.allclose(g[0].cpu().numpy(), ref, rtol=tol, atol=tol * max(1e-30, np.abs(ref).max()))
    H = torch.empty((1, 7, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H)
    st = torch.empty(1, dtype=torch.int32, device=DEV)
    nb = torch.empty(1, dtype=torch.int32, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t([1.0]), w.prior_lo, w.prior_hi, eig, status=st, n_bad=nb)
    torch.cuda.synchronize()
    assert int(st.item()) == P.OED_ENOTPD and int(nb.item()) == 1 and float(eig.item()) == 0.0
