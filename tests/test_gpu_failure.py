"""Failure detection without a GPU fault: a bounded wait that nothing completes.

The TMA streaming kernel's waits on its copies give up after a time limit, raise the
context's device flag and return; the Hessian combine turns the flag into OED_ETIMEOUT
for the nodes of that time loop, and the flag is cleared before the next one.  Here a
one-CTA kernel waits (50 ms limit) on a barrier phase that no agent completes: the call
must report OED_ETIMEOUT, and the same context must then run a forward solve and a
Hessian normally (status 0, results equal to a fresh context's) on the TMA kernel.
"""
import time

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


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _run(P, ctx, w, th):
    # the Hessian first: its status is the one the expired flag would have poisoned
    H = torch.empty((th.shape[0], 7, 7), dtype=torch.float64, device=DEV)
    st = torch.full((th.shape[0],), -1, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.05, H, status=st)
    g = torch.empty((th.shape[0], w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    torch.cuda.synchronize()
    return g.cpu().numpy(), H.cpu().numpy(), st.cpu().numpy()


def test_bounded_wait_expires_and_the_context_recovers(P):
    w = W.tiny(nx=75, nz=37, h=27.0, nsteps=80, nrec=4)
    rng = np.random.default_rng(3)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * rng.random((2, 7))
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=30)
    ctx.set_tuning(-1, 4, 4)   # the TMA kernel, whose waits are the bounded ones
    t0 = time.perf_counter()
    rc = P.oed_wait_selftest(ctx, 0.05)
    dt = time.perf_counter() - t0
    assert rc == P.OED_ETIMEOUT, P.library().oed_last_error(ctx.handle)
    assert 0.04 < dt < 5.0
    assert P.oed_wait_selftest(ctx, 3.0) == P.OED_EINVAL
    g, H, st = _run(P, ctx, w, th)
    assert st.tolist() == [0, 0]
    fresh = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=30)
    fresh.set_tuning(-1, 4, 4)
    g2, H2, st2 = _run(P, fresh, w, th)
    assert np.array_equal(g, g2) and np.array_equal(H, H2) and st2.tolist() == [0, 0]
