"""Serving loop: continuous batching with admission by device footprint.

Each request's EIG is the same alone and in a mix of concurrently running requests
of other grid sizes, media and Jacobian forms; a request larger than the budget is
refused; a budget that holds one request at a time serialises admission.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def _req(P, w, n, seed, sigma=0.05, jacobian=0, precision=0):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * rng.random((n, 7))
    wt = np.full(n, 1.0 / n)
    return P.make_request(P.problem_from_workload(w, precision), th, wt, w.prior_lo, w.prior_hi,
                          w.rel_step, sigma, jacobian)


def _mix(P):
    lay = W.THREE_LAYER
    return [
        _req(P, W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5), 9, 1),
        _req(P, W.tiny(nx=101, nz=51, h=20.0, nsteps=150, nrec=7, layers=lay), 6, 2, jacobian=1),
        _req(P, W.tiny(nx=201, nz=101, h=10.0, nsteps=100, nrec=9), 5, 3),
        _req(P, W.tiny(nx=61, nz=31, h=33.0, nsteps=90, nrec=4), 12, 4, jacobian=1),
        _req(P, W.tiny(nx=161, nz=81, h=12.5, nsteps=110, nrec=6, layers=lay), 4, 5),
    ]


def test_same_result_alone_and_in_the_mix(P):
    reqs = _mix(P)
    budget = 40 << 30
    alone = []
    for r in reqs:
        srv = P.Server(budget, max_active=1, chunk_nodes=4, autotune=False)
        res = srv.wait(srv.submit(r))
        srv.close()
        assert res.status == P.OED_OK
        alone.append(res.eig)
    srv = P.Server(budget, max_active=4, chunk_nodes=4, autotune=False)
    ids = [srv.submit(r) for r in reqs] + [srv.submit(r) for r in reqs]   # each twice, overlapping
    res = [srv.wait(i) for i in ids]
    srv.close()
    for k, r in enumerate(res):
        assert r.status == P.OED_OK
        a = alone[k % len(reqs)]
        assert abs(r.eig - a) <= 1e-12 * abs(a), (k, r.eig, a)
    # requests really overlapped: some request was admitted before another one finished
    spans = sorted((r.t_admit, r.t_done) for r in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_admission_by_footprint(P):
    w = W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5)
    reqs = [_req(P, w, 8, seed) for seed in (7, 8, 9)]
    srv0 = P.Server(1 << 40, max_active=1, chunk_nodes=4, autotune=False)
    sizes = [srv0.request_bytes(r) for r in reqs]
    srv0.close()
    assert all(s > 0 for s in sizes) and len(set(sizes)) == 1
    # a budget that holds one request but not two: one at a time
    budget = 2 * sizes[0] - 1
    srv = P.Server(budget, max_active=4, chunk_nodes=4, autotune=False)
    ids = [srv.submit(r) for r in reqs]
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert all(r.status == P.OED_OK for r in res)
    spans = sorted((r.t_admit, r.t_done) for r in res)
    for i in range(len(spans) - 1):
        assert spans[i + 1][0] >= spans[i][1] - 1e-6
    # first come, first served
    assert [r.t_admit for r in res] == sorted(r.t_admit for r in res)
    # larger than the whole budget: refused at submission
    small = P.Server(min(sizes) // 2, max_active=2, chunk_nodes=4, autotune=False)
    with pytest.raises(P.OedError) as e:
        small.submit(reqs[0])
    assert e.value.code == P.OED_ENOMEM
    small.close()


def test_server_matches_direct_calls(P):
    """A served request gives the EIG of the direct oed_hessian + oed_eig calls."""
    w = W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5)
    r = _req(P, w, 9, 1)
    srv = P.Server(8 << 30, max_active=2, chunk_nodes=4, autotune=False)
    res = srv.wait(srv.submit(r))
    srv.close()
    ctx = P.Context(P.problem_from_workload(w, 0), max_solves=60)
    th = torch.tensor(r._th, device="cuda")
    H = torch.empty((9, 7, 7), dtype=torch.float64, device="cuda")
    P.oed_hessian(ctx, th, w.prior_lo, w.prior_hi, w.rel_step, 0.05, H)
    eig = torch.empty(1, dtype=torch.float64, device="cuda")
    P.oed_eig(ctx, H, torch.tensor(r._w, device="cuda"), w.prior_lo, w.prior_hi, eig)
    assert abs(res.eig - float(eig.item())) <= 1e-12 * abs(res.eig)
