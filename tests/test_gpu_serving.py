"""Serving loop: continuous batching with admission by device footprint.

Each request's EIG matches the FP64 oracle and is the same alone and in a mix of
concurrently running requests of other grid sizes, media and Jacobian forms; a request
larger than the budget is run in smaller chunks or refused; a budget that holds one
request at a time serialises admission; pooled workspaces are reused across requests
of one grid shape; small requests pass a head blocked on memory only within the age
bound; a cancelled request resumes from its per-node checkpoint to the same EIG; every
finished request has a JSON metrics line.
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
    r = P.make_request(P.problem_from_workload(w, precision), th, wt, w.prior_lo, w.prior_hi,
                       w.rel_step, sigma, jacobian)
    r._workload, r._sigma, r._precision = w, sigma, precision
    return r


def _mix(P):
    """Grids, media, node counts and receiver counts of different sizes, in the forms the
    server is used with: the FP32 stencil with the difference-form Jacobian and the plain
    FP64 form with central-FD pairs."""
    lay = W.THREE_LAYER
    # every record is about 0.5 s long: a source starting at t_s = 0.3 s has reached the
    # receivers, so no node's H_1 is near-singular (a record that ends before the source
    # starts makes log det H_1 move by cond(H_1) times the rounding, even in FP64)
    return [
        _req(P, W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5), 9, 1, jacobian=1),
        _req(P, W.tiny(nx=101, nz=51, h=20.0, nsteps=230, nrec=7, layers=lay), 6, 2, jacobian=1),
        _req(P, W.tiny(nx=201, nz=101, h=10.0, nsteps=300, nrec=9), 5, 3, precision=1),
        _req(P, W.tiny(nx=61, nz=31, h=33.0, nsteps=90, nrec=4), 12, 4, jacobian=1),
        _req(P, W.tiny(nx=161, nz=81, h=12.5, nsteps=360, nrec=6, layers=lay), 4, 5, precision=1),
    ]


def _oracle_eig(oracle, r):
    w = r._workload
    ref = oracle.eig(oracle.Grid.from_workload(w), r._th, r._w, w.prior_lo, w.prior_hi, w.rel_step,
                     r._sigma)
    return ref["eig"]


def _bar(r):
    """The accuracy bar of a served EIG against the FP64 oracle: 1e-9 for the FP64
    stencil, 1e-3 for the mixed-precision path."""
    return 1e-9 if r._precision == 1 else 1e-3


def test_same_result_alone_and_in_the_mix(P, oracle):
    reqs = _mix(P)
    refs = [_oracle_eig(oracle, r) for r in reqs]
    budget = 40 << 30
    alone = []
    for r, ref in zip(reqs, refs):
        srv = P.Server(budget, max_active=1, chunk_nodes=4, autotune=False)
        res = srv.wait(srv.submit(r))
        srv.close()
        assert res.status == P.OED_OK
        assert abs(res.eig - ref) <= _bar(r) * abs(ref), (res.eig, ref)
        alone.append(res.eig)
    srv = P.Server(budget, max_active=4, chunk_nodes=4, autotune=False)
    ids = [srv.submit(r) for r in reqs] + [srv.submit(r) for r in reqs]   # each twice, overlapping
    res = [srv.wait(i) for i in ids]
    srv.close()
    for k, r in enumerate(res):
        assert r.status == P.OED_OK
        a = alone[k % len(reqs)]
        assert abs(r.eig - a) <= 1e-12 * abs(a), (k, r.eig, a)
        ref = refs[k % len(reqs)]
        assert abs(r.eig - ref) <= _bar(reqs[k % len(reqs)]) * abs(ref), (k, r.eig, ref)
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
    # larger than the whole budget even one node at a time: refused at submission
    one = P.Server(1 << 40, max_active=1, chunk_nodes=1, autotune=False)
    size1 = one.request_bytes(reqs[0])
    one.close()
    small = P.Server(size1 - 1, max_active=2, chunk_nodes=4, autotune=False)
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


def _theta(w, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    return lo + (hi - lo) * rng.random((n, 7))


def test_pooled_workspace_is_reused_and_gives_the_same_result(P, oracle):
    """Requests of one grid shape with different step counts, media and receivers: the
    later ones run in the first one's workspace (oed_rebind) and match a fresh server and
    the oracle."""
    ws = [W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5),
          W.tiny(nx=81, nz=41, h=25.0, nsteps=180, nrec=3, layers=W.THREE_LAYER),
          W.tiny(nx=81, nz=41, h=25.0, nsteps=110, nrec=4)]
    reqs = [_req(P, w, 6, 20 + k, jacobian=1) for k, w in enumerate(ws)]
    srv = P.Server(8 << 30, max_active=1, chunk_nodes=6, autotune=False)
    res = [srv.wait(srv.submit(r)) for r in reqs]
    idle, idle_b = srv.pool()
    srv.close()
    assert [r.status for r in res] == [P.OED_OK] * 3
    assert [r.workspace_reused for r in res] == [0, 1, 1]
    assert idle == 1 and idle_b > 0
    for r, q in zip(res, reqs):
        fresh = P.Server(8 << 30, max_active=1, chunk_nodes=6, autotune=False)
        f = fresh.wait(fresh.submit(q))
        fresh.close()
        assert f.workspace_reused == 0
        assert r.eig == f.eig
        ref = _oracle_eig(oracle, q)
        assert abs(r.eig - ref) <= 1e-3 * abs(ref)


def _blocked_head_order(P, max_wait_s):
    """A running request A and a queued request B of A's size under a budget that holds
    A plus one small request: B waits for memory at the head of the queue, and the small
    request C, submitted after B, is either admitted past it or not."""
    big = W.tiny(nx=201, nz=101, h=10.0, nsteps=400, nrec=5)
    small = W.tiny(nx=61, nz=31, h=33.0, nsteps=60, nrec=3)
    A = _req(P, big, 24, 31, precision=1)
    B = _req(P, big, 24, 32, precision=1)
    C = _req(P, small, 2, 33)
    probe = P.Server(1 << 40, max_active=1, chunk_nodes=24, autotune=False)
    fa, fc = probe.request_bytes(A), probe.request_bytes(C)
    probe.close()
    assert fa > fc
    srv = P.Server(fa + fc + 4096, max_active=3, chunk_nodes=24, autotune=False)
    srv.set_admission(max_wait_s)
    ia = srv.submit(A)
    ib = srv.submit(B)
    ic = srv.submit(C)
    ra, rb, rc = srv.wait(ia), srv.wait(ib), srv.wait(ic)
    srv.close()
    assert ra.status == rb.status == rc.status == P.OED_OK
    return ra, rb, rc


def test_small_requests_pass_a_blocked_head_only_within_the_age_bound(P):
    ra, rb, rc = _blocked_head_order(P, 60.0)
    assert rc.t_admit < ra.t_done <= rb.t_admit + 1e-6   # C ran while B waited for A's memory
    ra, rb, rc = _blocked_head_order(P, 0.0)              # no passing: first come, first served
    assert rb.t_admit <= rc.t_admit
    assert rb.t_admit >= ra.t_done - 1e-6


def test_cancel_then_resume_from_the_checkpoint_gives_the_same_eig(P):
    import time
    w = W.tiny(nx=201, nz=101, h=10.0, nsteps=300, nrec=6)
    n = 40
    th = _theta(w, n, 41)
    wt = np.full(n, 1.0 / n)
    prob = P.problem_from_workload(w, P.OED_FP64)
    full_req = P.make_request(prob, th, wt, w.prior_lo, w.prior_hi, w.rel_step, 0.05, P.OED_JAC_PAIRS, tag=7)
    srv = P.Server(16 << 30, max_active=1, chunk_nodes=2, autotune=False)
    full = srv.wait(srv.submit(full_req))
    assert full.status == P.OED_OK and full.nodes_done == n
    H_full = srv.checkpoint(1)
    assert H_full.shape == (n, 7, 7)
    # cancel mid-run
    rid = srv.submit(P.make_request(prob, th, wt, w.prior_lo, w.prior_hi, w.rel_step, 0.05, P.OED_JAC_PAIRS))
    t0 = time.time()
    while srv.poll(rid).nodes_done < 4 and time.time() - t0 < 60:
        time.sleep(0.001)
    srv.cancel(rid)
    r = srv.wait(rid)
    assert r.status == P.OED_ECANCELED
    k = r.nodes_done
    assert 4 <= k < n, k
    Hk = srv.checkpoint(rid)
    assert Hk.shape == (k, 7, 7)
    assert np.array_equal(Hk, H_full[:k])        # per-node Hessians do not depend on chunking
    m = srv.metrics(rid)
    assert m["status"] == "OED_ECANCELED" and m["nodes_done"] == k
    # resume: only the remaining nodes are computed
    res = srv.wait(srv.submit(P.make_request(prob, th, wt, w.prior_lo, w.prior_hi, w.rel_step, 0.05,
                                             P.OED_JAC_PAIRS, H_done=Hk, tag=8)))
    assert res.status == P.OED_OK and res.nodes_done == n
    assert res.eig == full.eig
    m = srv.metrics(3)
    assert m["nodes_resumed"] == k and m["tag"] == 8
    assert m["cell_updates"] == w.nx * w.nz * w.nsteps * 15 * (n - k)
    # resuming with every node done computes no solve: the EIG comes from the checkpoint
    res_all = srv.wait(srv.submit(P.make_request(prob, th, wt, w.prior_lo, w.prior_hi, w.rel_step, 0.05,
                                                 P.OED_JAC_PAIRS, H_done=H_full)))
    assert res_all.status == P.OED_OK and res_all.eig == full.eig
    assert srv.metrics(4)["cell_updates"] == 0
    # a queued request that is cancelled never runs
    srv2 = P.Server(16 << 30, max_active=1, chunk_nodes=2, autotune=False)
    ids = [srv2.submit(full_req), srv2.submit(full_req)]
    srv2.cancel(ids[1])
    r2 = srv2.wait(ids[1])
    assert r2.status == P.OED_ECANCELED and r2.nodes_done == 0
    assert srv2.wait(ids[0]).status == P.OED_OK
    srv2.close()
    srv.close()


def test_metrics_lines(P, tmp_path):
    import json
    w = W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5)
    log = tmp_path / "serve.jsonl"
    srv = P.Server(8 << 30, max_active=2, chunk_nodes=4, autotune=False)
    srv.set_log(str(log))
    ids = [srv.submit(P.make_request(P.problem_from_workload(w, 0), _theta(w, 5, s), np.full(5, 0.2),
                                     w.prior_lo, w.prior_hi, w.rel_step, 0.05, 1, tag=100 + s))
           for s in range(3)]
    res = [srv.wait(i) for i in ids]
    # a finished request's record can be dropped; its id is unknown afterwards
    assert srv.release(ids[0]) == P.OED_OK
    assert srv.release(ids[0]) == P.OED_EINVAL
    with pytest.raises(P.OedError):
        srv.poll(ids[0])
    srv.close()
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert sorted(d["tag"] for d in lines) == [100, 101, 102]
    for d in lines:
        r = res[d["id"] - 1]
        assert d["status"] == "OED_OK" and d["eig"] == r.eig
        assert d["grid"] == "81x41" and d["nsteps"] == 120 and d["receivers"] == 5 and d["nodes"] == 5
        assert d["precision"] == "f32" and d["jacobian"] == "difference"
        assert d["cell_updates"] == 81 * 41 * 120 * 7 * 5
        assert d["latency_s"] >= d["run_s"] > 0 and d["gcell_upd_per_s"] > 0


def test_chunks_shrink_to_fit_the_budget(P):
    """A request whose workspace at the configured chunk exceeds the budget runs in smaller
    chunks and gives the direct call's result."""
    w = W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5)
    r = _req(P, w, 16, 51, jacobian=1)
    big = P.Server(1 << 40, max_active=1, chunk_nodes=16, autotune=False)
    full = big.wait(big.submit(r))
    f16 = big.request_bytes(r)
    big.close()
    srv = P.Server(f16 // 2, max_active=1, chunk_nodes=16, autotune=False)
    res = srv.wait(srv.submit(r))
    srv.close()
    assert res.status == P.OED_OK and res.footprint_bytes <= f16 // 2
    assert res.eig == full.eig
