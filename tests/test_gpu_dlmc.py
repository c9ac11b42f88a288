"""Parity of the parameter-subset Laplace gain and of the double-loop Monte Carlo
estimator (Sec. 4.3-4.4) with the FP64 oracle, through the C ABI.

Both are FP64 end to end, so the bar is rounding: relative 1e-12 on log-determinants,
per-node gains, log-evidences and EIG values (1e-10 where a sum of ~1e3 exponentials
of values of size ~1e2 is involved)."""
import math

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


def test_eig_subset_matches_oracle(P, oracle):
    w = W.tiny(nx=60, nz=33, h=30.0, nsteps=90, nrec=5)
    rng = np.random.default_rng(3)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * rng.random((6, 7))
    G = oracle.Grid.from_workload(w)
    Hs = np.array([oracle.node_hessian(G, t, lo, hi, w.rel_step, 0.2)[0] for t in th])
    wts = rng.uniform(0.05, 0.3, 6)
    H = _t(Hs)
    for free in ([1, 3, 4], [0, 4], [2], [0, 1, 2, 3, 4, 5, 6], [4, 5, 6]):
        eig = torch.empty(1, dtype=torch.float64, device=DEV)
        dkl = torch.empty(6, dtype=torch.float64, device=DEV)
        st = torch.empty(6, dtype=torch.int32, device=DEV)
        P.oed_eig_subset(None, H, _t(wts), lo, hi, free, eig, dkl=dkl, status=st)
        lp = oracle.log_uniform_density(lo[free], hi[free])
        ref = []
        for k in range(6):
            ld, ok = oracle.scaled_logdet_sub(Hs[k], free)
            assert ok
            ref.append(oracle.dkl(ld, len(free), lp))
        ref = np.array(ref)
        assert st.cpu().tolist() == [0] * 6
        assert np.allclose(dkl.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert abs(float(eig.item()) - float(wts @ ref)) <= 1e-12 * abs(float(wts @ ref))
    # the full mask is oed_eig
    e1 = torch.empty(1, dtype=torch.float64, device=DEV)
    e2 = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(None, H, _t(wts), lo, hi, e1)
    P.oed_eig_subset(None, H, _t(wts), lo, hi, range(7), e2)
    assert float(e1.item()) == float(e2.item())
    with pytest.raises(P.OedError):
        P.oed_eig_subset(None, H, _t(wts), lo, hi, [], e2)


@pytest.mark.parametrize("N,M,D", [(1, 1, 1), (70, 150, 45), (33, 65, 64), (128, 7, 300)])
def test_dlmc_matches_oracle(P, oracle, N, M, D):
    """Ragged against the 32 x 64 x 32 tiles; data of unequal scale per dimension."""
    rng = np.random.default_rng(N * 1000 + M)
    scale = np.exp(rng.uniform(-2, 2, D))
    go = rng.standard_normal((N, D)) * scale
    gi = go[rng.integers(0, N, M)] + 0.3 * rng.standard_normal((M, D)) * scale
    eps = 0.2 * rng.standard_normal((N, D))
    sigma = 0.7
    le_ref, eig_ref = oracle.dlmc(go, eps, gi, sigma)
    le = torch.empty(N, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_dlmc(_t(go), _t(eps), _t(gi), sigma, le, eig)
    torch.cuda.synchronize()
    assert np.allclose(le.cpu().numpy(), le_ref, rtol=1e-12, atol=1e-10)
    assert abs(float(eig.item()) - eig_ref) <= 1e-12 * max(1.0, abs(eig_ref)) + 1e-10


def test_dlmc_one_inner_sample_equal_to_outer_gives_zero(P):
    rng = np.random.default_rng(9)
    go = rng.standard_normal((1, 50))
    eps = 0.1 * rng.standard_normal((1, 50))
    le = torch.empty(1, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_dlmc(_t(go), _t(eps), _t(go), 0.1, le, eig)
    assert abs(float(eig.item())) < 1e-12
    assert abs(float(le.item()) + float((eps * eps).sum()) / (2 * 0.01)) < 1e-10


def test_dlmc_on_seismograms_at_scale_sampled(P, oracle):
    """The paper's Sec. 4.4 setting at the size the benchmark runs it: the model problem to
    T = 1.25 s, two receivers, three unknown parameters; 4096 outer and 4096 inner samples
    from the GPU forward solver (FP64 stencil).  Eight outer samples' log-evidences against
    the oracle computed over all inner samples."""
    w = W.paper_study_model()
    rng = np.random.default_rng(17)
    N = M = 4096
    th_o, th_i = W.paper_study_thetas(rng.random((N, 3))), W.paper_study_thetas(rng.random((M, 3)))
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=1024)
    D = w.nlevels * w.nrec * 2
    go = torch.empty((N, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    gi = torch.empty((M, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    for a in range(0, N, 1024):
        P.oed_forward(ctx, _t(th_o[a:a + 1024]), go[a:a + 1024])
        P.oed_forward(ctx, _t(th_i[a:a + 1024]), gi[a:a + 1024])
    sigma = 0.01
    eps = sigma * rng.standard_normal((N, D))
    le = torch.empty(N, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_dlmc(go, _t(eps), gi, sigma, le, eig)
    torch.cuda.synchronize()
    gon = go.cpu().numpy().reshape(N, D)
    gin = gi.cpu().numpy().reshape(M, D)
    pick = rng.choice(N, 8, replace=False)
    le_ref, _ = oracle.dlmc(gon[pick], eps[pick], gin, sigma)
    assert np.allclose(le.cpu().numpy()[pick], le_ref, rtol=1e-10, atol=1e-9)
    # the GPU seismograms themselves against the oracle on two of the samples
    G = oracle.Grid.from_workload(w)
    for i in pick[:2]:
        ref = oracle.forward(G, th_o[i])
        assert np.max(np.abs(gon[i] - ref.ravel())) <= 1e-10 * np.max(np.abs(ref))
    assert math.isfinite(float(eig.item()))
