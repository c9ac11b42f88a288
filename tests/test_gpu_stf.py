"""The optional Ricker source time function through the C ABI, against the oracle.

The time function enters only the per-step source amplitudes, so one check per
stencil kernel suffices: FP64 seismograms to 1e-10 and FP32 to 1e-4 (normwise), the
resident and TMA kernels bit-identical to the streaming kernel, the pairs and
difference Jacobians' H_1 to 1e-9 (scaled, FP64), and the EIG to 1e-9 (FP64).  The
analytic time derivatives used by sensitivity solves and the dual solve exist for
the paper's Gaussian only; those calls are refused with OED_EINVAL.
"""
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


def _normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _scaled(H, Href):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Href)))
    return float(np.max(np.abs(H - Href) / (d[..., :, None] * d[..., None, :])))


def _thetas(w, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    return lo + (hi - lo) * rng.random((n, 7))


@pytest.fixture(scope="module")
def case(oracle):
    w = W.tiny(nx=75, nz=37, h=27.0, nsteps=150, nrec=4)
    th = _thetas(w, 4, seed=21)
    G = oracle.Grid.from_workload(w)
    ref = np.stack([oracle.forward(G, t, stf=oracle.STF_RICKER) for t in th])
    return w, th, G, ref


def test_ricker_forward_fp64_and_fp32(P, oracle, case):
    w, th, G, ref = case
    gauss = np.stack([oracle.forward(G, t) for t in th])
    for prec, tol in ((P.OED_FP64, 1e-10), (P.OED_FP32, 1e-4)):
        ctx = P.Context(P.problem_from_workload(w, prec, stf=P.OED_STF_RICKER), max_solves=15)
        g = torch.empty((4, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        out = g.cpu().numpy()
        for s in range(4):
            assert _normwise(out[s], ref[s]) <= tol, (prec, s, _normwise(out[s], ref[s]))
            assert _normwise(out[s], gauss[s]) > 1e-2   # the kind really reached the kernels


def test_ricker_resident_and_tma_bitwise_equal_streaming(P, case):
    w, th, G, ref = case
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32, stf=P.OED_STF_RICKER), max_solves=15)
    outs = []
    for C in (0, 1, -1):
        ctx.set_tuning(C, 4, 4)
        g = torch.empty((4, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        outs.append(g.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    assert _normwise(outs[0], ref) <= 1e-4


@pytest.mark.parametrize("jac", ["pairs", "difference"])
def test_ricker_hessian_and_eig_fp64(P, oracle, case, jac):
    w, th, G, ref = case
    sigma = 0.05
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64, stf=P.OED_STF_RICKER), max_solves=30)
    ctx.jacobian = P.OED_JAC_PAIRS if jac == "pairs" else P.OED_JAC_DIFFERENCE
    H = torch.empty((4, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.full((4,), -1, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, status=st)
    wt = np.full(4, 0.25)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(wt), w.prior_lo, w.prior_hi, eig)
    torch.cuda.synchronize()
    assert st.cpu().numpy().tolist() == [0, 0, 0, 0]
    Href = np.stack([oracle.node_hessian(G, t, w.prior_lo, w.prior_hi, w.rel_step, sigma,
                                         stf=oracle.STF_RICKER)[0] for t in th])
    assert _scaled(H.cpu().numpy(), Href) <= 1e-9
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    ref_e = float(sum(wt[k] * oracle.dkl(oracle.scaled_logdet(Href[k])[0], 7, lp) for k in range(4)))
    assert abs(float(eig.item()) - ref_e) <= 1e-9 * abs(ref_e)


def test_ricker_refuses_gaussian_only_paths(P, case):
    w, th, G, ref = case
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64, stf=P.OED_STF_RICKER), max_solves=15)
    with pytest.raises(P.OedError) as e:
        ctx.jacobian = P.OED_JAC_SENSITIVITY
    assert e.value.code == P.OED_EINVAL
    assert ctx.jacobian == P.OED_JAC_PAIRS
    y = torch.zeros((1, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    H = torch.zeros((1, 7, 7), dtype=torch.float64, device=DEV)
    grad = torch.zeros((1, 7), dtype=torch.float64, device=DEV)
    with pytest.raises(P.OedError) as e:
        P.oed_hessian_ii(ctx, _t(th[:1]), y, 0.1, H, grad)
    assert e.value.code == P.OED_EINVAL
    with pytest.raises(P.OedError) as e:
        P.oed_hessian_map(ctx, _t(th[:1]), y, w.prior_lo, w.prior_hi, w.rel_step, 0.1, 1, H, grad)
    assert e.value.code == P.OED_EINVAL
