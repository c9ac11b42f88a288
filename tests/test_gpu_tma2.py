"""The two-step TMA streaming kernel (two leap-frog steps per pass, Eq. Full_Disc).

On grids that do not fit the cluster-resident kernel (801x161 and 415x801, h = 5 m, three
layers; both odd widths, so the last column pair holds the zero ghost column), its
seismograms equal the register streaming kernel's bit for bit -- for an even and an odd
step count (the odd one ends with a single-step pass), with sources whose patches
straddle the 60-column tile boundaries and the 20-row bands, and on the replay of the
captured time loop -- and meet the FP32 bar against the FP64 oracle.  415 columns take
a little more memory per solve in the kernel's paired layout than in the planar one.
Hessians through it equal those of the register kernel.
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


def _normwise(g, ref):
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


def _thetas():
    """Sources on and around tile boundaries: x_s at 900 and 1200 m (columns 180 and 240,
    multiples of the 60-column tile), 1027 m (mid-tile); depths at 400, 500 and 600 m
    (rows 80, 100, 120, multiples of the 20-row band) and 455 m; early starts."""
    rows = []
    for xs, zs in ((900.0, 400.0), (1200.0, 500.0), (1027.0, 455.0), (900.0, 600.0), (1195.0, 405.0),
                   (1002.5, 597.5)):
        rows.append([xs, zs, 0.1, 7.0, 6e13, 3e13, 9e13])
        rows.append([xs, zs, 0.12, 5.0, 2e13, 8e13, 4e13])
    return np.array(rows)


@pytest.mark.parametrize("nx,nz,nsteps", [(801, 161, 400), (801, 161, 401), (415, 801, 401)])
def test_two_step_tma_bitwise_and_against_oracle(P, oracle, nx, nz, nsteps):
    w = W.tiny(nx=nx, nz=nz, h=5.0, nsteps=nsteps, nrec=10, layers=W.THREE_LAYER)
    th = _thetas()
    n = th.shape[0]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=n)
    assert ctx.resident_min_cluster == 0   # the grid does not fit on chip
    ctx.set_tuning(0, 4, 4)
    g_ref = torch.empty((n, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_ref)
    ctx.set_tuning(-2, 4, 4)
    assert ctx.tuning[0] == -2
    g = torch.empty_like(g_ref)
    for _ in range(2):   # the second call replays the captured time loop
        g.fill_(float("nan"))
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
    assert float(g_ref.abs().max()) > 0
    G = oracle.Grid.from_workload(w)
    for k in (0, 5):
        assert _normwise(g[k].cpu().numpy(), oracle.forward(G, th[k])) <= 1e-4
    ctx.close()


def test_two_step_tma_hessians_equal_the_register_kernel(P):
    w = W.tiny(nx=801, nz=161, h=5.0, nsteps=300, nrec=8)
    th = _thetas()[:4]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=28)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    H = {}
    for tune in ((0, 4, 4), (-2, 4, 4)):
        ctx.set_tuning(*tune)
        H[tune[0]] = torch.empty((4, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H[tune[0]])
    torch.cuda.synchronize()
    assert torch.equal(H[0], H[-2])
    ctx.close()


def test_two_step_needs_a_grid_that_does_not_fit_on_chip(P):
    w = W.tiny(nx=401, nz=201, h=5.0, nsteps=10, nrec=4)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=4)
    with pytest.raises(P.OedError):
        ctx.set_tuning(-2, 4, 4)
    ctx.close()
