"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  - FP64 stencil: seismograms normwise max|g - g_ref| / max|g_ref| <= 1e-10, scaled
    Hessian entries |H - H_ref|_ij / sqrt(H_ii H_jj) <= 1e-9, EIG relative <= 1e-9.
  - FP32 stencil (FP64 Jacobian / Hessian / log-det): seismograms <= 1e-4, EIG
    relative <= 1e-3.
Sizes span several 32-column tiles and 8-row segments with ragged tails.
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


GRIDS = {
    "homog_75x37": dict(nx=75, nz=37, h=27.0, nsteps=150, nrec=4),
    "layered_70x41": dict(nx=70, nz=41, h=25.0, nsteps=140, nrec=5,
                          layers=((0.0, 2000.0, 1155.0, 2200.0), (300.0, 3000.0, 1732.0, 2500.0),
                                  (600.0, 4500.0, 2598.0, 2700.0))),
}


def _thetas(w, n, seed=5):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    return lo + (hi - lo) * rng.random((n, 7))


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-4)])
def test_forward_matches_oracle(P, oracle, grid, prec, tol):
    w = W.tiny(**GRIDS[grid])
    th = _thetas(w, 5)
    G = oracle.Grid.from_workload(w)
    ref = np.stack([oracle.forward(G, t) for t in th])
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=15)
    g = torch.empty((5, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    torch.cuda.synchronize()
    out = g.cpu().numpy()
    for s in range(5):
        assert _normwise(out[s], ref[s]) <= tol, (s, _normwise(out[s], ref[s]))


def test_forward_chunks_and_empty(P, oracle):
    """n > max_solves runs in chunks (15, 15, 7); n = 0 is a no-op."""
    w = W.tiny(nx=41, nz=21, nsteps=60, nrec=3)
    th = _thetas(w, 37, seed=9)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=15)
    g = torch.empty((37, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    P.oed_forward(ctx, _t(np.zeros((0, 7))), torch.empty((0, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    G = oracle.Grid.from_workload(w)
    for s in (0, 14, 15, 29, 30, 36):
        assert _normwise(g[s].cpu().numpy(), oracle.forward(G, th[s])) <= 1e-10


def test_forward_invalid_source_is_nan(P):
    w = W.tiny(nx=41, nz=21, nsteps=20, nrec=3)
    th = _thetas(w, 2)
    th[1, 0] = 10.0   # patch leaves the grid
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=15)
    g = torch.empty((2, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g)
    out = g.cpu().numpy()
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1]))


@pytest.mark.parametrize("grid", sorted(GRIDS))
def test_hessian_fp64_matches_oracle(P, oracle, grid):
    w = W.tiny(**GRIDS[grid])
    th = _thetas(w, 3, seed=2)
    wl = [31, 77, w.nlevels]
    G = oracle.Grid.from_workload(w)
    sigma = 0.07
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=30)   # chunks of 2 nodes
    H = torch.empty((3, 7, 7), dtype=torch.float64, device=DEV)
    Hr = torch.empty((3, w.nrec, 3, 28), dtype=torch.float64, device=DEV)
    st = torch.full((3,), -1, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=wl,
                  H_rec=Hr, status=st)
    torch.cuda.synchronize()
    iu = np.triu_indices(7)
    for i in range(3):
        Href, Hrref = oracle.node_hessian(G, th[i], w.prior_lo, w.prior_hi, w.rel_step, sigma, wl)
        assert _scaled(H[i].cpu().numpy(), Href) <= 1e-9
        for r in range(w.nrec):
            for k in range(3):
                ref_u = Hrref[r, k][iu]
                dd = np.sqrt(np.outer(np.diag(Href), np.diag(Href)))[iu]
                assert np.max(np.abs(Hr[i, r, k].cpu().numpy() - ref_u) / dd) <= 1e-9
    assert st.cpu().numpy().tolist() == [0, 0, 0]


def test_eig_plain_small_fp64_and_fp32(P, oracle):
    """The 81x41 / 400-step / 16-node workload end to end: FP64 to 1e-9, FP32 to 1e-3."""
    w = W.plain_small()
    G = oracle.Grid.from_workload(w)
    th, wt = oracle.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    sigma = 0.4
    ref = oracle.eig(G, th, wt, w.prior_lo, w.prior_hi, w.rel_step, sigma, want_h=True)
    for prec, tol in ((P.OED_FP64, 1e-9), (P.OED_FP32, 1e-3)):
        ctx = P.Context(P.problem_from_workload(w, prec), max_solves=240)
        H = torch.empty((16, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
        eig = torch.empty(1, dtype=torch.float64, device=DEV)
        dkl = torch.empty(16, dtype=torch.float64, device=DEV)
        nb = torch.empty(1, dtype=torch.int32, device=DEV)
        P.oed_eig(ctx, H, _t(wt), w.prior_lo, w.prior_hi, eig, dkl=dkl, n_bad=nb)
        torch.cuda.synchronize()
        assert int(nb.item()) == 0
        e = float(eig.item())
        assert abs(e - ref["eig"]) / abs(ref["eig"]) <= tol, (prec, e, ref["eig"])
        assert np.max(np.abs(dkl.cpu().numpy() - ref["dkl"]) / np.abs(ref["dkl"])) <= tol * 10
        if prec == P.OED_FP64:
            assert _scaled(H.cpu().numpy(), ref["H"]) <= 1e-9


def test_chunking_and_launch_shape_are_bitwise_invariant(P):
    """Chunk size and the streaming kernel's launch shape change scheduling only."""
    w = W.tiny(nx=41, nz=21, nsteps=50, nrec=3)
    th = _thetas(w, 7, seed=3)
    out = []
    for ms, shape in ((45, None), (150, (0, 2, 1)), (150, (0, 8, 8)), (150, (0, 4, 2))):
        ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=ms)
        if shape:
            ctx.set_tuning(*shape)
            assert ctx.tuning == shape
        H = torch.empty((7, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H)
        out.append(H.cpu().numpy())
    for o in out[1:]:
        assert np.array_equal(out[0], o)


RESIDENT_CASES = [  # grid, cluster sizes to try (1 CTA, and multi-CTA with DSMEM halos)
    ("homog_75x37", (1, 2, 3, 5)),
    ("layered_70x41", (1, 2, 4, 7)),
]


@pytest.mark.parametrize("grid,clusters", RESIDENT_CASES)
def test_resident_matches_oracle_and_streaming(P, oracle, grid, clusters):
    """The cluster-resident kernel (wavefield in distributed shared memory) against the
    oracle (FP32 tolerance) and against the streaming kernel, bit for bit: both evaluate
    the same factored node update with explicit multiply-adds."""
    w = W.tiny(**GRIDS[grid])
    th = _thetas(w, 4, seed=12)
    G = oracle.Grid.from_workload(w)
    ref = [oracle.forward(G, t) for t in th]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=30)
    assert ctx.resident_min_cluster == 1
    g_stream = torch.empty((4, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_stream)
    for C in clusters:
        ctx.set_tuning(C, 4, 4)
        g = torch.empty_like(g_stream)
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        for k in range(4):
            out = g[k].cpu().numpy()
            assert _normwise(out, ref[k]) <= 1e-4, (C, k, _normwise(out, ref[k]))
            # same node update with every rounding spelled out: identical bits
            assert np.array_equal(out, g_stream[k].cpu().numpy()), (C, k)
    # the gain through the resident path; the layered grid's FP32 pairs Jacobian loses too
    # many digits to cancellation, so there the difference form is used
    if grid != "homog_75x37":
        ctx.jacobian = P.OED_JAC_DIFFERENCE
    H = torch.empty((4, 7, 7), dtype=torch.float64, device=DEV)
    ctx.set_tuning(clusters[-1], 4, 4)
    sigma = 0.05
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
    dkl = torch.empty(4, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(np.full(4, 0.25)), w.prior_lo, w.prior_hi, eig, dkl=dkl)
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    for k in range(4):
        Href, _ = oracle.node_hessian(G, th[k], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, ok = oracle.scaled_logdet(Href)
        d_ref = oracle.dkl(ld, 7, lp)
        assert abs(float(dkl[k].item()) - d_ref) <= 1e-3 * abs(d_ref)


@pytest.mark.parametrize("prec,tol_h,tol_d", [(1, 1e-9, 1e-10), (0, None, 1e-4)])
def test_difference_jacobian_matches_oracle(P, oracle, prec, tol_h, tol_d):
    """The difference-form Jacobian (one solve per parameter driven by the FP64 forcing
    difference) against the oracle's literal +/- pairs.  Node 0 sits exactly on a grid
    node in x and z, so x_s - d and x_s + d fall in different cells (7-wide patch)."""
    w = W.tiny(**GRIDS["layered_70x41"])
    th = _thetas(w, 3, seed=21)
    th[0, 0] = 40 * w.h
    th[0, 1] = 18 * w.h
    G = oracle.Grid.from_workload(w)
    sigma = 0.05
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=14)   # chunks of 2 nodes
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    assert ctx.chunk_nodes == 2
    H = torch.empty((3, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.empty(3, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, status=st)
    dkl = torch.empty(3, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(np.full(3, 1 / 3)), w.prior_lo, w.prior_hi, eig, dkl=dkl)
    assert st.cpu().tolist() == [0, 0, 0]
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    for k in range(3):
        Href, _ = oracle.node_hessian(G, th[k], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        if tol_h:
            assert _scaled(H[k].cpu().numpy(), Href) <= tol_h
        ld, _, ok = oracle.scaled_logdet(Href)
        d_ref = oracle.dkl(ld, 7, lp)
        assert abs(float(dkl[k].item()) - d_ref) <= tol_d * abs(d_ref), (k, float(dkl[k].item()), d_ref)


@pytest.mark.parametrize("grid", sorted(GRIDS))
def test_tma_streaming_kernel_matches_oracle(P, oracle, grid):
    """The TMA-pipelined streaming kernel (halo tiles by cp.async.bulk.tensor into an
    mbarrier ring) against the oracle and the register streaming kernel."""
    w = W.tiny(**GRIDS[grid])
    th = _thetas(w, 5, seed=31)
    G = oracle.Grid.from_workload(w)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=35)
    g_ref = torch.empty((5, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_ref)
    ctx.set_tuning(-1, 4, 4)
    assert ctx.tuning[0] == -1
    g = torch.empty_like(g_ref)
    P.oed_forward(ctx, _t(th), g)
    torch.cuda.synchronize()
    for k in range(5):
        out = g[k].cpu().numpy()
        assert _normwise(out, oracle.forward(G, th[k])) <= 1e-4
        assert np.array_equal(out, g_ref[k].cpu().numpy()), k   # same node update, same bits
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    H = torch.empty((5, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.full((5,), -1, dtype=torch.int32, device=DEV)
    sigma = 0.05
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, status=st)
    assert st.cpu().tolist() == [0] * 5
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    for k in range(2):
        Href, _ = oracle.node_hessian(G, th[k], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, _ = oracle.scaled_logdet(Href)
        ldg, _, ok = oracle.scaled_logdet(H[k].cpu().numpy())
        assert ok and abs(oracle.dkl(ldg, 7, lp) - oracle.dkl(ld, 7, lp)) <= 1e-4 * abs(oracle.dkl(ld, 7, lp))


@pytest.mark.parametrize("prec", [1, 0])
def test_sensitivity_jacobian_matches_oracle(P, oracle, prec):
    """Algorithm 1 steps 1-5 (sensitivity solves driven by the analytic df/dtheta_j) against
    the oracle's own sensitivity H_I: FP64 to 1e-9 (scaled), FP32 D_KL-hat to 1e-4."""
    w = W.tiny(**GRIDS["layered_70x41"])
    th = _thetas(w, 3, seed=41)
    G = oracle.Grid.from_workload(w)
    sigma = 0.05
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=21)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    assert ctx.chunk_nodes == 3
    H = torch.empty((3, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.empty(3, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, status=st)
    assert st.cpu().tolist() == [0, 0, 0]
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    for k in range(3):
        Hs = oracle.node_hessian_sensitivity(G, th[k], sigma)
        if prec == 1:
            assert _scaled(H[k].cpu().numpy(), Hs) <= 1e-9
        ld, _, _ = oracle.scaled_logdet(Hs)
        ldg, _, ok = oracle.scaled_logdet(H[k].cpu().numpy())
        d_ref = oracle.dkl(ld, 7, lp)
        assert ok and abs(oracle.dkl(ldg, 7, lp) - d_ref) <= 1e-4 * abs(d_ref)


def test_resident_rejects_grids_that_do_not_fit(P):
    w = W.tiny(nx=801, nz=401, h=2.5, nsteps=2, nrec=3)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=15)
    assert ctx.resident_min_cluster == 0
    with pytest.raises(P.OedError):
        ctx.set_tuning(8, 4, 4)
    w64 = W.tiny(nx=401, nz=201, h=5.0, nsteps=2, nrec=3)
    ctx64 = P.Context(P.problem_from_workload(w64, P.OED_FP64), max_solves=15)
    assert ctx64.resident_min_cluster == 0


def test_status_invalid_source_and_not_pd(P):
    w = W.tiny(nx=41, nz=21, nsteps=40, nrec=3)
    th = _thetas(w, 3, seed=4)
    th[1, 1] = 5.0   # depth 5 m: the 6x6 patch leaves the grid through the surface
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=45)
    H = torch.empty((3, 7, 7), dtype=torch.float64, device=DEV)
    st = torch.empty(3, dtype=torch.int32, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H, status=st)
    assert st.cpu().tolist() == [0, P.OED_EINVAL, 0]
    assert torch.isnan(H[1]).all()
    # an indefinite matrix is flagged, excluded from the sum and counted
    H[2] = torch.eye(7, dtype=torch.float64, device=DEV)
    H[2, 2, 3] = H[2, 3, 2] = 1.5
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    s2 = torch.empty(3, dtype=torch.int32, device=DEV)
    nb = torch.empty(1, dtype=torch.int32, device=DEV)
    dkl = torch.empty(3, dtype=torch.float64, device=DEV)
    wt = _t([0.25, 0.25, 0.5])
    P.oed_eig(ctx, H, wt, w.prior_lo, w.prior_hi, eig, dkl=dkl, status=s2, n_bad=nb)
    assert s2.cpu().tolist() == [0, P.OED_ENOTPD, P.OED_ENOTPD]
    assert int(nb.item()) == 2
    assert abs(float(eig.item()) - 0.25 * float(dkl[0].item())) < 1e-12 * abs(float(eig.item()))


def test_designs_match_oracle(P, oracle):
    """EIG of receiver subsets from per-receiver, per-window partial Hessians.

    Two checks: (a) the design kernel's log-det / weighted sum equals the oracle's on the
    same partial Hessians (the GPU's own H_rec), tightly; (b) end to end against the
    oracle's H_rec within the EIG tolerance (few-receiver, short-window designs are
    ill-conditioned, so the ~1e-9 FD-Jacobian rounding grows to ~1e-4 in log det)."""
    w = W.tiny(nx=61, nz=25, h=33.0, nsteps=90, nrec=6, win_seconds=None)
    th = _thetas(w, 4, seed=8)
    wt = np.array([0.1, 0.2, 0.3, 0.4])
    wl = [46, w.nlevels]
    sigma = 0.05
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=60)
    H = torch.empty((4, 7, 7), dtype=torch.float64, device=DEV)
    Hr = torch.empty((4, w.nrec, 2, 28), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=wl, H_rec=Hr)
    rng = np.random.default_rng(0)
    masks = (rng.random((9, w.nrec)) < 0.5).astype(np.uint8)
    masks[0] = 1
    masks[1] = 0
    masks[1, 2] = 1
    G = oracle.Grid.from_workload(w)
    refs = [oracle.node_hessian(G, t, w.prior_lo, w.prior_hi, w.rel_step, sigma, wl)[1] for t in th]
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    iu = np.triu_indices(7)
    Hr_gpu = Hr.cpu().numpy()

    def unpack(v):
        M = np.zeros((7, 7))
        M[iu] = v
        return M + np.triu(M, 1).T

    def oracle_eig(get):
        """(EIG, rejected nodes, rounding bound sum_i |w_i| cond(Ht_i))."""
        tot, nbad, cnd = 0.0, 0, 0.0
        for i in range(4):
            Hd = sum((get(i, r) for r in sel), np.zeros((7, 7)))
            ld, Ht, ok = oracle.scaled_logdet(Hd)
            if ok:
                tot += wt[i] * oracle.dkl(ld, 7, lp)
                cnd += abs(wt[i]) * np.linalg.cond(Ht)
            else:
                nbad += 1
        return tot, nbad, cnd

    for win in (0, 1):
        eig = torch.empty(9, dtype=torch.float64, device=DEV)
        nb = torch.empty(9, dtype=torch.int32, device=DEV)
        P.oed_eig_designs(ctx, Hr, win, _t(masks, torch.uint8), _t(wt), w.prior_lo, w.prior_hi, eig, n_bad=nb)
        e = eig.cpu().numpy()
        bad = nb.cpu().numpy()
        for d in range(9):
            sel = np.nonzero(masks[d])[0]
            same, nbad, cnd = oracle_eig(lambda i, r: unpack(Hr_gpu[i, r, win]))
            assert bad[d] == nbad
            full, nbad_ref, _ = oracle_eig(lambda i, r: refs[i][r, win])
            assert nbad_ref == nbad
            if nbad:
                continue
            # log det of a matrix with condition number c moves by ~c * eps under rounding
            assert abs(e[d] - same) <= 1e-11 * max(1.0, abs(same)) + 1e-14 * cnd, (win, d, e[d], same, cnd)
            # end to end: the FD-Jacobian rounding (~1e-9 of H) is amplified the same way
            assert abs(e[d] - full) <= 1e-3 * abs(full) + 1e-9 * cnd, (win, d, e[d], full, cnd)
            if cnd < 1e8:
                assert abs(e[d] - full) <= 1e-6 * abs(full), (win, d, e[d], full, cnd)
    # all receivers over the full window equals the plain EIG
    e_all = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(wt), w.prior_lo, w.prior_hi, e_all)
    eig = torch.empty(9, dtype=torch.float64, device=DEV)
    P.oed_eig_designs(ctx, Hr, 1, _t(masks, torch.uint8), _t(wt), w.prior_lo, w.prior_hi, eig)
    assert abs(float(eig[0].item()) - float(e_all.item())) <= 1e-10 * abs(float(e_all.item()))


def test_eig_host_matches_device_path(P, oracle):
    w = W.tiny(nx=41, nz=21, nsteps=60, nrec=4, n_nodes=5)
    th, wt = oracle.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=45)
    e_host, dkl, nb = P.oed_eig_host(ctx, th, wt, w.prior_lo, w.prior_hi, w.rel_step, 0.1, want_dkl=True)
    H = torch.empty((5, 7, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, 0.1, H)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    P.oed_eig(ctx, H, _t(wt), w.prior_lo, w.prior_hi, eig)
    assert nb == 0
    assert e_host == float(eig.item())


def test_nodes_mc_matches_oracle(P, oracle):
    w = W.batched()
    u = w.uniforms()
    th = torch.empty((u.shape[0], 7), dtype=torch.float64, device=DEV)
    wt = torch.empty(u.shape[0], dtype=torch.float64, device=DEV)
    P.oed_nodes_mc(_t(u), w.prior_lo, w.prior_hi, th, wt)
    rt, rw = oracle.mc_nodes(u, w.prior_lo, w.prior_hi)
    assert np.allclose(th.cpu().numpy(), rt, rtol=1e-15, atol=0)
    assert np.allclose(wt.cpu().numpy(), rw, rtol=1e-15, atol=0)


@pytest.mark.slow
def test_full_size_batched_sampled(P, oracle):
    """401x201 grid, 2000 steps, 256 nodes x 15 solves in one launch configuration (the
    benchmark's): sampled seismograms and the gains of ten nodes spread over the prior box
    against the oracle (the mixed-precision bar, 1e-3)."""
    w = W.batched()
    th, wt = oracle.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    sigma = 0.5
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=3840)
    ctx.autotune(3840)   # the launch configuration the benchmark uses
    H = torch.empty((256, 7, 7), dtype=torch.float64, device=DEV)
    P.oed_hessian(ctx, _t(th), w.prior_lo, w.prior_hi, w.rel_step, sigma, H)
    dkl = torch.empty(256, dtype=torch.float64, device=DEV)
    eig = torch.empty(1, dtype=torch.float64, device=DEV)
    nb = torch.empty(1, dtype=torch.int32, device=DEV)
    P.oed_eig(ctx, H, _t(wt), w.prior_lo, w.prior_hi, eig, dkl=dkl, n_bad=nb)
    torch.cuda.synchronize()
    assert int(nb.item()) == 0
    G = oracle.Grid.from_workload(w)
    lp = oracle.log_uniform_density(w.prior_lo, w.prior_hi)
    # ten nodes spread over the prior box: nodes 0 and 1, then the nodes nearest both ends
    # of the x_s, z_s, t_s and omega_s intervals (a late, low-frequency source gives the
    # smallest signal and the largest FP32 cancellation in the pairs Jacobian)
    sample = W.spread_sample(th, w.prior_lo, w.prior_hi)
    assert len(sample) == 10
    d_gpu = dkl.cpu().numpy()
    errs = []
    for i in sample:
        Href, _ = oracle.node_hessian(G, th[i], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, ok = oracle.scaled_logdet(Href)
        assert ok
        d_ref = oracle.dkl(ld, 7, lp)
        errs.append((abs(d_gpu[i] - d_ref) / abs(d_ref), i, d_gpu[i], d_ref))
    assert max(errs)[0] <= 1e-3, max(errs)
    # seismograms of two solves of the same launch shape
    g = torch.empty((2, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th[[5, 200]]), g)
    for k, i in enumerate((5, 200)):
        assert _normwise(g[k].cpu().numpy(), oracle.forward(G, th[i])) <= 1e-4


def test_tma_kernel_many_tiles_per_cta_bitwise(P):
    """The TMA streaming kernel with several tiles per persistent CTA, so every stage of the
    ring is refilled and both consumer groups cycle through their stages: 401x201, 20 solves
    (1540 tiles over at most 304 CTAs), 400 steps (the waves reach the receivers), bit for
    bit against the register streaming kernel, twice (the second run replays the graph)."""
    w = W.tiny(nx=401, nz=201, h=5.0, nsteps=400, nrec=20)
    rng = np.random.default_rng(77)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * rng.random((20, 7))
    th[:, 2] = lo[2]   # earliest start
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=20)
    g_ref = torch.empty((20, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_ref)
    ctx.set_tuning(-1, 4, 4)
    g = torch.empty_like(g_ref)
    for _ in range(2):
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
    assert float(g_ref.abs().max()) > 1e-3


def test_resident_source_patch_across_slabs_bitwise(P):
    """The source term of the cluster-resident kernel is added by the edge warp after the march
    warps that own patch nodes arrive at a named barrier.  Patches that straddle a CTA's slab
    boundary (each CTA adds its own rows) or a row-segment boundary (two groups of march warps
    arrive), at clusters of 6, 7 and 8 CTAs (slabs of 34, 29 and 26 rows, segments of about a
    third of a slab), bit for bit against the register streaming kernel."""
    w = W.tiny(nx=401, nz=201, h=5.0, nsteps=480, nrec=12)
    lo = np.array(w.prior_lo)
    depths = [510.0, 570.0, 402.5, 595.0, 436.0, 468.0, 532.0, 451.0]   # rows 102, 114, 80, ...
    th = np.array([[800.0 + 50.0 * k, d, lo[2], 6.0, 5e13, 2e13, 7e13] for k, d in enumerate(depths)])
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=len(depths))
    ctx.set_tuning(0, 4, 4)
    g_ref = torch.empty((len(depths), w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_ref)
    for C in (6, 7, 8):
        ctx.set_tuning(C, 4, 4)
        g = torch.empty_like(g_ref)
        P.oed_forward(ctx, _t(th), g)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref), C
    assert float(g_ref.abs().max()) > 1e-3


def test_resident_one_row_per_cta(P, oracle):
    """Eight CTAs of one row each (nz = 8, clusters of 8): the surface row's south row, every
    north and south row and the absorbing bottom row's north row come from neighbouring CTAs'
    shared memory.  Against the oracle (FP32 bar) and bit for bit against the streaming kernel."""
    w = W.tiny(nx=40, nz=8, h=50.0, nsteps=80, nrec=3)
    th = np.array([[1000.0, 120.0, 0.1, 6.0, 5e13, 2e13, 8e13], [930.0, 140.0, 0.15, 7.0, 9e13, 4e13, 1e13]])
    G = oracle.Grid.from_workload(w)
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=4)
    g_ref = torch.empty((2, w.nlevels, w.nrec, 2), dtype=torch.float64, device=DEV)
    P.oed_forward(ctx, _t(th), g_ref)
    ctx.set_tuning(8, 4, 4)
    g = torch.empty_like(g_ref)
    P.oed_forward(ctx, _t(th), g)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref)
    for k in range(2):
        ref = oracle.forward(G, th[k])
        assert _normwise(g[k].cpu().numpy(), ref) <= 1e-4


def test_rebind_matches_a_fresh_context(P):
    """oed_rebind re-targets a context's workspace at a problem of the same grid shape with
    another step count, medium and receivers: seismograms and Hessians equal a fresh
    context's bit for bit; another shape is refused (OED_EINVAL), a problem whose workspace
    does not fit is refused (OED_ENOMEM) and the context still works."""
    w1 = W.tiny(nx=81, nz=41, h=25.0, nsteps=120, nrec=5)
    w2 = W.tiny(nx=81, nz=41, h=25.0, nsteps=90, nrec=3, layers=W.THREE_LAYER)
    th = np.array([[1000.0, 480.0, 0.12, 6.0, 5e13, 2e13, 7e13], [950.0, 520.0, 0.2, 5.0, 3e13, 6e13, 2e13]])
    for prec in (P.OED_FP32, P.OED_FP64):
        ctx = P.Context(P.problem_from_workload(w1, prec), max_solves=30)
        g1 = torch.empty((2, w1.nlevels, w1.nrec, 2), dtype=torch.float64, device=DEV)
        P.oed_forward(ctx, _t(th), g1)
        torch.cuda.synchronize()   # oed_rebind wants the context's earlier work finished
        assert not torch.isnan(g1).any(), prec
        ctx.rebind(P.problem_from_workload(w2, prec))
        g2 = torch.empty((2, w2.nlevels, w2.nrec, 2), dtype=torch.float64, device=DEV)
        P.oed_forward(ctx, _t(th), g2)
        H2 = torch.empty((2, 7, 7), dtype=torch.float64, device=DEV)
        P.oed_hessian(ctx, _t(th), w2.prior_lo, w2.prior_hi, w2.rel_step, 0.05, H2)
        fresh = P.Context(P.problem_from_workload(w2, prec), max_solves=30)
        g2f = torch.empty_like(g2)
        P.oed_forward(fresh, _t(th), g2f)
        H2f = torch.empty_like(H2)
        P.oed_hessian(fresh, _t(th), w2.prior_lo, w2.prior_hi, w2.rel_step, 0.05, H2f)
        torch.cuda.synchronize()
        assert torch.equal(g2, g2f) and torch.equal(H2, H2f)
        with pytest.raises(P.OedError) as e:
            ctx.rebind(P.problem_from_workload(W.tiny(nx=61, nz=41, h=25.0, nsteps=90, nrec=3), prec))
        assert e.value.code == P.OED_EINVAL
        with pytest.raises(P.OedError) as e:   # a longer record needs a larger workspace
            ctx.rebind(P.problem_from_workload(W.tiny(nx=81, nz=41, h=25.0, nsteps=4000, nrec=5), prec))
        assert e.value.code == P.OED_ENOMEM
        ctx.rebind(P.problem_from_workload(w1, prec))
        g1b = torch.empty_like(g1)
        P.oed_forward(ctx, _t(th), g1b)
        torch.cuda.synchronize()
        assert torch.equal(g1, g1b)
        fresh.close()
        ctx.close()
