"""Seeded synthetic workloads for the Laplace expected-information-gain path.

This module is shared by the CUDA path, the CPU oracle and the tests.  It holds
only input *descriptions* and seeded random draws: grid sizes, layer tables,
receiver node indices, prior boxes and uniform variates.  None of the method's
arithmetic (Lame parameters, source discretisation, time stepping, Jacobians,
Hessians, log-determinants, quadrature rules) lives here; each side computes
those itself.

Physical setting (Sec. 2.1 and Sec. 4.1 of the paper, restated for the synthetic
workloads): a 2-D isotropic elastic half-plane, x horizontal in [0, Lx], depth z
in [0, Lz] with z = 0 the free surface, first-order absorbing boundaries on the
two sides and the bottom, a point moment-tensor source with a Gaussian time
function, receivers on surface grid nodes.  The parameter vector follows the
paper's order theta = (x_s, z_s, t_s, omega_s, m_xx, m_xz, m_zz).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

NTHETA = 7
THETA_NAMES = ("x_s", "z_s", "t_s", "omega_s", "m_xx", "m_xz", "m_zz")

# Uniform prior box used by every synthetic workload: source position in metres
# (z is depth), start time in s, frequency parameter in 1/s, moments in N*m.
PRIOR_LO = (800.0, 400.0, 0.1, 4.0, 1e13, 1e13, 1e13)
PRIOR_HI = (1200.0, 600.0, 0.3, 8.0, 1e14, 1e14, 1e14)

HOMOGENEOUS = ((0.0, 3000.0, 1732.0, 2500.0),)          # (z_top, vp, vs, rho)
THREE_LAYER = ((0.0, 2000.0, 1155.0, 2200.0),
               (300.0, 3000.0, 1732.0, 2500.0),
               (600.0, 4500.0, 2598.0, 2700.0))


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, medium, receivers, prior and node draws."""
    name: str
    nx: int
    nz: int
    h: float
    nsteps: int
    dt: float
    layers: tuple                  # ((z_top, vp, vs, rho), ...) with z_top increasing
    rec_ix: List[int]              # surface node index of every receiver
    prior_lo: tuple = PRIOR_LO
    prior_hi: tuple = PRIOR_HI
    rel_step: float = 1e-4         # FD step as a fraction of each prior width
    sigma_frac: float = 0.01       # noise std as a fraction of the peak surface amplitude
    n_nodes: int = 0
    node_rule: str = "mc"          # "mc" or "smolyak"
    smolyak_level: int = 3
    seed: int = 0
    win_seconds: Optional[Sequence[float]] = None

    @property
    def nlevels(self) -> int:
        return self.nsteps + 1

    @property
    def nrec(self) -> int:
        return len(self.rec_ix)

    @property
    def cells(self) -> int:
        return self.nx * self.nz

    def win_levels(self) -> List[int]:
        """Number of time levels (t_0 = 0 included) inside each window [0, T_w]."""
        if not self.win_seconds:
            return [self.nlevels]
        return [min(self.nlevels, int(math.floor(t / self.dt + 1e-9)) + 1)
                for t in self.win_seconds]

    def uniforms(self, n: Optional[int] = None, seed: Optional[int] = None) -> np.ndarray:
        """Seeded U(0,1) variates, shape [n][7]; the node rule maps them to the prior box."""
        n = self.n_nodes if n is None else n
        rng = np.random.default_rng(self.seed if seed is None else seed)
        return rng.random((n, NTHETA))

    def layer_arrays(self):
        z_top = np.array([l[0] for l in self.layers], dtype=np.float64)
        vp = np.array([l[1] for l in self.layers], dtype=np.float64)
        vs = np.array([l[2] for l in self.layers], dtype=np.float64)
        rho = np.array([l[3] for l in self.layers], dtype=np.float64)
        return z_top, vp, vs, rho


def surface_receivers(nx: int, h: float, nrec: int) -> List[int]:
    """Evenly spaced surface receivers: x_r = (r + 1/2) Lx / N_R snapped to the nearest node."""
    lx = (nx - 1) * h
    return [int(math.floor((r + 0.5) * lx / nrec / h + 0.5)) for r in range(nrec)]


def make(name: str, *, nx: int, nz: int, h: float, nsteps: int, layers=HOMOGENEOUS,
         nrec: int = 5, cfl: float = 0.5, **kw) -> Workload:
    vp_max = max(l[1] for l in layers)
    dt = cfl * h / vp_max
    return Workload(name=name, nx=nx, nz=nz, h=h, nsteps=nsteps, dt=dt, layers=tuple(layers),
                    rec_ix=surface_receivers(nx, h, nrec), **kw)


def plain_small() -> Workload:
    """81x41 grid, h = 25 m, 400 steps, 5 receivers, 16 MC nodes (seed 1): 240 solves."""
    return make("plain_small_81x41_fp64", nx=81, nz=41, h=25.0, nsteps=400, nrec=5,
                n_nodes=16, seed=1)


def batched() -> Workload:
    """401x201 grid, h = 5 m, 2000 steps, 20 receivers, 256 MC nodes (seed 2): 3840 solves."""
    return make("batched_401x201_2000steps_256nodes", nx=401, nz=201, h=5.0, nsteps=2000,
                nrec=20, n_nodes=256, seed=2)


def layered() -> Workload:
    """801x401 grid, h = 2.5 m, 3 layers, 4000 steps, 40 receivers, Smolyak level 3 (589 nodes)."""
    return make("layered_801x401_4000steps_smolyak3", nx=801, nz=401, h=2.5, nsteps=4000,
                layers=THREE_LAYER, nrec=40, node_rule="smolyak", smolyak_level=3, seed=3)


def design_sweep() -> Workload:
    """401x201 grid to T = 2 s (2400 steps), 40 candidate receivers, 1024 MC nodes (seed 4),
    windows T in {0.5, 1, 2} s."""
    return make("design_sweep_401x201_1024nodes", nx=401, nz=201, h=5.0, nsteps=2400, nrec=40,
                n_nodes=1024, seed=4, win_seconds=(0.5, 1.0, 2.0))


def design_subsets(nrec: int = 40, kmax: int = 10, per_k: int = 512, seed: int = 4) -> np.ndarray:
    """Seeded receiver subsets: for k = 1..kmax, per_k random k-subsets of nrec candidates.
    Returns a uint8 mask [kmax*per_k][nrec]."""
    rng = np.random.default_rng(seed + 1000)
    masks = np.zeros((kmax * per_k, nrec), dtype=np.uint8)
    for k in range(1, kmax + 1):
        for s in range(per_k):
            masks[(k - 1) * per_k + s, rng.choice(nrec, size=k, replace=False)] = 1
    return masks


def spread_sample(theta: np.ndarray, lo, hi, first=(0, 1), params=(0, 1, 2, 3)) -> List[int]:
    """Indices of nodes spread over the prior box, for sampled checks of a batch: the
    nodes in `first`, then for each parameter in `params` (default x_s, z_s, t_s,
    omega_s) the node nearest the low end and the node nearest the high end of its
    prior interval, skipping repeats (up to len(first) + 2 len(params) nodes)."""
    u = (np.asarray(theta) - np.asarray(lo)) / (np.asarray(hi) - np.asarray(lo))
    out = [int(i) for i in first if 0 <= int(i) < u.shape[0]]
    for j in params:
        for order in (np.argsort(u[:, j], kind="stable"), np.argsort(-u[:, j], kind="stable")):
            for i in order:
                if int(i) not in out:
                    out.append(int(i))
                    break
    return out


SERVING_GRIDS = ((201, 101, 10.0), (401, 201, 5.0), (801, 401, 2.5), (1601, 801, 1.25))


def serving_requests(n: int, rate_hz: float = 50.0, seed: int = 5, t_end: float = 0.5,
                     grids=SERVING_GRIDS, m_range=(64, 2048), nrec_range=(5, 40)):
    """Seeded Poisson arrivals of EIG requests mixing grid sizes, node counts, receiver
    counts and homogeneous / 3-layer media.  Each request integrates to T = t_end seconds."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    out = []
    for i in range(n):
        nx, nz, h = grids[int(rng.integers(len(grids)))]
        layers = THREE_LAYER if rng.random() < 0.5 else HOMOGENEOUS
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        nrec = int(rng.integers(nrec_range[0], nrec_range[1] + 1))
        vp_max = max(l[1] for l in layers)
        dt = 0.5 * h / vp_max
        nsteps = int(math.ceil(t_end / dt))
        w = Workload(name=f"req{i}", nx=nx, nz=nz, h=h, nsteps=nsteps, dt=dt, layers=layers,
                     rec_ix=surface_receivers(nx, h, nrec), n_nodes=m, seed=seed * 100003 + i)
        out.append((float(t[i]), w))
    return out


def tiny(nx=41, nz=21, h=50.0, nsteps=100, nrec=5, n_nodes=2, seed=11, layers=HOMOGENEOUS,
         **kw) -> Workload:
    """Small grid used by unit tests (a few tiles and a ragged tail on the GPU)."""
    return make(f"tiny_{nx}x{nz}", nx=nx, nz=nz, h=h, nsteps=nsteps, nrec=nrec, layers=layers,
                n_nodes=n_nodes, seed=seed, **kw)


# The paper's own model problem (Sec. 4.1): a two-layer LOH.1-like box
# [-10000, 10000] x [-15000, 0] m, here shifted to x in [0, 20000] and depth in
# [0, 15000]; top layer 1000 m thick.  h = 200 m, dt = 0.025 s, T = 8 s (321 levels),
# C_eps = 1e-4 I (sigma = 0.01).  Priors (Sec. 4.1) in the shifted coordinates.
PAPER_LAYERS = ((0.0, 4000.0, 2000.0, 2600.0), (1000.0, 6000.0, 3464.0, 2700.0))
PAPER_PRIOR_LO = (9000.0, 1000.0, 0.5, 3.0, 1e13, 1e13, 1e13)
PAPER_PRIOR_HI = (11000.0, 3000.0, 1.5, 5.0, 1e15, 1e15, 1e15)
PAPER_PRIOR_MEAN = (10000.0, 2000.0, 1.0, 4.0, 1e14, 1e14, 1e14)


PAPER_CANDIDATES = tuple(range(-9000, 9001, 200))   # x_1 of every candidate receiver


def paper_model(n_nodes: int = 0, seed: int = 6) -> Workload:
    """The paper's model problem with the 91 candidate receivers its scenarios use: every
    surface node with x_1 in [-9000, 9000] m (x = 1000 .. 19000 m here, 200 m apart)."""
    h = 200.0
    return Workload(name="paper_loh_101x76_320steps", nx=101, nz=76, h=h, nsteps=320, dt=0.025,
                    layers=PAPER_LAYERS, rec_ix=[int((x1 + 10000.0) / h) for x1 in PAPER_CANDIDATES],
                    prior_lo=PAPER_PRIOR_LO, prior_hi=PAPER_PRIOR_HI, n_nodes=n_nodes, seed=seed)


def paper_scenarios():
    """Receiver designs of Sec. 4.5 as masks over the candidates of paper_model().
    Returns a list of (scenario, parameter value, mask)."""
    cand = list(PAPER_CANDIDATES)

    def mask(positions):
        m = np.zeros(len(cand), dtype=np.uint8)
        for x in positions:
            m[cand.index(int(round(x)))] = 1
        return m

    out = []
    for nr, dr in zip((3, 5, 9, 17, 41, 81), (8000, 4000, 2000, 1000, 400, 200)):   # Scenario I
        out.append(("I", nr, mask([(k - (nr - 1) / 2) * dr for k in range(nr)])))
    for nr in range(1, 20, 2):                                                       # Scenario II
        out.append(("II", nr, mask([(k - (nr - 1) / 2) * 1000 for k in range(nr)])))
    for dr in range(200, 4001, 200):                                                 # Scenario III
        out.append(("III", dr, mask([(k - 2) * dr for k in range(5)])))
    return out


# Sec. 4.3-4.4: three unknowns (theta_2 = depth, theta_4 = omega, theta_5 = m_xx), the other
# four known: theta_1 = -1000 m (x = 9000 m here), theta_3 = 1 s, theta_6 = theta_7 = 1e14.
PAPER_STUDY_UNKNOWN = (1, 3, 4)
PAPER_STUDY_KNOWN = (9000.0, 2000.0, 1.0, 4.0, 1e14, 1e14, 1e14)   # unknown entries unused


def paper_study_model() -> Workload:
    """Sec. 4.4's setting: the model problem observed for T = 1.25 s (50 steps) at two
    receivers, x_1 = -9000 m and x_1 = 1000 m (x = 1000 m and 11000 m here)."""
    w = paper_model()
    return Workload(name="paper_loh_101x76_50steps_2rec", nx=w.nx, nz=w.nz, h=w.h, nsteps=50, dt=w.dt,
                    layers=w.layers, rec_ix=[5, 55], prior_lo=w.prior_lo, prior_hi=w.prior_hi)


def paper_study_thetas(u: np.ndarray, unknown=PAPER_STUDY_UNKNOWN) -> np.ndarray:
    """Full parameter vectors from uniform variates u[n][len(unknown)] of the unknowns (the
    others take their known values)."""
    lo, hi = np.array(PAPER_PRIOR_LO), np.array(PAPER_PRIOR_HI)
    th = np.tile(np.array(PAPER_STUDY_KNOWN), (u.shape[0], 1))
    for k, j in enumerate(unknown):
        th[:, j] = lo[j] + (hi[j] - lo[j]) * u[:, k]
    return th


ALL = {"plain_small": plain_small, "batched": batched, "layered": layered,
       "design_sweep": design_sweep}
