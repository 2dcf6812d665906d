"""Structured polar meshes and run parameters for a 2D coaxial-cable cross-section.

Geometry (the paper's cable model of Sec. 4 is not specified, so this stands
in for it): a stranded copper core ``r < 1 mm`` carrying an impressed uniform
current density, insulation ``1-2 mm``, a solid steel sheath ``2-2.5 mm``
(conductive, nonlinear Brauer reluctivity) and air out to ``4 mm`` where the
vector potential is fixed to zero.

Mesh: a centre node plus ``nr`` rings of ``ntheta`` nodes; the outermost ring
is the Dirichlet boundary.  Radial intervals are shared among the four regions
in proportion to their thickness (1 : 1 : 0.5 : 1.5), with at least two in the
sheath.  Node ``(i, j)`` (ring ``i >= 1``, sector ``j``) has global index
``1 + (i - 1) * ntheta + j``; node 0 is the centre.  Every quad cell is split
along the same diagonal, giving ``ntheta + 2 * ntheta * (nr - 1)`` triangles,
all counter-clockwise.  Nodes on rings strictly inside a region are jittered
by at most ``jitter`` times the local radial and angular spacing, drawn from
``numpy.random.default_rng(seed)``; the centre, the region interfaces and the
outer ring stay on their nominal circles.

Only data is produced here.  Element integrals, time stepping and solves live
in the oracle and in the CUDA library, which share none of their code.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NU0 = 1.0 / (4.0e-7 * math.pi)          # reluctivity of vacuum [m/H]
RADII = (1.0e-3, 2.0e-3, 2.5e-3, 4.0e-3)  # outer radii of core, insulation, sheath, air [m]
_THICKNESS_HALF_MM = (2, 2, 1, 3)         # region thicknesses in units of 0.5 mm
REGION_CORE, REGION_INSULATION, REGION_SHEATH, REGION_AIR = 0, 1, 2, 3
BRAUER_STEEL = (3.8, 2.17, 396.2)         # nu(B^2) = k1 * exp(k2 * B^2) + k3
BRAUER_BMAX = 3.0                         # |B| [T] past which the fit continues along its tangent

NU_LINEAR, NU_BRAUER = 0, 1


def radial_intervals(nr: int, min_sheath: int = 2) -> tuple[int, int, int, int]:
    """Split ``nr`` radial intervals among core, insulation, sheath and air.

    Largest-remainder rounding of ``nr`` times the thickness fractions, in
    integer arithmetic so that ties break the same way on every machine (ties
    go to the lower region index among equal remainders, after the sheath).
    Every region then gets at least one interval and the sheath at least
    ``min_sheath``, taken from the region with the most intervals.
    """
    w = _THICKNESS_HALF_MM
    total = sum(w)
    if nr < 3 + min_sheath:
        raise ValueError(f"nr={nr} too small: need >= {3 + min_sheath} radial intervals")
    counts = [nr * wk // total for wk in w]
    rem = [nr * wk % total for wk in w]
    order = sorted(range(4), key=lambda k: (-rem[k], 0 if k == REGION_SHEATH else 1, k))
    for k in order[: nr - sum(counts)]:
        counts[k] += 1
    need = {k: 1 for k in range(4)}
    need[REGION_SHEATH] = min_sheath
    for k in range(4):
        while counts[k] < need[k]:
            donor = max((d for d in range(4) if d != k and counts[d] > need[d]),
                        key=lambda d: (counts[d], -d))
            counts[donor] -= 1
            counts[k] += 1
    assert sum(counts) == nr
    return tuple(counts)  # type: ignore[return-value]


@dataclass
class CoaxMesh:
    xy: np.ndarray          # (n_nodes, 2) float64, metres
    tri: np.ndarray         # (n_tri, 3) int32, counter-clockwise
    region: np.ndarray      # (n_tri,) int32, REGION_*
    dirichlet: np.ndarray   # (n_nodes,) uint8, 1 on the outer ring
    nr: int
    ntheta: int
    counts: tuple           # radial intervals per region
    ring_radius: np.ndarray  # (nr + 1,) nominal ring radii, ring 0 = centre

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_tri(self) -> int:
        return self.tri.shape[0]

    @property
    def ndof(self) -> int:
        return int(self.n_nodes - int(self.dirichlet.sum()))


def _node(i: int, j, ntheta: int):
    return 1 + (i - 1) * ntheta + np.mod(j, ntheta)


def coax_mesh(nr: int, ntheta: int, seed: int = 0, jitter: float = 0.10) -> CoaxMesh:
    """Seeded structured polar triangulation of the coax cross-section."""
    if ntheta < 3:
        raise ValueError("ntheta must be >= 3")
    counts = radial_intervals(nr)
    bounds = np.concatenate([[0], np.cumsum(counts)])          # ring index of each interface
    r_inner = (0.0,) + RADII[:3]
    ring_radius = np.zeros(nr + 1)
    ring_region = np.zeros(nr + 1, dtype=np.int64)              # region whose interior holds the ring
    ring_dr = np.zeros(nr + 1)
    for k in range(4):
        for i in range(bounds[k], bounds[k + 1] + 1):
            ring_radius[i] = r_inner[k] + (i - bounds[k]) * (RADII[k] - r_inner[k]) / counts[k]
        for i in range(bounds[k] + 1, bounds[k + 1]):
            ring_region[i] = k
            ring_dr[i] = (RADII[k] - r_inner[k]) / counts[k]
    interface = np.zeros(nr + 1, dtype=bool)
    interface[bounds] = True

    n_nodes = 1 + nr * ntheta
    rng = np.random.default_rng(seed)
    draw = rng.uniform(-1.0, 1.0, size=(n_nodes, 2))

    dtheta = 2.0 * math.pi / ntheta
    xy = np.zeros((n_nodes, 2))
    j = np.arange(ntheta)
    for i in range(1, nr + 1):
        idx = _node(i, j, ntheta)
        r = np.full(ntheta, ring_radius[i])
        th = j * dtheta
        if not interface[i] and jitter > 0.0:
            r = r + jitter * ring_dr[i] * draw[idx, 0]
            th = th + jitter * dtheta * draw[idx, 1]
        xy[idx, 0] = r * np.cos(th)
        xy[idx, 1] = r * np.sin(th)

    tris = []
    regs = []
    # centre fan (radial interval 0 belongs to the core)
    fan = np.stack([np.zeros(ntheta, dtype=np.int64), _node(1, j, ntheta), _node(1, j + 1, ntheta)], axis=1)
    tris.append(fan)
    regs.append(np.full(ntheta, REGION_CORE))
    for q in range(1, nr):
        k = int(np.searchsorted(bounds, q, side="right") - 1)
        a = _node(q, j, ntheta)
        b = _node(q + 1, j, ntheta)
        c = _node(q + 1, j + 1, ntheta)
        d = _node(q, j + 1, ntheta)
        t1 = np.stack([a, b, c], axis=1)
        t2 = np.stack([a, c, d], axis=1)
        tris.append(np.stack([t1, t2], axis=1).reshape(-1, 3))
        regs.append(np.full(2 * ntheta, k))
    tri = np.concatenate(tris).astype(np.int32)
    region = np.concatenate(regs).astype(np.int32)
    dirichlet = np.zeros(n_nodes, dtype=np.uint8)
    dirichlet[_node(nr, j, ntheta)] = 1
    return CoaxMesh(xy=xy, tri=tri, region=region, dirichlet=dirichlet, nr=nr, ntheta=ntheta,
                    counts=counts, ring_radius=ring_radius)


@dataclass
class Problem:
    """One periodic eddy-current run: mesh, per-region materials, excitation, time grid."""

    name: str
    mesh: CoaxMesh
    sigma: np.ndarray        # (4,) conductivity per region [S/m]
    nu_model: np.ndarray     # (4,) NU_LINEAR or NU_BRAUER
    nu: np.ndarray           # (4,) linear reluctivity [m/H] (used when NU_LINEAR)
    brauer: np.ndarray       # (4, 3) k1, k2, k3 (used when NU_BRAUER)
    is_source: np.ndarray    # (4,) 1 where the impressed current flows
    amp: np.ndarray          # (n_harm,) current amplitudes [A]
    freq: np.ndarray         # (n_harm,) frequencies [Hz]
    phase: np.ndarray        # (n_harm,) phases [rad]
    T: float = 0.02          # period [s]
    N: int = 16              # subintervals
    n_fine: int = 20         # fine implicit-Euler steps per subinterval
    kmax: int = 10
    extra: dict = field(default_factory=dict)
    bmax: np.ndarray = None  # (4,) |B| [T] past which the Brauer fit continues linearly in B^2 (0: never)

    def __post_init__(self):
        if self.bmax is None:
            self.bmax = np.zeros(4)

    @property
    def L(self) -> int:
        return self.N * self.n_fine


def make_problem(name: str, nr: int, ntheta: int, N: int, n_fine: int, sigma_sheath: float,
                 amp=(10.0,), freq=(50.0,), phase=None, seed: int = 0, T: float = 0.02,
                 kmax: int = 10, linear_sheath: bool = False, jitter: float = 0.10,
                 bmax: float = BRAUER_BMAX) -> Problem:
    mesh = coax_mesh(nr, ntheta, seed=seed, jitter=jitter)
    sigma = np.array([0.0, 0.0, sigma_sheath, 0.0])
    nu_model = np.array([NU_LINEAR, NU_LINEAR, NU_LINEAR if linear_sheath else NU_BRAUER, NU_LINEAR],
                        dtype=np.int32)
    k1, k2, k3 = BRAUER_STEEL
    nu = np.array([NU0, NU0, k1 + k3, NU0])       # linear sheath uses the small-field Brauer value
    brauer = np.zeros((4, 3))
    brauer[REGION_SHEATH] = BRAUER_STEEL
    is_source = np.array([1, 0, 0, 0], dtype=np.int32)
    amp = np.asarray(amp, dtype=np.float64)
    freq = np.asarray(freq, dtype=np.float64)
    phase = np.zeros_like(amp) if phase is None else np.asarray(phase, dtype=np.float64)
    bm = np.zeros(4)
    bm[REGION_SHEATH] = bmax
    return Problem(name=name, mesh=mesh, sigma=sigma, nu_model=nu_model, nu=nu, brauer=brauer,
                   is_source=is_source, amp=amp, freq=freq, phase=phase, T=T, N=N,
                   n_fine=n_fine, kmax=kmax, bmax=bm)


# Workloads by name.  Sizes follow the coax cases the method is exercised on:
# the small FP64 case, the medium nonlinear case, the adjoint case, the large
# case, the paper-shaped case (2269 DOFs, N=20, 100 fine steps per
# subinterval, Sec. 4) and a tiny case for brute-force checks.
WORKLOADS = {
    "tiny":    dict(nr=5, ntheta=8, N=4, n_fine=3, sigma_sheath=5e6),
    "small":   dict(nr=20, ntheta=40, N=16, n_fine=20, sigma_sheath=5e6),
    "medium":  dict(nr=100, ntheta=200, N=64, n_fine=50, sigma_sheath=2e7),
    "adjoint": dict(nr=160, ntheta=320, N=128, n_fine=40, sigma_sheath=2e7),
    "large":   dict(nr=500, ntheta=1000, N=256, n_fine=200, sigma_sheath=3e7,
                    amp=(40.0, 8.0), freq=(50.0, 150.0)),
    "paper":   dict(nr=28, ntheta=84, N=20, n_fine=100, sigma_sheath=5e6),
}


def workload(name: str, **over) -> Problem:
    params = dict(WORKLOADS[name])
    params.update(over)
    return make_problem(name, **params)


def batched_cables(count: int = 32, seed: int = 2026) -> list[Problem]:
    """Independent cables of uneven size: nr in [20,200], ntheta in [40,400],
    amplitude in [1,50] A, sheath sigma log-uniform in [1e6,3e7] S/m,
    N in {16,32,64}, 20-50 fine steps per subinterval."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        nr = int(rng.integers(20, 201))
        nth = int(rng.integers(40, 401))
        amp = float(rng.uniform(1.0, 50.0))
        sig = float(10.0 ** rng.uniform(6.0, math.log10(3e7)))
        N = int(rng.choice([16, 32, 64]))
        nf = int(rng.integers(20, 51))
        out.append(make_problem(f"cable{c}", nr, nth, N, nf, sig, amp=(amp,), seed=seed + c))
    return out
