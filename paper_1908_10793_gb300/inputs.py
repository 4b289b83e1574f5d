"""Seeded synthetic workloads for the dust drag-coupling step.

This module only draws random numbers and lays out arrays.  It holds none of
the method's arithmetic and is the one piece shared by the oracle-side tests
and the CUDA-side tests and benchmark.

Every workload stands in for a setup of the paper (no dataset is involved):

* ``box2d``      2-D Cartesian periodic box, 64x64 zones, 16,384 grains, gas at
                 rest density 1 moving with (0.3, -0.2); tau_s = 0.1, dt = 0.01,
                 100 steps, TSC, feedback on (the deceleration setup of Sec. 4.1
                 on a grid).
* ``sbox3d``     3-D shearing box (orbital-advection frame), 128^3 zones,
                 8 grains per zone (16.8M), St = 0.1, dust-to-gas ratio 0.02,
                 residual gas velocity N(0, 1e-3) per component (Secs. 2.1, 4.3).
* ``cyldisk``    cylindrical global disk, (R, phi, z) = 384 x 1024 x 64 zones,
                 log-spaced R in [0.4, 2.5], Sigma ~ 1/R, Keplerian gas with 1e-3
                 noise, 50M grains in 4 species St in {0.01, 0.1, 1, 10}
                 (Secs. 4.5, 4.8).
* ``sphdisk``    spherical disk, (r, theta, phi) = 256 x 128 x 512 zones,
                 log-spaced r in [0.5, 3], theta within 0.3 of the midplane,
                 rho ~ r^-1.5 exp(-cot^2(theta) / (2 h^2)), h = 0.05, 33M
                 grains with log-uniform St in [1e-4, 10] (Sec. 4.6).
* ``si2d_batch`` 64 axisymmetric streaming-instability shearing boxes (x, z),
                 32^2 .. 512^2 zones, 1-16 grains per zone, NSH equilibrium
                 (Eq. SI_equil) with eta v_K = 0.05 c_s plus 1e-3 noise.

``scale="small"`` gives reduced grids with the same structure, for tests that
the oracle finishes in seconds.

Constants below use the numeric values of the C interface (geometry kinds,
boundary kinds, weight kinds, stopping-time modes).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

CARTESIAN, SHEARING_BOX, CYLINDRICAL, SPHERICAL = 0, 1, 2, 3
PERIODIC, OUTFLOW = 0, 1
CIC, TSC, VOLUME = 0, 1, 2
TAU_CONST, TAU_STOKES, TAU_EPSTEIN = 0, 1, 2

BASE_SEED = 20190828


@dataclass
class Workload:
    name: str
    geom: int
    edges: List[np.ndarray]
    bc: List[int]
    weight: int
    species_mass: List[float]
    species_tau_mode: List[int]
    species_tau: List[float]
    rho: np.ndarray              # [ncell] zone index i + n0 (j + n1 k)
    vgas: List[np.ndarray]       # physical gas velocity components, [ncell] each
    q: List[np.ndarray]          # grain coordinates (float64)
    v: List[np.ndarray]          # grain physical velocity components (float64)
    dt: float
    steps: int
    feedback: int
    species: Optional[np.ndarray] = None   # uint8 per grain, or None
    param: Optional[np.ndarray] = None     # float64 per grain, or None
    fargo: int = 0
    omega: float = 1.0
    qshear: float = 1.5
    gm: float = 0.0
    vertical_gravity: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def n(self):
        return [len(e) - 1 for e in self.edges]

    @property
    def ncell(self):
        n = self.n
        return n[0] * n[1] * n[2]

    @property
    def ngrains(self):
        return len(self.q[0])


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def _uniform_edges(lo, hi, n):
    return lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n


def _log_edges(lo, hi, n):
    e = lo * (hi / lo) ** (np.arange(n + 1, dtype=np.float64) / n)
    e[0], e[-1] = lo, hi
    return e


def _centres(e):
    return 0.5 * (e[:-1] + e[1:])


def _grid3(edges):
    """Zone-centre coordinate arrays flattened in i + n0 (j + n1 k) order."""
    c = [_centres(e) for e in edges]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def box2d(scale="full", seed=BASE_SEED + 0):
    """2-D Cartesian periodic box, 64^2 zones, 4 grains per zone."""
    r = _rng(seed)
    nx = 64 if scale == "full" else 16
    ng = 16384 if scale == "full" else 1024
    edges = [_uniform_edges(0.0, 1.0, nx), _uniform_edges(0.0, 1.0, nx),
             np.array([0.0, 1.0])]
    ncell = nx * nx
    q = [r.uniform(0.0, 1.0, ng), r.uniform(0.0, 1.0, ng), np.full(ng, 0.5)]
    v = [r.standard_normal(ng), r.standard_normal(ng), np.zeros(ng)]
    return Workload(
        name="box2d", geom=CARTESIAN, edges=edges, bc=[PERIODIC] * 3, weight=TSC,
        species_mass=[1.0 / ng], species_tau_mode=[TAU_CONST], species_tau=[0.1],
        rho=np.ones(ncell), vgas=[np.full(ncell, 0.3), np.full(ncell, -0.2), np.zeros(ncell)],
        q=q, v=v, dt=0.01, steps=100, feedback=1,
        notes={"dust_to_gas": 1.0, "grains_per_zone": ng / ncell})


def _per_zone_positions(r, edges, ppc):
    """ppc grains per zone, uniform inside each zone, zones in storage order."""
    n = [len(e) - 1 for e in edges]
    ncell = n[0] * n[1] * n[2]
    cell = np.repeat(np.arange(ncell, dtype=np.int64), ppc)
    i = cell % n[0]
    j = (cell // n[0]) % n[1]
    k = cell // (n[0] * n[1])
    q = []
    for d, idx in enumerate((i, j, k)):
        lo = edges[d][idx]
        hi = edges[d][idx + 1]
        q.append(lo + (hi - lo) * r.uniform(0.0, 1.0, len(cell)))
    return q


def sbox3d(scale="full", seed=BASE_SEED + 1, ppc=8):
    """3-D shearing box in the orbital-advection frame, 128^3 zones."""
    r = _rng(seed)
    n = 128 if scale == "full" else (16 if scale == "small" else int(scale))
    L = 0.2
    edges = [_uniform_edges(-0.5 * L, 0.5 * L, n) for _ in range(3)]
    ncell = n ** 3
    q = _per_zone_positions(r, edges, ppc)
    ng = len(q[0])
    amp = 1e-3
    v = [amp * r.standard_normal(ng) for _ in range(3)]
    vgas = [amp * r.standard_normal(ncell) for _ in range(3)]
    dV = (L / n) ** 3
    mass = 0.02 * 1.0 * dV / ppc
    return Workload(
        name="sbox3d", geom=SHEARING_BOX, edges=edges, bc=[PERIODIC] * 3, weight=TSC,
        species_mass=[mass], species_tau_mode=[TAU_STOKES], species_tau=[0.1],
        rho=np.ones(ncell), vgas=vgas, q=q, v=v, dt=5e-3, steps=200, feedback=1,
        fargo=1, omega=1.0, qshear=1.5,
        notes={"dust_to_gas": 0.02, "grains_per_zone": ppc, "L": L})


def cyldisk(scale="full", seed=BASE_SEED + 2):
    """Cylindrical global disk, log-spaced R, 4 Stokes-number species."""
    r = _rng(seed)
    if scale == "full":
        nR, nphi, nz, ng = 384, 1024, 64, 50_000_000
    elif scale == "mid":
        # an eighth of the zones and grains (profiling size, same structure)
        nR, nphi, nz, ng = 192, 512, 32, 6_250_000
    else:
        nR, nphi, nz, ng = 24, 32, 8, 24_000
    R0, R1, zh = 0.4, 2.5, 0.15
    edges = [_log_edges(R0, R1, nR), _uniform_edges(0.0, 2.0 * np.pi, nphi),
             _uniform_edges(-zh, zh, nz)]
    Rc, _, _ = _grid3(edges)
    ncell = len(Rc)
    rho = 1.0 / Rc
    vk = Rc ** -0.5
    amp = 1e-3
    vgas = [amp * vk * r.standard_normal(ncell),
            vk * (1.0 + amp * r.standard_normal(ncell)),
            amp * vk * r.standard_normal(ncell)]
    # Sigma ~ 1/R makes Sigma R dR flat, so R is uniform (inverse CDF, Sec. 4.7)
    R = r.uniform(R0, R1, ng)
    phi = r.uniform(0.0, 2.0 * np.pi, ng)
    z = r.uniform(-zh, zh, ng)
    species = (np.arange(ng) % 4).astype(np.uint8)
    r.shuffle(species)
    gas_mass = (R1 - R0) * 2.0 * np.pi * (2.0 * zh)
    mass = 0.01 * gas_mass / ng
    v = [np.zeros(ng), R ** -0.5, np.zeros(ng)]
    return Workload(
        name="cyldisk", geom=CYLINDRICAL, edges=edges, bc=[OUTFLOW, PERIODIC, PERIODIC],
        weight=TSC, species_mass=[mass] * 4, species_tau_mode=[TAU_STOKES] * 4,
        species_tau=[0.01, 0.1, 1.0, 10.0], rho=rho, vgas=vgas, q=[R, phi, z], v=v,
        dt=1e-3, steps=200, feedback=1, species=species, gm=1.0, vertical_gravity=0,
        notes={"dust_to_gas": 0.01})


def sphdisk(scale="full", seed=BASE_SEED + 3):
    """Spherical disk, log-spaced r, theta within 0.3 of the midplane."""
    r = _rng(seed)
    if scale == "full":
        nr, nth, nphi, ng = 256, 128, 512, 33_000_000
    else:
        nr, nth, nphi, ng = 16, 16, 16, 20_000
    r0, r1, dth, hh = 0.5, 3.0, 0.3, 0.05
    edges = [_log_edges(r0, r1, nr),
             _uniform_edges(0.5 * np.pi - dth, 0.5 * np.pi + dth, nth),
             _uniform_edges(0.0, 2.0 * np.pi, nphi)]
    rc, thc, _ = _grid3(edges)
    ncell = len(rc)
    rho = rc ** -1.5 * np.exp(-(1.0 / np.tan(thc)) ** 2 / (2.0 * hh * hh))
    vk = (rc * np.sin(thc)) ** -0.5
    amp = 1e-3
    vgas = [amp * vk * r.standard_normal(ncell), amp * vk * r.standard_normal(ncell),
            vk * (1.0 + amp * r.standard_normal(ncell))]
    # r from the inverse CDF of rho r^2 ~ r^0.5
    u = r.uniform(0.0, 1.0, ng)
    rr = (r0 ** 1.5 + u * (r1 ** 1.5 - r0 ** 1.5)) ** (2.0 / 3.0)
    th = np.empty(ng)
    todo = np.arange(ng)
    while len(todo):
        t = 0.5 * np.pi - np.arctan(hh * r.standard_normal(len(todo)))
        ok = (t >= edges[1][0]) & (t < edges[1][-1])
        th[todo[ok]] = t[ok]
        todo = todo[~ok]
    phi = r.uniform(0.0, 2.0 * np.pi, ng)
    st = 10.0 ** r.uniform(-4.0, 1.0, ng)
    dV = ((edges[0][1:] ** 3 - edges[0][:-1] ** 3) / 3.0)[None, None, :] \
        * (np.cos(edges[1][:-1]) - np.cos(edges[1][1:]))[None, :, None] \
        * np.diff(edges[2])[:, None, None]
    gas_mass = float((rho.reshape(nphi, nth, nr) * dV).sum())
    mass = 0.01 * gas_mass / ng
    v = [np.zeros(ng), np.zeros(ng), (rr * np.sin(th)) ** -0.5]
    return Workload(
        name="sphdisk", geom=SPHERICAL, edges=edges, bc=[OUTFLOW, OUTFLOW, PERIODIC],
        weight=TSC, species_mass=[mass], species_tau_mode=[TAU_STOKES], species_tau=[1.0],
        rho=rho, vgas=vgas, q=[rr, th, phi], v=v, dt=2e-3, steps=100, feedback=1,
        param=st, gm=1.0, notes={"dust_to_gas": 0.01})


def si2d_instance(k, scale="full", seed=None):
    """Instance k (0..63) of the batched streaming-instability workload."""
    seed = BASE_SEED + 4 + k if seed is None else seed
    r = _rng(seed)
    side = 32 * 2 ** (k % 5) if scale == "full" else 8 * (1 + k % 3)
    ppc = 1 + (k % 16) if scale == "full" else 1 + (k % 4)
    st = (0.01, 0.1, 1.0)[k % 3]
    eps = (0.01, 0.02, 0.1)[(k // 3) % 3]
    L = 0.2
    edges = [_uniform_edges(-0.5 * L, 0.5 * L, side), np.array([-0.5 * L, 0.5 * L]),
             _uniform_edges(-0.5 * L, 0.5 * L, side)]
    ncell = side * side
    q = _per_zone_positions(r, edges, ppc)
    ng = len(q[0])
    etavk = 0.05  # eta v_K = c_s / 20 with c_s = 1 (Sec. 4.3)
    dlt = (1.0 + eps) ** 2 + st ** 2
    amp = 1e-3
    vg = [np.full(ncell, 2.0 * eps * st / dlt * etavk),
          np.full(ncell, -(1.0 + eps * st ** 2 / dlt) / (1.0 + eps) * etavk),
          np.zeros(ncell)]
    vgas = [x + amp * r.standard_normal(ncell) for x in vg]
    # dust: the printed x-component of Eq. SI_equil carries an extra factor eps;
    # the steady state of the dust equation of motion is -2 St / Delta eta v_K
    v = [np.full(ng, -2.0 * st / dlt * etavk),
         np.full(ng, -(1.0 - st ** 2 / dlt) / (1.0 + eps) * etavk),
         np.zeros(ng)]
    dV = (L / side) ** 2 * L
    mass = eps * dV / ppc
    return Workload(
        name="si2d_%02d" % k, geom=SHEARING_BOX, edges=edges, bc=[PERIODIC] * 3, weight=TSC,
        species_mass=[mass], species_tau_mode=[TAU_STOKES], species_tau=[st],
        rho=np.ones(ncell), vgas=vgas, q=q, v=v, dt=5e-3, steps=200, feedback=1,
        fargo=1, omega=1.0, qshear=1.5,
        notes={"dust_to_gas": eps, "grains_per_zone": ppc, "stokes": st})


def si2d_batch(scale="full", count=64):
    return [si2d_instance(k, scale) for k in range(count)]


WORKLOADS = {"box2d": box2d, "sbox3d": sbox3d, "cyldisk": cyldisk, "sphdisk": sphdisk}


def subsample(w: Workload, n: int, seed: int = 7) -> Workload:
    """The same workload restricted to a seeded random subset of n grains."""
    import copy
    idx = np.sort(_rng(seed).choice(w.ngrains, size=min(n, w.ngrains), replace=False))
    s = copy.copy(w)
    s.q = [a[idx].copy() for a in w.q]
    s.v = [a[idx].copy() for a in w.v]
    s.species = None if w.species is None else w.species[idx].copy()
    s.param = None if w.param is None else w.param[idx].copy()
    return s
