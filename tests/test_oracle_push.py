"""Pins of the oracle's exponential-midpoint push and feedback deposit against
what the paper and the mathematics fix (none of them re-types the oracle):

* exact exponential relaxation toward uniform gas (Eq. kick_modified,
  "exact solution when G is constant", Sec. 3.2.2);
* second-order convergence (Sec. 3.2.2, Secs. 4.1, 4.4, 4.5);
* the stiff limit tau_s -> 0 (Sec. 3.2.2, correct asymptotic solution);
* time reversibility (Sec. 3.2.2);
* epicyclic motion: energy exactly conserved with orbital advection,
  oscillating in the standard frame (Sec. 4.2, Eqs. epicyclic,
  epicyclic_energy);
* the circular Kepler orbit is exact; eccentric and inclined orbits converge
  at second order against the Kepler-equation solution (Sec. 4.4);
* the NSH equilibrium is a fixed point of the orbital-advection kick
  (Eq. SI_equil, Sec. 4.3);
* momentum (and angular momentum) conservation of the feedback (Sec. 3.1,
  Eq. dust_feedback_final) and the energy identity of the energy channel
  (exact in Cartesian coordinates; minus the grain's mechanical energy
  change to third order per step in the shearing box, cylindrical and
  spherical geometries);
* the shear-periodic boundary is the sheared image of the central box: a
  grain crossing it ends where it ends in a wider box, mapped back;
* the printed stiff-deceleration L1 errors (Sec. 4.1, tests/golden);
* radial drift against the NSH prediction (Sec. 4.5).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1908_10793_gb300 import inputs as I

INF = float("inf")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def box_problem(n=(4, 4, 4), lo=-100.0, hi=100.0, **kw):
    edges = [np.linspace(lo, hi, k + 1) if k > 1 else np.array([lo, hi]) for k in n]
    return O.Problem(edges=edges, **kw)


def gas_uniform(prob, rho=1.0, v=(0.0, 0.0, 0.0)):
    nc = prob.ncell
    return np.full(nc, float(rho)), [np.full(nc, float(x)) for x in v]


def run(prob, q, p, dt, steps, rho, pg, t0=0.0, param=None, species=None, active=None):
    q = [np.array(x, dtype=np.float64) for x in q]
    p = [np.array(x, dtype=np.float64) for x in p]
    n = len(q[0])
    active = np.ones(n, np.uint8) if active is None else active
    dep_tot = np.zeros((prob.ncell, 4))
    for s in range(steps):
        dep, _ = O.step(prob, q, p, active, t0 + s * dt, dt, rho, pg, species, param)
        dep_tot += dep
    return q, p, active, dep_tot


# --------------------------------------------------------------------------
def test_exact_exponential_relaxation_toward_uniform_gas():
    prob = box_problem(geom=O.OG_CARTESIAN, species_tau=(1.0,))
    vg = (0.3, -0.2, 0.1)
    rho, pg = gas_uniform(prob, 1.0, vg)
    rng = np.random.default_rng(3)
    n = 8
    q0 = [rng.uniform(-5, 5, n) for _ in range(3)]
    v0 = [rng.normal(0, 1, n) for _ in range(3)]
    dt = 0.1
    for ratio in (0.01, 0.5, 3.0, 40.0):
        tau = dt / ratio
        param = np.full(n, tau)
        steps = 7
        _, p, _, _ = run(prob, q0, v0, dt, steps, rho, pg, param=param)
        for d in range(3):
            exact = vg[d] + (v0[d] - vg[d]) * np.exp(-steps * dt / tau)
            assert np.abs(p[d] - exact).max() < 1e-14 * (1 + np.abs(v0[d]).max())


def test_position_converges_at_second_order_for_uniform_gas():
    prob = box_problem(geom=O.OG_CARTESIAN)
    vg = (0.3, 0.0, 0.0)
    rho, pg = gas_uniform(prob, 1.0, vg)
    tau, T, x0, v0 = 0.2, 1.0, 0.1, 2.0
    exact = x0 + vg[0] * T + tau * (v0 - vg[0]) * (1 - np.exp(-T / tau))
    errs = []
    for N in (10, 20, 40, 80):
        q, _, _, _ = run(prob, [[x0], [0.0], [0.0]], [[v0], [0.0], [0.0]], T / N, N, rho, pg,
                         param=np.array([tau]))
        errs.append(abs(q[0][0] - exact))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


def test_second_order_convergence_with_gridded_gas_and_drag():
    n = 64
    edges = [np.linspace(0.0, 1.0, n + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC)
    xc = 0.5 * (edges[0][1:] + edges[0][:-1])
    rho = np.ones(n)
    pg = [0.4 * np.sin(2 * np.pi * xc), np.zeros(n), np.zeros(n)]
    tau, T = 0.05, 0.5
    q0, v0 = [[0.31], [0.5], [0.5]], [[0.7], [0.0], [0.0]]

    def final(N):
        q, p, _, _ = run(prob, q0, v0, T / N, N, rho, pg, param=np.array([tau]))
        return q[0][0], p[0][0]

    ref = final(25600)
    errs = [abs(final(N)[0] - ref[0]) for N in (50, 100, 200, 400)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 1.75) & (slopes < 2.3)), slopes


@pytest.mark.parametrize("tau_over_dt", [1e-8, 1e-300, 0.0])
def test_stiff_limit_gives_gathered_gas_velocity(tau_over_dt):
    n = 16
    edges = [np.linspace(0.0, 1.0, n + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC)
    xc = 0.5 * (edges[0][1:] + edges[0][:-1])
    rho = np.ones(n)
    pg = [np.cos(2 * np.pi * xc), np.zeros(n), np.zeros(n)]
    dt, x0, v0 = 0.01, 0.4, 3.0
    q, p, _, _ = run(prob, [[x0], [0.5], [0.5]], [[v0], [0.0], [0.0]], dt, 1, rho, pg,
                     param=np.array([tau_over_dt * dt]))
    # textbook TSC interpolation at the midpoint x0 + dt/2 v0 (Eq. b1 shape)
    xm = x0 + 0.5 * dt * v0
    i = int(xm * n)
    d = xm * n - (i + 0.5)
    w = [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]
    vint = sum(w[k] * pg[0][(i - 1 + k) % n] for k in range(3))
    assert np.isfinite(p[0][0])
    assert abs(p[0][0] - vint) < 1e-14
    assert abs(q[0][0] - (xm + 0.5 * dt * vint)) < 1e-15


def test_stiff_limit_shearing_box_tends_to_gas_velocity():
    prob = box_problem(geom=O.OG_SHEARING_BOX, fargo=0, omega=1.0, q=1.5)
    vg = (0.02, -0.01, 0.0)
    rho, pg = gas_uniform(prob, 1.0, vg)
    dt = 0.1
    _, p, _, _ = run(prob, [[0.3], [0.1], [0.0]], [[1.0], [2.0], [0.5]], dt, 1, rho, pg,
                     param=np.array([1e-10 * dt]))
    # h1 ~ tau: Omega_1 -> 0, R^-1 -> I, E -> 0: v -> v_g + O(tau)
    assert abs(p[0][0] - vg[0]) < 1e-9 and abs(p[1][0] - vg[1]) < 1e-9 and abs(p[2][0]) < 1e-12


# --------------------------------------------------------------------------
def _reverse(prob, q0, p0, dt, N, rho, pg, param):
    q, p, _, _ = run(prob, q0, p0, dt, N, rho, pg, param=param)
    q2, p2, _, _ = run(prob, q, p, -dt, N, rho, pg, t0=N * dt, param=param)
    return q2, p2


def test_time_reversibility_cartesian_gridded_gas():
    n = 32
    edges = [np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1), np.array([0.0, 1.0])]
    prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC)
    X, Y, _ = I._grid3(edges)
    rho = np.ones(n * n)
    pg = [0.2 * np.sin(2 * np.pi * X), 0.1 * np.cos(2 * np.pi * Y), np.zeros(n * n)]
    q0 = [[0.4, 0.6], [0.45, 0.52], [0.5, 0.5]]
    p0 = [[0.1, -0.05], [0.05, 0.02], [0.0, 0.0]]
    dt, N = 0.01, 10
    q, p = _reverse(prob, q0, p0, dt, N, rho, pg, param=np.array([0.02, 0.02]))  # N dt/tau = 5
    for d in range(3):
        assert np.abs(q[d] - np.array(q0[d])).max() < 1e-11
        assert np.abs(p[d] - np.array(p0[d])).max() < 1e-11


@pytest.mark.parametrize("fargo", [0, 1])
def test_time_reversibility_shearing_box(fargo):
    prob = box_problem(n=(8, 8, 8), lo=-1.0, hi=1.0, geom=O.OG_SHEARING_BOX, fargo=fargo,
                       omega=1.0, q=1.5, vertical_gravity=1)
    X, Y, Z = I._grid3(prob.edges)
    rho = np.ones(prob.ncell)
    pg = [0.05 * np.sin(np.pi * Y), 0.03 * np.cos(np.pi * X), 0.02 * np.sin(np.pi * Z)]
    q0 = [[0.2], [-0.1], [0.05]]
    p0 = [[0.01], [-0.02], [0.03]]
    q, p = _reverse(prob, q0, p0, 0.05, 20, rho, pg, param=np.array([0.5]))
    for d in range(3):
        assert abs(q[d][0] - q0[d][0]) < 1e-12 and abs(p[d][0] - p0[d][0]) < 1e-12


def _cyl_problem(nR=16, nphi=32, nz=8, weight=O.OW_TSC, **kw):
    edges = [np.geomspace(0.5, 2.0, nR + 1), np.linspace(0, 2 * np.pi, nphi + 1),
             np.linspace(-0.3, 0.3, nz + 1)]
    return O.Problem(geom=O.OG_CYLINDRICAL, edges=edges, bc=(O.OB_OUTFLOW, 0, 0),
                     weight=weight, gm=1.0, vertical_gravity=1, **kw)


def test_time_reversibility_cylindrical_with_drag():
    prob = _cyl_problem()
    R, PHI, Z = I._grid3(prob.edges)
    rho = np.ones(prob.ncell)
    pg = O.gas_momentum(prob, [0.01 * np.sin(PHI), R ** -0.5 * (1 + 0.01 * np.cos(PHI)),
                               0.01 * Z])
    q0 = [[1.1], [0.3], [0.05]]
    p0 = [[0.02], [1.1 * 0.95], [-0.01]]
    q, p = _reverse(prob, q0, p0, 0.02, 50, rho, pg, param=np.array([0.3]))
    for d in range(3):
        assert abs(q[d][0] - q0[d][0]) < 1e-12 and abs(p[d][0] - p0[d][0]) < 1e-12


def _sph_problem(weight=O.OW_TSC, dth=0.6, **kw):
    edges = [np.geomspace(0.5, 1.6, 17), np.linspace(np.pi / 2 - dth, np.pi / 2 + dth, 17),
             np.linspace(0, 2 * np.pi, 33)]
    return O.Problem(geom=O.OG_SPHERICAL, edges=edges, bc=(O.OB_OUTFLOW, O.OB_OUTFLOW, 0),
                     weight=weight, gm=1.0, **kw)


def test_time_reversibility_spherical_with_drag():
    prob = _sph_problem()
    R, TH, PHI = I._grid3(prob.edges)
    rho = np.ones(prob.ncell)
    pg = O.gas_momentum(prob, [0.01 * np.cos(PHI), 0.01 * np.sin(PHI),
                               (R * np.sin(TH)) ** -0.5])
    q0 = [[1.05], [1.4], [0.7]]
    p0 = [[0.01], [0.1], [0.9]]
    q, p = _reverse(prob, q0, p0, 0.02, 50, rho, pg, param=np.array([0.4]))
    for d in range(3):
        assert abs(q[d][0] - q0[d][0]) < 1e-12 and abs(p[d][0] - p0[d][0]) < 1e-12


# --------------------------------------------------------------------------
def _epicycle(fargo, dt, T, A=0.4, Om=1.0, qs=1.5):
    prob = box_problem(n=(4, 4, 4), lo=-1.0, hi=1.0, geom=O.OG_SHEARING_BOX, fargo=fargo,
                       omega=Om, q=qs)
    rho, pg = gas_uniform(prob)
    vy0 = -2.0 * Om * A + (qs * Om * A if fargo else 0.0)
    q = [np.array([A]), np.array([0.0]), np.array([0.0])]
    p = [np.array([0.0]), np.array([vy0]), np.array([0.0])]
    active = np.ones(1, np.uint8)
    energies, xs = [], []
    N = int(round(T / dt))
    for s in range(N):
        O.step(prob, q, p, active, s * dt, dt, rho, pg, None, np.array([INF]))
        vy = p[1][0] - (qs * Om * q[0][0] if fargo else 0.0)
        energies.append(0.5 * (p[0][0] ** 2 + vy ** 2) - qs * Om * Om * q[0][0] ** 2)
        xs.append((q[0][0], q[1][0]))
    return np.array(energies), np.array(xs)


def test_epicycle_energy_conserved_with_orbital_advection():
    # Sec. 4.2: A = 0.4, Omega = 1, dt = 0.4, t_f = 40; exact energy omega^2 A^2 / 2
    E, _ = _epicycle(fargo=1, dt=0.4, T=40.0)
    E0 = 0.5 * 1.0 * 0.4 ** 2
    assert np.abs(E / E0 - 1.0).max() < 1e-13


def test_epicycle_energy_bounded_in_standard_frame():
    E, _ = _epicycle(fargo=0, dt=0.4, T=40.0)
    E0 = 0.5 * 0.4 ** 2
    dev = E / E0 - 1.0
    assert np.abs(dev).max() < 0.15          # oscillates around the exact value
    assert np.abs(dev).max() > 1e-3          # (it does oscillate at this large dt)
    assert abs(dev[-25:].mean() - dev[:25].mean()) < 0.02   # no secular drift


@pytest.mark.parametrize("fargo", [0, 1])
def test_epicycle_orbit_second_order(fargo):
    T = 10.0
    errs = []
    for N in (100, 200, 400, 800):
        _, xs = _epicycle(fargo, T / N, T)
        x_ex = 0.4 * np.cos(T)
        y_ex = -2.0 * 0.4 * np.sin(T)
        errs.append(np.hypot(xs[-1][0] - x_ex, xs[-1][1] - y_ex))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


# --------------------------------------------------------------------------
def _kepler(e, t):
    M = t % (2 * np.pi)
    E = M if e < 0.8 else np.pi
    for _ in range(60):
        E -= (E - e * np.sin(E) - M) / (1 - e * np.cos(E))
    R = 1.0 - e * np.cos(E)
    f = 2.0 * np.arctan2(np.sqrt(1 + e) * np.sin(E / 2), np.sqrt(1 - e) * np.cos(E / 2))
    return R, f % (2 * np.pi)


def test_circular_kepler_orbit_is_exact():
    # Sec. 4.4: R = 1, l = 1, dt = 0.1, 20 orbits: R and l stay exactly 1
    prob = _cyl_problem()
    rho, pg = gas_uniform(prob)
    dt = 0.1
    N = int(round(20 * 2 * np.pi / dt))
    q, p, active, _ = run(prob, [[1.0], [0.0], [0.0]], [[0.0], [1.0], [0.0]], dt, N, rho, pg,
                          param=np.array([INF]))
    assert active[0] == 1
    assert q[0][0] == 1.0 and p[1][0] == 1.0 and p[0][0] == 0.0


def test_eccentric_kepler_orbit_second_order():
    prob = _cyl_problem()
    rho, pg = gas_uniform(prob)
    e = 0.3
    R0 = 1.0 - e
    l0 = np.sqrt(1.0 * (1.0 - e * e))  # sqrt(GM a (1-e^2)), a = 1
    T = 2 * np.pi
    Rex, fex = _kepler(e, T)
    errs = []
    for N in (200, 400, 800, 1600):
        q, p, _, _ = run(prob, [[R0], [0.0], [0.0]], [[0.0], [l0], [0.0]], T / N, N, rho, pg,
                         param=np.array([INF]))
        x, y = q[0][0] * np.cos(q[1][0]), q[0][0] * np.sin(q[1][0])
        errs.append(np.hypot(x - Rex * np.cos(fex), y - Rex * np.sin(fex)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


def test_inclined_circular_orbit_spherical_second_order():
    # Sec. 4.4: orbit tilted by 30 degrees, one period, against the exact orbit
    prob = _sph_problem(dth=0.6)
    rho, pg = gas_uniform(prob)
    inc = np.radians(30.0)
    q0 = [[1.0], [np.pi / 2], [0.0]]
    p0 = [[0.0], [-np.sin(inc)], [np.cos(inc)]]
    T = 2 * np.pi
    errs, lerr = [], []
    for N in (200, 400, 800, 1600):
        q, p, active, _ = run(prob, q0, p0, T / N, N, rho, pg, param=np.array([INF]))
        assert active[0] == 1
        r, th, ph = q[0][0], q[1][0], q[2][0]
        xyz = r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        errs.append(np.linalg.norm(xyz - np.array([1.0, 0.0, 0.0])))
        L = np.sqrt(p[1][0] ** 2 + p[2][0] ** 2 / np.sin(th) ** 2)
        lerr.append(abs(L - 1.0))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.15), slopes
    assert max(lerr) < 1e-3


# --------------------------------------------------------------------------
def _nsh(eps, st, etavk=0.05, printed=False):
    dl = (1 + eps) ** 2 + st ** 2
    vg = (2 * eps * st / dl * etavk, -(1 + eps * st ** 2 / dl) / (1 + eps) * etavk, 0.0)
    vpx = -(2 * eps * st if printed else 2 * st) / dl * etavk
    vp = (vpx, -(1 - st ** 2 / dl) / (1 + eps) * etavk, 0.0)
    return vg, vp


@pytest.mark.parametrize("st", [0.01, 0.1, 1.0, 10.0])
def test_nsh_equilibrium_is_fixed_point_of_fargo_kick(st):
    prob = box_problem(n=(4, 4, 4), lo=-1.0, hi=1.0, geom=O.OG_SHEARING_BOX, fargo=1,
                       omega=1.0, q=1.5, species_tau_mode=(O.OT_STOKES,), species_tau=(st,))
    for eps in (0.2, 3.0):
        vg, vp = _nsh(eps, st)
        rho, pg = gas_uniform(prob, 1.0, vg)
        for dt in (1e-3, 0.1, 10.0):
            _, p, _, _ = run(prob, [[0.1], [0.2], [0.0]], [[vp[0]], [vp[1]], [0.0]], dt, 1,
                             rho, pg)
            assert abs(p[0][0] - vp[0]) < 1e-16 and abs(p[1][0] - vp[1]) < 1e-16
        # the printed dust x-velocity (extra factor eps) is not a steady state
        _, vpp = _nsh(eps, st, printed=True)
        _, p, _, _ = run(prob, [[0.1], [0.2], [0.0]], [[vpp[0]], [vpp[1]], [0.0]], 0.1, 1,
                         rho, pg)
        assert abs(p[0][0] - vpp[0]) + abs(p[1][0] - vpp[1]) > 1e-6


# --------------------------------------------------------------------------
def _oracle_state(w):
    """Oracle problem, particle and gas arrays from a workload."""
    prob = O.Problem(geom=w.geom, edges=w.edges, bc=w.bc, weight=w.weight,
                     species_mass=w.species_mass, species_tau_mode=w.species_tau_mode,
                     species_tau=w.species_tau, fargo=w.fargo, omega=w.omega, q=w.qshear,
                     gm=w.gm, vertical_gravity=w.vertical_gravity, feedback_apply=w.feedback)
    q = [x.copy() for x in w.q]
    p = [x.copy() for x in w.v]
    if w.geom == O.OG_CYLINDRICAL:
        p[1] = q[0] * w.v[1]
    if w.geom == O.OG_SPHERICAL:
        p[1] = q[0] * w.v[1]
        p[2] = q[0] * np.sin(q[1]) * w.v[2]
    pg = O.gas_momentum(prob, w.vgas)
    return prob, q, p, w.rho.copy(), pg


def _zone_volumes(prob):
    e = prob.edges
    if prob.geom == O.OG_CYLINDRICAL:
        a = 0.5 * np.diff(e[0] ** 2)
        b = np.diff(e[1])
    elif prob.geom == O.OG_SPHERICAL:
        a = np.diff(e[0] ** 3) / 3.0
        b = -np.diff(np.cos(e[1]))
    else:
        a, b = np.diff(e[0]), np.diff(e[1])
    c = np.diff(e[2])
    return (c[:, None, None] * b[None, :, None] * a[None, None, :]).ravel()


def test_feedback_conserves_total_momentum_cartesian():
    w = I.box2d("small")
    prob, q, p, rho, pg = _oracle_state(w)
    dV = _zone_volumes(prob)
    m = w.species_mass[0]

    def total():
        return np.array([(rho * pg[d] * dV).sum() + m * p[d].sum() for d in range(3)])

    before = total()
    active = np.ones(w.ngrains, np.uint8)
    for s in range(5):
        O.step(prob, q, p, active, s * w.dt, w.dt, rho, pg)
    after = total()
    assert np.abs(after - before).max() < 1e-14 * max(1.0, np.abs(before).max())
    assert np.abs(pg[0] - 0.3).max() > 1e-4   # the gas really was changed


def test_feedback_conserves_angular_and_vertical_momentum_cylindrical():
    w = I.cyldisk("small")
    prob, q, p, rho, pg = _oracle_state(w)
    dV = _zone_volumes(prob)
    ms = np.array(w.species_mass)[w.species]

    def total():
        return np.array([(rho * pg[d] * dV).sum() + (ms * p[d]).sum() for d in (1, 2)])

    before = total()
    active = np.ones(w.ngrains, np.uint8)
    for s in range(3):
        _, removed = O.step(prob, q, p, active, s * w.dt, w.dt, rho, pg, w.species)
        assert removed == 0
    after = total()
    assert np.abs(after - before).max() < 1e-13 * np.abs(before).max()


def test_energy_channel_equals_minus_dust_kinetic_energy_change():
    # Cartesian, no external force: dE = -m v^{n+1/2} . (v^{n+1} - v^n)
    #                                  = -m (|v^{n+1}|^2 - |v^n|^2) / 2
    w = I.box2d("small")
    w.feedback = 0
    prob, q, p, rho, pg = _oracle_state(w)
    m = w.species_mass[0]
    ke0 = 0.5 * m * sum((x ** 2).sum() for x in p)
    dep, _ = O.step(prob, q, p, np.ones(w.ngrains, np.uint8), 0.0, w.dt, rho, pg)
    ke1 = 0.5 * m * sum((x ** 2).sum() for x in p)
    assert abs(dep[:, 3].sum() + (ke1 - ke0)) < 1e-13 * abs(ke1 - ke0) + 1e-17


def _mechanical_energy_case(case):
    """One grain inside a 4^3-zone grid with non-uniform gas and drag, and its
    specific kinetic and potential energy in physical terms: the shearing box
    in the standard frame (Jacobi form: tidal -q Omega^2 x^2, vertical
    Omega^2 z^2 / 2), the cylindrical and spherical disk around a point mass
    (with or without the z part of the gravity in cylindrical coordinates)."""
    mass, tau = 0.3, 0.1
    if case.startswith("sbox"):
        vg = case.endswith("vgrav")
        prob = box_problem(n=(4, 4, 4), lo=-0.5, hi=0.5, geom=O.OG_SHEARING_BOX,
                           species_mass=(mass,), species_tau=(tau,), omega=1.0, q=1.5,
                           vertical_gravity=int(vg))
        q, p = [0.07, -0.03, 0.05], [0.11, -0.08, 0.04]

        def energy(q, p):
            return 0.5 * (p[0] ** 2 + p[1] ** 2 + p[2] ** 2) - 1.5 * q[0] ** 2 + \
                (0.5 * q[2] ** 2 if vg else 0.0)
    elif case.startswith("cyl"):
        vg = case.endswith("vgrav")
        edges = [np.linspace(0.5, 1.5, 5), np.linspace(0.0, 2 * np.pi, 9), np.linspace(-0.2, 0.2, 5)]
        prob = O.Problem(geom=O.OG_CYLINDRICAL, edges=edges, species_mass=(mass,),
                         species_tau=(tau,), gm=1.0, vertical_gravity=int(vg))
        q, p = [1.03, 1.1, 0.04], [0.05, 1.03 * 0.93, 0.02]   # (v_R, l = R v_phi, v_z)

        def energy(q, p):
            phi = -1.0 / np.hypot(q[0], q[2]) if vg else -1.0 / q[0]
            return 0.5 * (p[0] ** 2 + (p[1] / q[0]) ** 2 + p[2] ** 2) + phi
    else:
        th = 0.5 * np.pi - 0.1
        edges = [np.linspace(0.5, 1.5, 5), np.linspace(0.5 * np.pi - 0.3, 0.5 * np.pi + 0.3, 5),
                 np.linspace(0.0, 2 * np.pi, 9)]
        prob = O.Problem(geom=O.OG_SPHERICAL, edges=edges, species_mass=(mass,),
                         species_tau=(tau,), gm=1.0)
        # (v_r, l_theta = r v_theta, l_phi = r sin(theta) v_phi)
        q, p = [1.02, th, 1.1], [0.05, 0.03, 1.02 * np.sin(th) * 0.95]

        def energy(q, p):
            r, st = q[0], np.sin(q[1])
            return 0.5 * (p[0] ** 2 + (p[1] / r) ** 2 + (p[2] / (r * st)) ** 2) - 1.0 / r
    return prob, q, p, energy


@pytest.mark.parametrize("case", ["sbox", "sbox_vgrav", "cyl", "cyl_vgrav", "sph"])
def test_energy_channel_equals_minus_mechanical_energy_change_at_third_order(case):
    # Drag is the only non-conservative force on a grain, and the energy
    # channel is minus its impulse times the midpoint dH/dp: it must equal
    # minus the grain's change of kinetic plus potential energy, up to the
    # local error of a second-order step, O(dt^3).  A wrong metric factor or
    # an end-point instead of a midpoint value leaves O(dt) or O(dt^2).
    def one(dt):
        prob, q0, p0, energy = _mechanical_energy_case(case)
        rng = np.random.default_rng(5)
        rho = rng.uniform(0.8, 1.2, prob.ncell)
        pg = [p0[d] + rng.uniform(-0.1, 0.1, prob.ncell) for d in range(3)]
        q = [np.array([x]) for x in q0]
        p = [np.array([x]) for x in p0]
        m = prob.sp_mass[0]
        e0 = m * energy([x[0] for x in q], [x[0] for x in p])
        dep, removed = O.step(prob, q, p, np.ones(1, np.uint8), 0.0, dt, rho, pg)
        assert removed == 0
        e1 = m * energy([x[0] for x in q], [x[0] for x in p])
        return dep[:, 3].sum(), dep[:, 3].sum() + (e1 - e0)

    res = [one(h) for h in (0.02, 0.01, 0.005)]
    for de, r in res:
        assert abs(de) > 1e-5             # the drag really exchanged energy
        assert abs(r) < 1e-3 * abs(de)
    for k in range(2):
        assert abs(res[k][1]) > 6.0 * abs(res[k + 1][1]), (case, res)


@pytest.mark.parametrize("fargo", [0, 1])
def test_shear_periodic_boundary_matches_the_sheared_image_of_a_wider_box(fargo):
    # Shearing-sheet symmetry (Sec. 4.2 setup): the flow -q Omega x makes the
    # box at x + L_x the central box moved by -q Omega L_x t in y, so a grain
    # that leaves through +x is the image (x - L_x, y + q Omega L_x t,
    # v_y + q Omega L_x in the standard frame; the residual velocity is
    # unchanged).  Without drag, grains crossing the x boundaries of a box
    # of width 1 must therefore end where the same grains end in a box of
    # width 3 (no crossing there), mapped back by that image.
    Om, qs, L = 1.0, 1.5, 1.0

    def evolve(xlo, xhi, nx, q0, p0, t0, dt, steps):
        edges = [np.linspace(xlo, xhi, nx + 1), np.linspace(-0.5, 0.5, 5), np.linspace(-0.5, 0.5, 5)]
        prob = O.Problem(geom=O.OG_SHEARING_BOX, edges=edges, species_tau=(INF,), omega=Om, q=qs,
                         fargo=fargo)
        rho = np.ones(prob.ncell)
        pg = [np.zeros(prob.ncell) for _ in range(3)]
        q, p, active, _ = run(prob, q0, p0, dt, steps, rho, pg, t0=t0)
        assert active.all()
        return q, p

    x0 = [0.4, -0.4, 0.45, -0.3]
    q0 = [x0, [0.1, -0.2, -0.45, 0.3], [0.0, 0.1, 0.2, -0.1]]
    res = [[0.5, -0.5, 0.2, -0.45], [0.2, 0.1, 0.3, -0.2], [0.0, 0.05, 0.0, 0.02]]
    if fargo:
        p0 = res
    else:   # the same motion in the standard frame: v_y = v'_y - q Omega x
        p0 = [res[0], [v - qs * Om * x for v, x in zip(res[1], x0)], res[2]]
    t0, dt, steps = 0.3, 0.05, 30
    T = t0 + steps * dt
    qa, pa = evolve(-0.5 * L, 0.5 * L, 4, q0, p0, t0, dt, steps)
    qb, pb = evolve(-1.5 * L, 1.5 * L, 12, q0, p0, t0, dt, steps)
    k = np.floor((qb[0] + 0.5 * L) / L)
    assert (k == 1).any() and (k == -1).any()     # both boundaries crossed
    x = qb[0] - k * L
    y = qb[1] + k * qs * Om * L * T
    vy = pb[1] + (0.0 if fargo else k * qs * Om * L)

    def wrapped(a):
        return (a + 0.5) % 1.0 - 0.5

    assert np.abs(qa[0] - x).max() < 1e-13
    assert np.abs(wrapped(qa[1] - y)).max() < 1e-13
    assert np.abs(qa[2] - qb[2]).max() < 1e-13
    assert np.abs(pa[0] - pb[0]).max() < 1e-13
    assert np.abs(pa[1] - vy).max() < 1e-13
    assert np.abs(pa[2] - pb[2]).max() < 1e-13


# --------------------------------------------------------------------------
def _read_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "deceleration_stiff.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                rows[k] = float(v)
    return rows


def _deceleration_stiff(tau, pusher=O.OP_EM):
    """Sec. 4.1 stiff deceleration with the gas coupled through the oracle's
    half-step drag predictor (Eq. f_D with tau <- max(tau, dt)) and the
    corrector with the final deposit (Eq. dust_feedback_final).  One grain per
    zone, eps = 1."""
    n = 8
    edges = [np.linspace(0.0, 1.0, n + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    dV = 1.0 / n
    eps = 1.0
    prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC,
                     species_mass=(eps * dV,), species_tau=(tau,), pusher=pusher)
    q = [(np.arange(n) + 0.5) / n, np.full(n, 0.5), np.full(n, 0.5)]
    p = [np.ones(n), np.zeros(n), np.zeros(n)]
    pg = [np.full(n, -1.0), np.zeros(n), np.zeros(n)]
    rho = np.ones(n)
    active = np.ones(n, np.uint8)
    dt, tf = 1.0, 10
    vp_hist = [p[0].mean()]
    for s in range(tf):
        _, half = O.gas_predictor(prob, q, p, active, dt, rho, pg)      # predictor
        dep, _ = O.step(prob, q, p, active, s * dt, dt, rho, half)
        pg = [pg[c] + dep[:, c] / (rho * dV) for c in range(3)]       # corrector
        vp_hist.append(p[0].mean())
    t = np.arange(tf + 1) * dt
    exact = np.exp(-(1 + eps) * t / tau)
    return np.abs(np.array(vp_hist) - exact).mean(), vp_hist


def test_gas_predictor_single_zone_closed_form():
    """Eqs. Delta_vp, f_D: a grain at rest in the middle of one zone of a
    1-zone periodic box with uniform gas; the predicted half-step gas velocity
    is v_g + (dt/2) (m / (rho dV)) (v_p - v_g) / max(tau, dt), for tau below and
    above dt."""
    edges = [np.array([0.0, 2.0]), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    for tau, dt in ((0.3, 0.1), (0.3, 1.0), (INF, 0.5)):
        prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, species_mass=(0.4,),
                         species_tau=(tau,))
        imp, half = O.gas_predictor(prob, [[1.0], [0.5], [0.5]], [[0.7], [-0.2], [0.1]],
                                    np.ones(1, np.uint8), dt, np.array([1.5]),
                                    [np.array([0.1]), np.array([0.3]), np.array([-0.4])])
        k = 0.5 * dt * 0.4 / (1.5 * 2.0) / max(tau, dt)
        for c, (vp, vg) in enumerate(((0.7, 0.1), (-0.2, 0.3), (0.1, -0.4))):
            assert half[c][0] == pytest.approx(vg + k * (vp - vg), rel=1e-14, abs=1e-16)


@pytest.mark.parametrize("tau", [0.2, 0.02])
def test_stiff_deceleration_matches_printed_l1_errors(tau):
    printed = _read_golden()[str(tau)]
    l1, hist = _deceleration_stiff(tau)
    # printed to two significant digits
    assert abs(l1 - printed) <= 0.5 * 10 ** (np.floor(np.log10(printed)) - 1) + 1e-30, l1
    if tau == 0.02:
        single = _read_golden()["single_step_tau0.02"]
        assert 0.3 * single < abs(hist[1]) < 3 * single


@pytest.mark.parametrize("tau", [0.2, 0.02])
def test_semi_implicit_deceleration_matches_printed_l1_errors(tau):
    """Sec. 4.1: the semi-implicit scheme of Sec. 3.2.1 in the same coupled
    stiff setup oscillates with little damping; printed L1 errors about 0.068
    and 0.6 (one and two significant digits)."""
    printed = _read_golden()["si_%s" % tau]
    l1, hist = _deceleration_stiff(tau, O.OP_SEMI_IMPLICIT)
    digits = 2 if tau == 0.2 else 1
    assert abs(l1 - printed) <= 0.5 * 10 ** (np.floor(np.log10(printed)) - digits + 1), l1
    # the oscillation the paper describes: the sign alternates every step
    assert all(hist[k] * hist[k + 1] < 0 for k in range(len(hist) - 1))


def test_semi_implicit_uniform_gas_is_the_trapezoidal_rule():
    """For uniform fixed gas and no other force, the semi-implicit kick is the
    trapezoidal (Crank-Nicolson) rule for dv/dt = -(v - v_g)/tau, whose
    one-step factor on v - v_g is (1 - b)/(1 + b), b = dt/(2 tau)."""
    prob = box_problem(geom=O.OG_CARTESIAN, species_tau=(0.3,), pusher=O.OP_SEMI_IMPLICIT)
    rho, pg = gas_uniform(prob, 1.0, (0.2, -0.1, 0.05))
    v0 = [[0.7, -0.4], [0.3, 0.2], [-0.5, 0.9]]
    for dt in (0.01, 0.3, 2.0, 50.0):
        _, p, _, _ = run(prob, [[1.0, -3.0], [2.0, 5.0], [0.5, -1.0]], v0, dt, 1, rho, pg)
        b = dt / 0.6
        for d, vg in enumerate((0.2, -0.1, 0.05)):
            expect = vg + (np.array(v0[d]) - vg) * (1 - b) / (1 + b)
            assert np.allclose(p[d], expect, rtol=1e-13, atol=1e-15), (dt, d)


@pytest.mark.parametrize("fargo", [0, 1])
def test_semi_implicit_equals_exponential_midpoint_without_drag(fargo):
    """Sec. 3.2.2: for infinite stopping time the exponential midpoint kick
    reduces to the semi-implicit one (shearing box, both frames)."""
    res = []
    for pusher in (O.OP_EM, O.OP_SEMI_IMPLICIT):
        prob = box_problem(n=(4, 4, 4), lo=-1.0, hi=1.0, geom=O.OG_SHEARING_BOX, fargo=fargo,
                           omega=1.0, q=1.5, vertical_gravity=1, pusher=pusher)
        rho, pg = gas_uniform(prob, 1.0, (0.1, 0.2, 0.3))
        q, p, _, _ = run(prob, [[0.3, -0.2], [0.1, 0.4], [0.2, -0.3]],
                         [[0.05, -0.1], [-0.4, 0.2], [0.1, 0.0]], 0.05, 40, rho, pg,
                         param=np.array([INF, INF]))
        res.append(np.concatenate([np.ravel(q), np.ravel(p)]))
    assert np.allclose(res[0], res[1], rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("st", [0.1, 1.0, 10.0])
def test_radial_drift_matches_nsh_prediction(st):
    """Sec. 4.5: fixed gas of Eq. Nelson_equil (p = -1, q = -0.5, H0 = 0.1 at
    R0 = 1), 64 x 16 zones in R in [0.2, 1.6], z in [-0.2, 0.2]; grains start at
    R = 1 on Keplerian orbits; time-averaged v_R over 10 orbits against
    -(3/2)(H0/R0)^2 St / (1 + St^2) v_K (v_K = 1 at R = 1; with p = 2q the
    predicted drift speed does not depend on R)."""
    pp, qq, H0 = -1.0, -0.5, 0.1
    edges = [np.linspace(0.2, 1.6, 65), np.array([0.0, 2 * np.pi]), np.linspace(-0.2, 0.2, 17)]
    prob = O.Problem(geom=O.OG_CYLINDRICAL, edges=edges, bc=(O.OB_OUTFLOW, 0, 0),
                     weight=O.OW_TSC, gm=1.0, species_tau_mode=(O.OT_STOKES,),
                     species_tau=(st,))
    R, _, Z = I._grid3(edges)
    r = np.hypot(R, Z)
    H = H0 * R ** ((qq + 3) / 2)
    Om = R ** -1.5 * np.sqrt((pp + qq) * (H / R) ** 2 + (1 + qq) - qq * R / r)
    pg = O.gas_momentum(prob, [np.zeros_like(R), R * Om, np.zeros_like(R)])
    rho = np.ones_like(R)
    dt = 0.01
    N = int(round(20 * np.pi / dt))
    q = [np.array([1.0]), np.array([0.0]), np.array([0.0])]
    p = [np.array([0.0]), np.array([1.0]), np.array([0.0])]
    active = np.ones(1, np.uint8)
    R0 = q[0][0]
    for s in range(N):
        O.step(prob, q, p, active, s * dt, dt, rho, pg)
    vmean = (q[0][0] - R0) / (N * dt)
    pred = -1.5 * H0 ** 2 * st / (1 + st * st)
    assert abs(vmean - pred) < 0.05 * abs(pred), (vmean, pred)


@pytest.mark.parametrize("geom", ["sb_std", "sb_fargo", "cyl", "sph"])
def test_no_drag_means_no_back_reaction(geom):
    """Eq. dust_feedback_final deducts the non-frictional forces: with
    tau_s = infinity the velocity change is dt a^{n+1/2} exactly and the
    deposit must vanish in every geometry."""
    if geom.startswith("sb"):
        prob = box_problem(n=(4, 4, 4), lo=-1.0, hi=1.0, geom=O.OG_SHEARING_BOX,
                           fargo=int(geom == "sb_fargo"), omega=1.0, q=1.5,
                           vertical_gravity=1)
        q0, p0 = [[0.3], [0.1], [0.2]], [[0.05], [-0.4], [0.1]]
    elif geom == "cyl":
        prob = _cyl_problem()
        q0, p0 = [[1.2], [0.5], [0.1]], [[0.05], [1.0], [0.02]]
    else:
        prob = _sph_problem()
        q0, p0 = [[1.1], [1.3], [0.5]], [[0.03], [0.2], [0.8]]
    rho, pg = gas_uniform(prob, 1.0, (0.1, 0.2, 0.3))
    _, p, _, dep = run(prob, q0, p0, 0.05, 3, rho, pg, param=np.array([INF]))
    assert np.abs(dep[:, :3]).max() < 1e-15
    assert np.abs(p[0][0] - p0[0][0]) > 1e-4   # the grain was accelerated


@pytest.mark.parametrize("geom", ["cyl", "sph"])
def test_stokes_number_mode_is_st_over_local_keplerian_frequency(geom):
    """Secs. 4.5-4.6 fix the Stokes number St = tau_s Omega_K with Omega_K =
    sqrt(GM / R^3) at the grain's cylindrical radius.  A grain with no radial
    (and no polar) motion keeps its radius through the half drift, so one step
    in Stokes-number mode must equal one step with the constant stopping time
    St / Omega_K(R) (R = r sin(theta) in spherical coordinates), and differ
    from the one at R = 1."""
    st = 0.3
    if geom == "cyl":
        mk, Rc = _cyl_problem, 1.5
        q0, p0 = [[1.5], [0.4], [0.05]], [[0.0], [1.5 ** 0.5 * 0.9], [0.0]]
    else:
        mk, Rc = _sph_problem, 1.3 * np.sin(1.2)
        q0, p0 = [[1.3], [1.2], [0.5]], [[0.0], [0.0], [0.8]]
    results = []
    for mode, value in ((O.OT_STOKES, st), (O.OT_CONST, st * np.sqrt(Rc ** 3)),
                        (O.OT_CONST, st)):
        prob = mk(species_tau_mode=(mode,), species_tau=(value,))
        R, _, _ = I._grid3(prob.edges)
        rho = np.ones(prob.ncell)
        pg = O.gas_momentum(prob, [np.zeros_like(R), 0.8 * R ** -0.5, np.zeros_like(R)])
        q, p, _, dep = run(prob, q0, p0, 0.05, 1, rho, pg)
        results.append(np.concatenate([np.ravel(q), np.ravel(p)]))
    assert np.allclose(results[0], results[1], rtol=1e-14, atol=1e-15)
    assert np.abs(results[0] - results[2]).max() > 1e-6


# --------------------------------------------------------------------------
def _drift_vr_error(geom, weight, st=1.0, dt=0.1):
    """Sec. 4.5 radial drift, set up as in the paper's weighting comparison:
    fixed gas of Eq. Nelson_equil (p = -1, q = -0.5, H0 = 0.1 at R0 = 1),
    64 x 16 equally spaced zones (cylindrical R in [0.2, 1.6], z in [-0.2,
    0.2]; spherical r in [0.2, 1.8], theta in pi/2 -+ 0.2), one grain of
    St = 1 starting at R = 1 in the midplane on a Keplerian orbit, dt = 0.1,
    10 orbits.  Returns the largest |v_R - v_R,ref| over the steps, the
    reference being the midplane equations of motion with the gas velocity
    assigned analytically, integrated with an adaptive 8th-order Runge-Kutta
    method (scipy DOP853) to 1e-11."""
    from scipy.integrate import solve_ivp
    pp, qq, H0 = -1.0, -0.5, 0.1
    if geom == "cyl":
        edges = [np.linspace(0.2, 1.6, 65), np.array([0.0, 2 * np.pi]), np.linspace(-0.2, 0.2, 17)]
        prob = O.Problem(geom=O.OG_CYLINDRICAL, edges=edges, bc=(O.OB_OUTFLOW, 0, 0),
                         weight=weight, gm=1.0, species_tau_mode=(O.OT_STOKES,),
                         species_tau=(st,))
        R, _, Z = I._grid3(edges)
        r = np.hypot(R, Z)
    else:
        edges = [np.linspace(0.2, 1.8, 65), np.linspace(np.pi / 2 - 0.2, np.pi / 2 + 0.2, 17),
                 np.array([0.0, 2 * np.pi])]
        prob = O.Problem(geom=O.OG_SPHERICAL, edges=edges, bc=(O.OB_OUTFLOW, O.OB_OUTFLOW, 0),
                         weight=weight, gm=1.0, species_tau_mode=(O.OT_STOKES,),
                         species_tau=(st,))
        r, TH, _ = I._grid3(edges)
        R = r * np.sin(TH)
    H = H0 * R ** ((qq + 3) / 2)
    vphi = R * R ** -1.5 * np.sqrt((pp + qq) * (H / R) ** 2 + (1 + qq) - qq * R / r)
    zero = np.zeros_like(R)
    if geom == "cyl":
        pg = O.gas_momentum(prob, [zero, vphi, zero])
        q = [np.array([1.0]), np.array([0.0]), np.array([0.0])]
        p = [np.array([0.0]), np.array([1.0]), np.array([0.0])]
    else:
        pg = O.gas_momentum(prob, [zero, zero, vphi])
        q = [np.array([1.0]), np.array([np.pi / 2]), np.array([0.0])]
        p = [np.array([0.0]), np.array([0.0]), np.array([1.0])]
    rho = np.ones(prob.ncell)
    N = int(round(20 * np.pi / dt))
    active = np.ones(1, np.uint8)
    vr = [0.0]
    for s in range(N):
        O.step(prob, q, p, active, s * dt, dt, rho, pg)
        vr.append(p[0][0])

    def rhs(_, y):
        Rg, vR, l = y
        tau = st * Rg ** 1.5
        vg = Rg ** -0.5 * np.sqrt(1.0 + (pp + qq) * H0 ** 2 * Rg ** 0.5)
        return [vR, l * l / Rg ** 3 - 1.0 / Rg ** 2 - vR / tau, -(l - Rg * vg) / tau]
    t = np.arange(N + 1) * dt
    ref = solve_ivp(rhs, (0.0, t[-1]), [1.0, 0.0, 1.0], t_eval=t, rtol=1e-11, atol=1e-13,
                    method="DOP853").y[1]
    return np.abs(np.array(vr) - ref).max()


@pytest.mark.parametrize("geom,factor", [("cyl", 4.0), ("sph", 1.5)])
def test_radial_volume_weighting_has_the_largest_drift_error(geom, factor):
    """Sec. 4.5: of the weightings compared on the radial drift of an St = 1
    grain with dt = 0.1, the traditional volume weighting of Eq. CIC_vol
    gives the largest errors in v_R.  The paper reports TSC more than ten
    times better on its figure; here (same set-up, the weights of Sec. 3.4)
    volume weighting is 6.5 (cylindrical) and 1.7 (spherical) times worse
    than TSC, and worse than CIC, so the test asks for the ordering with the
    margin given."""
    vol = _drift_vr_error(geom, O.OW_VOLUME)
    cic = _drift_vr_error(geom, O.OW_CIC)
    tsc = _drift_vr_error(geom, O.OW_TSC)
    assert vol > factor * max(cic, tsc), (vol, cic, tsc)


def test_volume_weighting_is_cic_in_linear_coordinates():
    """The volume coordinate of a Cartesian direction is the coordinate
    itself: a Cartesian step with volume weighting equals the CIC step."""
    outs = []
    for weight in (O.OW_CIC, O.OW_VOLUME):
        prob = box_problem(n=(8, 8, 8), lo=-1.0, hi=1.0, geom=O.OG_CARTESIAN, weight=weight)
        rng = np.random.default_rng(3)
        rho = rng.uniform(0.5, 2.0, prob.ncell)
        _, pg = gas_uniform(prob, 1.0, (0.1, -0.2, 0.3))
        pg = [g + 0.1 * rng.standard_normal(prob.ncell) for g in pg]
        q0 = rng.uniform(-1.0, 1.0, (3, 20))
        p0 = 0.3 * rng.standard_normal((3, 20))
        q, p, _, dep = run(prob, q0, p0, 0.05, 3, rho, pg, param=np.full(20, 0.2))
        outs.append((np.ravel(q), np.ravel(p), dep))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
