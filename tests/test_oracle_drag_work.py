"""Pins of the oracle's deposit channels in the shearing box, in both frames,
and of the Epstein stopping time, against references built outside the
oracle (CPU only):

* the momentum-like channels are minus the drag impulse and the energy
  channel is minus the drag work, sum_c (drag impulse)_c dH/dp_c, along the
  grain's trajectory (Eq. dust_feedback_final; energy: the reading that the
  fourth channel is the deposited impulse times the half-step dH/dp).  The
  reference integrates the equations of motion of the frame (orbital
  advection, Eq. FARGO_SB_p; standard frame, Eq. standard_SB_g) with an
  adaptive high-order solver, with the gas velocity interpolated by the
  textbook TSC spline (Eq. b1) at the grain's position.  A second-order step
  must reproduce both integrals to O(dt^3) per step, which step halving
  shows; a wrong frame velocity in the energy channel, a wrong
  non-frictional force or an end-point value leaves O(dt) or O(dt^2);
* Epstein drag, tau_s = value / rho (Sec. 2, tau_s proportional to 1/rho):
  the density is the one gathered at x^{n+1/2} by the TSC weights, so a
  grain in uniform gas flow relaxes exactly like a constant-tau grain with
  that tau.
"""
import numpy as np
import pytest

import oracle as O

scipy_integrate = pytest.importorskip("scipy.integrate")


def _tsc_periodic(field, n, lo, hi, x):
    """Textbook TSC interpolation (b1 spline of width one zone) of a
    periodic gridded field [n2, n1, n0] at the point x (3 coordinates)."""
    w, idx = [], []
    for d in range(3):
        dx = (hi - lo) / n[d]
        s = (x[d] - lo) / dx
        i = int(np.floor(s))
        dl = s - (i + 0.5)
        w.append([0.5 * (0.5 - dl) ** 2, 0.75 - dl * dl, 0.5 * (0.5 + dl) ** 2])
        idx.append([(i - 1 + k) % n[d] for k in range(3)])
    v = 0.0
    for c in range(3):
        for b in range(3):
            for a in range(3):
                v += w[0][a] * w[1][b] * w[2][c] * field[idx[2][c], idx[1][b], idx[0][a]]
    return v


def _drag_integrals(fargo, vgrav, x0, v0, pg3, n, lo, hi, tau, dt, Om=1.0, qs=1.5):
    """Drag impulse and drag work per unit mass over one step of length dt,
    from the frame's equations of motion integrated to 1e-13.  The work is
    the drag acceleration dotted with the frame's own velocity (v in the
    standard frame, the residual velocity v' in the orbital-advection frame)."""
    def rhs(t, s):
        x, v = s[0:3], s[3:6]
        vg = np.array([_tsc_periodic(pg3[c], n, lo, hi, x) for c in range(3)])
        f = (vg - v) / tau
        if fargo:   # Eq. FARGO_SB_p: dy/dt = v'_y - q Omega x
            dx = [v[0], v[1] - qs * Om * x[0], v[2]]
            a = [2.0 * Om * v[1], (qs - 2.0) * Om * v[0]]
        else:       # standard frame: Coriolis plus tidal force
            dx = [v[0], v[1], v[2]]
            a = [2.0 * Om * (v[1] + qs * Om * x[0]), -2.0 * Om * v[0]]
        az = -Om * Om * x[2] if vgrav else 0.0
        dv = [a[0] + f[0], a[1] + f[1], az + f[2]]
        return np.concatenate([dx, dv, f, [f @ v]])

    s0 = np.concatenate([x0, v0, np.zeros(4)])
    sol = scipy_integrate.solve_ivp(rhs, (0.0, dt), s0, method="DOP853", rtol=1e-13,
                                    atol=1e-16)
    assert sol.success
    return sol.y[6:9, -1], sol.y[9, -1]


@pytest.mark.parametrize("fargo,vgrav", [(1, 0), (1, 1), (0, 0), (0, 1)])
def test_deposit_channels_are_minus_drag_impulse_and_work_at_third_order(fargo, vgrav):
    n, lo, hi = (8, 8, 8), -0.5, 0.5
    mass, tau = 0.3, 0.1
    edges = [np.linspace(lo, hi, k + 1) for k in n]
    prob = O.Problem(geom=O.OG_SHEARING_BOX, edges=edges, weight=O.OW_TSC, fargo=fargo,
                     omega=1.0, q=1.5, vertical_gravity=vgrav, species_mass=(mass,),
                     species_tau=(tau,))
    rng = np.random.default_rng(11)
    rho = rng.uniform(0.8, 1.2, prob.ncell)
    # gas velocity of the frame (residual in the orbital-advection frame)
    pg = [0.05 * rng.uniform(-1.0, 1.0, prob.ncell) + off for off in (0.02, -0.03, 0.01)]
    pg3 = [x.reshape(n[2], n[1], n[0]) for x in pg]
    x0 = np.array([0.07, -0.03, 0.05])
    v0 = np.array([0.11, -0.08, 0.04])

    def one(dt):
        q = [np.array([x]) for x in x0]
        p = [np.array([x]) for x in v0]
        dep, removed = O.step(prob, q, p, np.ones(1, np.uint8), 0.0, dt, rho,
                              [x.copy() for x in pg])
        assert removed == 0
        imp, work = _drag_integrals(fargo, vgrav, x0, v0, pg3, n, lo, hi, tau, dt)
        dP = dep[:, :3].sum(axis=0)
        dE = dep[:, 3].sum()
        return dP, -mass * imp, dE, -mass * work

    res = [one(h) for h in (0.02, 0.01, 0.005)]
    for dP, rP, dE, rE in res:
        assert np.abs(rP).max() > 1e-4 and abs(rE) > 1e-6   # the drag really acted
        assert np.abs(dP - rP).max() < 1e-3 * np.abs(rP).max()
        assert abs(dE - rE) < 1e-3 * abs(rE)
    # local error O(dt^3): halving dt divides it by about 8.  In the standard
    # frame the energy channel's local error changes sign between these
    # steps (its size is checked above; the grain's mechanical-energy change
    # pins that channel at third order in test_oracle_push.py)
    for k in range(2):
        eP = [np.abs(r[0] - r[1]).max() for r in res[k:k + 2]]
        assert eP[0] > 6.0 * eP[1], (fargo, vgrav, eP)
        if fargo:
            eE = [abs(r[2] - r[3]) for r in res[k:k + 2]]
            assert eE[0] > 6.0 * eE[1], (fargo, vgrav, eE)


def _epstein_problem(mode, value):
    n = 16
    edges = [np.linspace(0.0, 1.0, n + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    return O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC,
                     species_tau_mode=(mode,), species_tau=(value,)), n, edges


def _tsc_1d(field, n, x):
    i = int(np.floor(x * n))
    dl = x * n - (i + 0.5)
    w = [0.5 * (0.5 - dl) ** 2, 0.75 - dl * dl, 0.5 * (0.5 + dl) ** 2]
    return sum(w[k] * field[(i - 1 + k) % n] for k in range(3)), i


def test_epstein_stopping_time_uses_the_density_gathered_at_the_half_step():
    c = 0.07
    prob, n, edges = _epstein_problem(O.OT_EPSTEIN, c)
    xc = 0.5 * (edges[0][1:] + edges[0][:-1])
    rho = 1.0 + 0.6 * np.sin(2 * np.pi * xc)
    vg = (0.3, -0.1, 0.05)
    pg = [np.full(n, v) for v in vg]
    x0 = np.array([0.13, 0.41, 0.77, 0.52])
    v0 = [np.array([0.9, -1.3, 0.4, 2.1]), np.array([0.2, 0.0, -0.3, 0.1]),
          np.array([0.0, 0.5, 0.1, -0.2])]
    dt = 0.05
    q = [x0.copy(), np.full(4, 0.5), np.full(4, 0.5)]
    p = [x.copy() for x in v0]
    O.step(prob, q, p, np.ones(4, np.uint8), 0.0, dt, rho, [x.copy() for x in pg])
    for g in range(4):
        xm = x0[g] + 0.5 * dt * v0[0][g]
        rt, host = _tsc_1d(rho, n, xm)
        E = np.exp(-dt * rt / c)
        for d in range(3):
            expect = vg[d] + (v0[d][g] - vg[d]) * E
            assert abs(p[d][g] - expect) < 1e-14 * (1.0 + abs(v0[d][g])), (g, d)
        assert abs(q[0][g] - (xm + 0.5 * dt * p[0][g])) < 1e-15
        # the test can tell the gathered density from the host zone's and
        # from the density gathered at x^n
        r0, _ = _tsc_1d(rho, n, x0[g])
        for other in (rho[host % n], r0):
            alt = vg[0] + (v0[0][g] - vg[0]) * np.exp(-dt * other / c)
            assert abs(alt - p[0][g]) > 1e-6


def test_epstein_in_uniform_density_equals_constant_stopping_time():
    c, rho0 = 0.07, 2.5
    rng = np.random.default_rng(2)
    x0 = rng.uniform(0.0, 1.0, 6)
    v0 = [rng.normal(0.0, 1.0, 6) for _ in range(3)]
    out = []
    for mode, value in ((O.OT_EPSTEIN, c), (O.OT_CONST, c / rho0)):
        prob, n, _ = _epstein_problem(mode, value)
        q = [x0.copy(), np.full(6, 0.5), np.full(6, 0.5)]
        p = [x.copy() for x in v0]
        dep, _ = O.step(prob, q, p, np.ones(6, np.uint8), 0.0, 0.05, np.full(n, rho0),
                        [np.full(n, 0.3), np.full(n, -0.1), np.zeros(n)])
        out.append(np.concatenate([np.ravel(q), np.ravel(p), dep.ravel()]))
    # the gathered density is a sum of weights times rho0, equal to rho0 up
    # to rounding of the weights' sum
    scale = np.maximum(np.abs(out[1]), 1e-3)
    assert np.all(np.abs(out[0] - out[1]) <= 1e-14 * scale)


def test_epstein_predictor_uses_the_density_gathered_at_x_n():
    # Sec. 3.1 predictor: impulse dt/2 m / max(tau, dt) (v_p - v_g) with
    # tau = value / rho~(x^n); uniform gas velocity, so the zones' impulses
    # sum to the grain's
    c, dt, m = 0.9, 0.05, 1.0
    prob, n, edges = _epstein_problem(O.OT_EPSTEIN, c)
    xc = 0.5 * (edges[0][1:] + edges[0][:-1])
    rho = 1.0 + 0.6 * np.sin(2 * np.pi * xc)
    vg = (0.3, -0.1, 0.05)
    x0, v0 = 0.37, (1.1, 0.4, -0.2)
    imp, _ = O.gas_predictor(prob, [np.array([x0]), np.array([0.5]), np.array([0.5])],
                             [np.array([v]) for v in v0], np.ones(1, np.uint8), dt, rho,
                             [np.full(n, v) for v in vg])
    rt, _ = _tsc_1d(rho, n, x0)
    tau = c / rt
    assert tau > dt
    expect = np.array([0.5 * dt * m / tau * (v0[k] - vg[k]) for k in range(3)])
    assert np.allclose(imp.sum(axis=0), expect, rtol=1e-13, atol=0)
