"""Helpers shared by the GPU parity tests: run a workload through the oracle
and through the CUDA library (C interface) and compare."""
import numpy as np

import oracle as O


def default_quantum(w, precision):
    """The library's default fixed-point quantum: 2^-44 (FP64, precision 0) or
    2^-40 (mixed, precision 1) times the largest species mass."""
    return np.ldexp(max(abs(m) for m in w.species_mass), -44 if precision == 0 else -40)


def oracle_problem(w, feedback=None):
    return O.Problem(geom=w.geom, edges=w.edges, bc=w.bc, weight=w.weight,
                     species_mass=w.species_mass, species_tau_mode=w.species_tau_mode,
                     species_tau=w.species_tau, fargo=w.fargo, omega=w.omega, q=w.qshear,
                     gm=w.gm, vertical_gravity=w.vertical_gravity,
                     feedback_apply=w.feedback if feedback is None else feedback,
                     pusher=getattr(w, "pusher", O.OP_EM))


def to_momentum(w, q, v):
    """Physical velocity -> momentum-like variables (oracle side)."""
    p = [x.copy() for x in v]
    if w.geom == O.OG_CYLINDRICAL:
        p[1] = q[0] * v[1]
    if w.geom == O.OG_SPHERICAL:
        p[1] = q[0] * v[1]
        p[2] = q[0] * np.sin(q[1]) * v[2]
    return p


def to_physical(w, q, p):
    v = [x.copy() for x in p]
    if w.geom == O.OG_CYLINDRICAL:
        v[1] = p[1] / q[0]
    if w.geom == O.OG_SPHERICAL:
        v[1] = p[1] / q[0]
        v[2] = p[2] / (q[0] * np.sin(q[1]))
    return v


def run_oracle(w, steps, dt=None, feedback=None, predictor=False):
    """Returns (q, v physical, active, last deposit, gas pg).  predictor: the
    gas half-step drag predictor before every step; the step gathers from it
    and the feedback (if on) corrects the gas at t^n."""
    dt = w.dt if dt is None else dt
    fb = w.feedback if feedback is None else feedback
    prob = oracle_problem(w, 0 if predictor else feedback)
    q = [x.copy() for x in w.q]
    p = to_momentum(w, q, w.v)
    rho = w.rho.copy()
    pg = O.gas_momentum(prob, w.vgas)
    active = np.ones(w.ngrains, np.uint8)
    dep = None
    if predictor:
        dV = zone_volumes(w)
    for s in range(steps):
        if predictor:
            _, half = O.gas_predictor(prob, q, p, active, dt, rho, pg, w.species, w.param)
            dep, _ = O.step(prob, q, p, active, s * dt, dt, rho, half, w.species, w.param)
            if fb:
                pg = [pg[c] + dep[:, c] / (rho * dV) for c in range(3)]
        else:
            dep, _ = O.step(prob, q, p, active, s * dt, dt, rho, pg, w.species, w.param)
    return q, to_physical(w, q, p), active, dep, pg


def zone_volumes(w):
    """Zone volumes in storage order (R dR dphi dz, r^2 dr sin dtheta dphi)."""
    e = w.edges
    d = [np.diff(x) for x in e]
    if w.geom == O.OG_CYLINDRICAL:
        d[0] = 0.5 * np.diff(e[0] ** 2)
    elif w.geom == O.OG_SPHERICAL:
        d[0] = np.diff(e[0] ** 3) / 3.0
        d[1] = -np.diff(np.cos(e[1]))
    Z, Y, X = np.meshgrid(d[2], d[1], d[0], indexing="ij")
    return (X * Y * Z).ravel()


def run_gpu(w, steps, precision, dt=None, feedback=None, **kw):
    from paper_1908_10793_gb300 import dust as D
    dt = w.dt if dt is None else dt
    ctx = D.Context(w, precision=precision, feedback=feedback, **kw)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v, w.species, w.param)
        # dt may be a sequence of step lengths, one per step
        for s in range(steps):
            ctx.step(dt[s] if isinstance(dt, (list, tuple)) else dt)
        rc, st = ctx.sync(check=False)
        fixed, quantum = ctx.deposit()
        q, v, ids = ctx.particles()
        rho, vgas = ctx.gas()
    finally:
        ctx.close()
    order = np.argsort(ids)
    q = [x[order] for x in q]
    v = [x[order] for x in v]
    return dict(q=q, v=v, ids=ids[order], fixed=fixed, quantum=quantum, rc=rc, stats=st,
                rho=rho, vgas=vgas)


def periodic_diff(w, d, a, b):
    """a - b in direction d, reduced into (-L/2, L/2] for periodic directions."""
    diff = a - b
    if w.bc[d] == O.OB_PERIODIC:
        L = w.edges[d][-1] - w.edges[d][0]
        diff = diff - L * np.round(diff / L)
    return diff
