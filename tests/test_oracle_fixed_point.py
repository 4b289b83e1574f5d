"""Pins of the oracle's fixed-point deposit rule (CPU only).

The paper deposits the drag back-reaction in floating point (Eq.
dust_feedback_final); this project also states it in integers so that the
deposited grid does not depend on the order of the grains.  Per grain and
channel, in units of the quantum: the non-host nodes get the nearest
integer of W_j D, the host zone the rest of the nearest integer of D.  What
fixes it without re-typing it:

* the zones of one grain receive exactly the nearest integer of that
  grain's total impulse, and a whole step deposits the sum of these
  integers (integer equality, i.e. momentum conserved to the quantum);
* each piece is within half a quantum of its exact share, and the host
  zone within half a quantum per piece of its own;
* the integers do not depend on the order of the grains, and a step of all
  grains equals the sum of the steps of the grains one at a time;
* a grain at a zone centre has the dyadic TSC weights 1/8, 3/4, 1/8 per
  direction, whose pieces of an impulse that is a whole number of quanta
  are known in closed form;
* fixed point times the quantum tends to the dense deposit as the quantum
  shrinks.
"""
import numpy as np

import oracle as O
from paper_1908_10793_gb300 import inputs as I


def _state(w):
    prob = O.Problem(geom=w.geom, edges=w.edges, bc=w.bc, weight=w.weight,
                     species_mass=w.species_mass, species_tau_mode=w.species_tau_mode,
                     species_tau=w.species_tau, fargo=w.fargo, omega=w.omega, q=w.qshear,
                     gm=w.gm, vertical_gravity=w.vertical_gravity, feedback_apply=0)
    q = [x.copy() for x in w.q]
    p = [x.copy() for x in w.v]
    if w.geom == O.OG_CYLINDRICAL:
        p[1] = q[0] * w.v[1]
    pg = O.gas_momentum(prob, w.vgas)
    return prob, q, p, w.rho.copy(), pg


def _one_by_one(prob, q, p, dt, rho, pg, quantum, species=None, idx=None):
    """Per-grain dense and fixed deposits, each grain stepped alone."""
    n = len(q[0])
    idx = range(n) if idx is None else idx
    out = []
    for g in idx:
        qq = [np.array([x[g]]) for x in q]
        pp = [np.array([x[g]]) for x in p]
        sp = None if species is None else species[g:g + 1]
        dep, fx, _ = O.step_fixed(prob, qq, pp, np.ones(1, np.uint8), 0.0, dt, rho,
                                  [x.copy() for x in pg], quantum, species=sp)
        out.append((dep, fx))
    return out


def test_each_grain_deposits_the_nearest_integer_of_its_impulse():
    w = I.sbox3d("small")
    w = I.subsample(w, 64)
    prob, q, p, rho, pg = _state(w)
    quantum = 2.0 ** -44 * max(w.species_mass)
    for dep, fx in _one_by_one(prob, q, p, w.dt, rho, pg, quantum):
        D = dep.sum(axis=0) / quantum          # the grain's impulse in quanta
        tot = fx.sum(axis=0)
        assert np.all(np.abs(tot - D) <= 0.5 + 1e-9 * np.abs(D))
        # every piece within half a quantum of its exact share; one zone per
        # channel (the host) carries the others' rounding as well
        err = np.abs(fx - dep / quantum)
        tol = 1e-9 * np.abs(D).max()
        assert np.all(fx[np.all(dep == 0.0, axis=1)] == 0)
        for ch in range(4):
            st = np.nonzero(dep[:, ch])[0]
            assert len(st) == 27
            assert (err[st, ch] > 0.5 + tol).sum() <= 1
            assert err[st, ch].max() <= 0.5 * 27 + tol


def test_step_deposit_is_the_sum_of_the_grains_integers_in_any_order():
    w = I.box2d("small")
    w = I.subsample(w, 200)
    prob, q, p, rho, pg = _state(w)
    quantum = 2.0 ** -44 * max(w.species_mass)
    _, fx_all, _ = O.step_fixed(prob, [x.copy() for x in q], [x.copy() for x in p],
                                np.ones(w.ngrains, np.uint8), 0.0, w.dt, rho,
                                [x.copy() for x in pg], quantum)
    per = _one_by_one(prob, q, p, w.dt, rho, pg, quantum)
    assert np.array_equal(fx_all, sum(f for _, f in per))
    # the step's total is the sum of each grain's nearest integer
    nearest = sum(np.rint(d.sum(axis=0) / quantum) for d, _ in per)
    assert np.all(np.abs(fx_all.sum(axis=0) - nearest) <= 1e-9 * np.abs(nearest) + 1)
    perm = np.random.default_rng(4).permutation(w.ngrains)
    _, fx_perm, _ = O.step_fixed(prob, [x[perm].copy() for x in q], [x[perm].copy() for x in p],
                                 np.ones(w.ngrains, np.uint8), 0.0, w.dt, rho,
                                 [x.copy() for x in pg], quantum)
    assert np.array_equal(fx_all, fx_perm)


def test_zone_centre_grain_has_closed_form_pieces():
    # 3-D Cartesian periodic box, one grain that sits at a zone centre at the
    # half step (zero velocity) in uniform gas with velocity along x: the
    # impulse is D = -m (v^{n+1} - v^n) along x only.  Weights per direction
    # (1/8, 3/4, 1/8), so W_j is one of 1/512, 3/256, 9/128, 27/64 (host).
    n = 4
    edges = [np.linspace(0.0, 1.0, n + 1) for _ in range(3)]
    tau, dt, m = 0.5, 0.1, 1.0
    prob = O.Problem(geom=O.OG_CARTESIAN, edges=edges, weight=O.OW_TSC, species_mass=(m,),
                     species_tau=(tau,))
    rho = np.ones(n ** 3)
    pg = [np.full(n ** 3, 0.25), np.zeros(n ** 3), np.zeros(n ** 3)]
    c = 0.375   # centre of zone 1
    q = [np.array([c]), np.array([c]), np.array([c])]
    p = [np.zeros(1), np.zeros(1), np.zeros(1)]
    D = -m * 0.25 * (-np.expm1(-dt / tau))
    quantum = abs(D) / 123456789.0   # D is -123456789 quanta (to rounding)
    dep, fx, _ = O.step_fixed(prob, q, p, np.ones(1, np.uint8), 0.0, dt, rho, pg, quantum)
    Dq = round(D / quantum)
    assert Dq == -123456789
    fx3 = fx[:, 0].reshape(n, n, n)   # [k, j, i]
    host = (1, 1, 1)
    wts = {0: 0.125, 1: 0.75, 2: 0.125}
    rest = Dq
    for k in range(3):
        for j in range(3):
            for i in range(3):
                if (i, j, k) == (1, 1, 1):
                    continue
                Wj = wts[i] * wts[j] * wts[k]
                piece = int(np.rint(Wj * D / quantum))
                assert fx3[k, j, i] == piece, (i, j, k)
                rest -= piece
    assert fx3[host] == rest
    assert np.all(fx[:, 1:3] == 0)
    assert fx[:, 0].sum() == Dq


def test_fixed_point_tends_to_the_dense_deposit():
    w = I.box2d("small")
    w = I.subsample(w, 300)
    prob, q, p, rho, pg = _state(w)
    errs = []
    for k in (30, 38, 46):
        quantum = 2.0 ** -k * max(w.species_mass)
        dep, fx, _ = O.step_fixed(prob, [x.copy() for x in q], [x.copy() for x in p],
                                  np.ones(w.ngrains, np.uint8), 0.0, w.dt, rho,
                                  [x.copy() for x in pg], quantum)
        errs.append(np.abs(fx * quantum - dep).max())
        # at most half a quantum per piece a zone can receive
        assert errs[-1] <= 0.5 * 9 * w.ngrains * quantum
    assert errs[0] > 100 * errs[1] > 10000 * errs[2]
