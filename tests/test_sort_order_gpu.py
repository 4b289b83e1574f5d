"""The zone sort's order, checked against an independent host computation.

The store is sorted by zone key and, within a key, by grain id (the
deterministic order that replaces the per-cell linked list of Sec. 3).  The
key of a grain is the zone of its predicted half-step position (first half
drift, Eq. exp_midpoint and Eq. drift1_cylindrical) numbered tile by tile.
Here the host computes that zone with the oracle's zone search, and the
live grains read back after a step must come out exactly in the order
np.lexsort((ids, keys)), with removed grains after all of them.  A grain
whose half-step position lies within 1e-5 of a zone width of an edge may
take either zone (the library predicts keys in single precision relative to
the zone); the check then picks the key that keeps the order valid, if any.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_10793_gb300 import inputs as I
from parity_util import to_momentum

pytestmark = pytest.mark.gpu

BAND = 1e-5


def _half_drift(w, q, p, h):
    """First half drift of the momentum-like variables p (host, FP64)."""
    x = [a.astype(np.float64).copy() for a in q]
    if w.geom == O.OG_CYLINDRICAL:
        x[0] = x[0] + h * p[0]
        x[1] = x[1] + h * p[1] / (x[0] * x[0])
        x[2] = x[2] + h * p[2]
    elif w.geom == O.OG_SHEARING_BOX and w.fargo:
        x[0] = x[0] + h * p[0]
        x[1] = x[1] + h * (p[1] - w.qshear * w.omega * x[0])
        x[2] = x[2] + h * p[2]
    elif w.geom in (O.OG_CARTESIAN, O.OG_SHEARING_BOX):
        for d in range(3):
            x[d] = x[d] + h * p[d]
    else:
        raise ValueError("geometry not covered here")
    return x


def _zone_options(w, x, d):
    """Zone index of coordinate x in direction d (periodic wrap once, clamped
    onto the grid otherwise), and the neighbour it may also take when it lies
    within BAND of an edge (-1: none)."""
    e = w.edges[d]
    n = len(e) - 1
    if n <= 1:
        return np.zeros(len(x), np.int64), np.full(len(x), -1)
    lo, hi = e[0], e[-1]
    x = x.copy()
    if w.bc[d] == O.OB_PERIODIC:
        x = np.where(x >= hi, x - (hi - lo), np.where(x < lo, x + (hi - lo), x))
    # clamped onto the grid when outside it (outflow directions)
    x = np.where(x >= hi, e[-2], np.where(x < lo, lo, x))
    i = np.array([O.locate(e, float(v)) for v in x], np.int64)
    f = (x - e[i]) / (e[i + 1] - e[i])
    alt = np.full(len(x), -1)
    low, high = f < BAND, f > 1.0 - BAND
    periodic = w.bc[d] == O.OB_PERIODIC
    alt[low] = np.where(i[low] > 0, i[low] - 1, n - 1 if periodic else -1)
    alt[high] = np.where(i[high] < n - 1, i[high] + 1, 0 if periodic else -1)
    return i, alt


def _key(i, j, k, n, T):
    nt = [(n[d] + T[d] - 1) // T[d] for d in range(3)]
    tile = (i // T[0]) + nt[0] * ((j // T[1]) + nt[1] * (k // T[2]))
    loc = (i % T[0]) + T[0] * ((j % T[1]) + T[1] * (k % T[2]))
    return tile * (T[0] * T[1] * T[2]) + loc


def _allowed_keys(w, q, v, dt, T):
    p = to_momentum(w, q, v)
    x = _half_drift(w, q, p, 0.5 * dt)
    opts = [_zone_options(w, x[d], d) for d in range(3)]
    base = _key(opts[0][0], opts[1][0], opts[2][0], w.n, T)
    allowed = [[int(b)] for b in base]
    for g in np.nonzero((opts[0][1] >= 0) | (opts[1][1] >= 0) | (opts[2][1] >= 0))[0]:
        cand = set()
        for a in (opts[0][0][g], opts[0][1][g]):
            for b in (opts[1][0][g], opts[1][1][g]):
                for c in (opts[2][0][g], opts[2][1][g]):
                    if min(a, b, c) >= 0:
                        cand.add(int(_key(a, b, c, w.n, T)))
        allowed[g] = sorted(cand)
    return allowed, int(sum(len(a) > 1 for a in allowed))


def _check_order(ids_sorted, allowed_by_id, alive_by_id):
    """Live grains in (key, id) order, every key one of the grain's allowed
    keys (greedy: the smallest allowed key that keeps the order), removed
    grains after the live ones."""
    live = alive_by_id[ids_sorted]
    nlive = int(live.sum())
    assert np.all(live[:nlive]) and not np.any(live[nlive:]), "removed grains inside the order"
    cur_key, last_id = -1, -1
    for gid in ids_sorted[:nlive]:
        ok = [k for k in allowed_by_id[gid] if k > cur_key or (k == cur_key and gid > last_id)]
        assert ok, "grain %d out of order (keys %s after key %d, id %d)" % (
            gid, allowed_by_id[gid], cur_key, last_id)
        cur_key, last_id = ok[0], gid


CASES = {
    "box2d": (lambda: I.box2d("small"), (16, 16, 1)),
    "sbox3d": (lambda: I.sbox3d("small"), (8, 8, 8)),
    "sbox3d_tile844": (lambda: I.sbox3d("small"), (8, 4, 4)),
    "cyldisk": (lambda: I.cyldisk("small"), (8, 8, 8)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_sorted_order_is_lexsort_of_zone_key_and_id(name, precision):
    from paper_1908_10793_gb300 import dust as D
    make, tile = CASES[name]
    w = make()
    T = [min(tile[d], w.n[d]) if w.n[d] > 1 else 1 for d in range(3)]
    ctx = D.Context(w, precision=precision, tile=tile)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v, w.species, w.param)
        # the first step sorts the loaded store by the keys of (q^0, p^0); the
        # second by the keys the first step predicted from (q^1, p^1)
        q_prev = [x.copy() for x in w.q]
        v_prev = [x.copy() for x in w.v]
        alive_prev = np.ones(w.ngrains, bool)
        nambig = 0
        for s in range(3):
            ctx.step(w.dt)
            rc, _ = ctx.sync(check=False)
            assert rc in (0, -4)
            q, v, ids = ctx.particles()
            allowed, na = _allowed_keys(w, q_prev, v_prev, w.dt, T)
            nambig += na
            _check_order(ids, allowed, alive_prev)
            # the state after this step, by id, keys the next sort
            order = np.argsort(ids)
            q_prev = [x[order] for x in q]
            v_prev = [x[order] for x in v]
            alive_prev = ~np.isnan(q_prev[0])
            for d in range(3):
                q_prev[d][~alive_prev] = w.edges[d][0]
                v_prev[d][~alive_prev] = 0.0
        assert nambig <= 1e-3 * 3 * w.ngrains + 4
    finally:
        ctx.close()
