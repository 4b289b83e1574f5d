"""Zone sort with very dense zones: a clump of 50,000 grains in one zone and
a few hundred to a few thousand in others, as the clumps of the streaming
instability produce (Sec. 4.3 setups).  Segments longer than the warp's
staging go to the block sort (bitonic chunks and merge passes); the order
must still be exactly (zone key, id) against the host computation, and the
step must still match the oracle.  The sort's time on the clump is printed.  A
second case puts 70,000 grains in one zone: its tile then holds more than
65535 grains, so the step kernel keeps that tile's deposit box as int64 words
(the form for dense tiles) instead of the two carry-free 32-bit counters."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I
from test_sort_order_gpu import _allowed_keys, _check_order

pytestmark = pytest.mark.gpu

CLUMPS = (((7, 7, 7), 50_000), ((3, 9, 12), 3_000), ((12, 2, 5), 600), ((1, 14, 3), 100),
          ((10, 10, 1), 40))
DENSE_TILE = (((7, 7, 7), 70_000),)


def _clumped_box(seed=5, clumps=CLUMPS):
    import copy
    w = copy.copy(I.sbox3d("small"))
    r = np.random.Generator(np.random.Philox(seed))
    q = [np.asarray(x) for x in w.q]
    v = [np.asarray(x) for x in w.v]
    add_q = [[], [], []]
    add_v = [[], [], []]
    for (i, j, k), m in clumps:
        for d, c in enumerate((i, j, k)):
            lo, hi = w.edges[d][c], w.edges[d][c + 1]
            # inside the zone, away from its edges, slow: the half step keeps
            # them in it
            add_q[d].append(lo + (hi - lo) * r.uniform(0.2, 0.8, m))
            add_v[d].append(1e-4 * r.standard_normal(m))
    # the clump grains interleaved with the others in id order
    w.q = [np.concatenate([q[d]] + add_q[d]) for d in range(3)]
    w.v = [np.concatenate([v[d]] + add_v[d]) for d in range(3)]
    perm = r.permutation(len(w.q[0]))
    w.q = [x[perm].copy() for x in w.q]
    w.v = [x[perm].copy() for x in w.v]
    return w


@pytest.mark.parametrize("clumps", [CLUMPS, DENSE_TILE], ids=["clumps", "dense_tile"])
@pytest.mark.parametrize("precision", [0, 1])
def test_dense_zones_sort_in_key_and_id_order_and_match_the_oracle(precision, clumps):
    from paper_1908_10793_gb300 import dust as D
    from test_parity_gpu import check_against_oracle
    from parity_util import run_oracle
    w = _clumped_box(clumps=clumps)
    T = (8, 8, 8)
    ctx = D.Context(w, precision=precision, tile=T, timing=1, feedback=0)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v)
        ctx.kernel_times(reset=True)
        ctx.step(w.dt)
        rc, st = ctx.sync(check=False)
        kt = ctx.kernel_times(reset=True)
        q, v, ids = ctx.particles()
        fixed, quantum = ctx.deposit()
        allowed, _ = _allowed_keys(w, w.q, w.v, w.dt, T)
        _check_order(ids, allowed, np.ones(w.ngrains, bool))
        print("dense sort: %d grains, sort %.3f ms, step %.3f ms" % (
            w.ngrains, kt.sort_ms, kt.step_ms))
        order = np.argsort(ids)
        g = dict(q=[x[order] for x in q], v=[x[order] for x in v], fixed=fixed,
                 quantum=quantum, rc=rc)
        qo, vo, active, dep_o, _ = run_oracle(w, 1, feedback=0)
        check_against_oracle(w, g, (qo, vo, active, dep_o), 1, precision, w.dt)
    finally:
        ctx.close()
