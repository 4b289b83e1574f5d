"""Batched stepping (dust_batch_*): several independent instances advanced
through one captured graph give, bit for bit, what stepping each context on
its own with dust_step gives (same kernels, same sort order, the time and
shear-periodic shifts read from the device instead of the arguments)."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _instances():
    ws = [I.si2d_instance(k, "small") for k in range(5)]
    # other geometries and a grain leaving through the outflow boundary
    cyl = I.subsample(I.cyldisk("small"), 3000)
    cyl.q[0][:50] = cyl.edges[0][0] + 1e-5
    cyl.v[0][:50] = -0.5
    ws.append(cyl)
    ws.append(I.box2d("small"))
    return ws


def _make(D, w, precision, **kw):
    ctx = D.Context(w, precision=precision, sort_interval=1, **kw)
    ctx.set_gas(w.rho, w.vgas)
    ctx.load(w.q, w.v, w.species, w.param)
    return ctx


def _state(ctx):
    q, v, ids = ctx.particles()
    o = np.argsort(ids)
    fixed, _ = ctx.deposit()
    rho, vg = ctx.gas()
    _, st = ctx.sync(check=False)
    return [x[o] for x in q], [x[o] for x in v], fixed, vg, st


def _assert_same(a, b, what):
    for d in range(3):
        assert np.array_equal(a[0][d], b[0][d], equal_nan=True), (what, "q", d)
        assert np.array_equal(a[1][d], b[1][d], equal_nan=True), (what, "v", d)
        assert np.array_equal(a[3][d], b[3][d]), (what, "gas", d)
    assert np.array_equal(a[2], b[2]), (what, "deposit")
    assert a[4].steps == b[4].steps and a[4].time == b[4].time, what
    assert a[4].n_removed == b[4].n_removed, what


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_one_context_at_a_time(precision):
    from paper_1908_10793_gb300 import dust as D
    ws = _instances()
    ref = [_make(D, w, precision) for w in ws]
    bat = [_make(D, w, precision) for w in ws]
    b = D.dust_batch_create([c.handle for c in bat])
    try:
        dts = [w.dt for w in ws]
        done = 0
        # two replays; an odd count (graph then one eager step); a new step
        # length (capture again); a step on its own in between
        for nsteps, scale in ((4, 1.0), (3, 1.0), (2, 0.5), (2, 0.5)):
            dt = [x * scale for x in dts]
            D.dust_batch_step(b, dt, nsteps)
            for c, x in zip(ref, dt):
                for _ in range(nsteps):
                    c.step(x)
            done += nsteps
            for i, (c0, c1) in enumerate(zip(ref, bat)):
                _assert_same(_state(c0), _state(c1), (nsteps, scale, i))
        for c0, c1, x in zip(ref, bat, dts):
            c0.step(x)
            c1.step(x)
        D.dust_batch_step(b, dts, 2)
        for c, x in zip(ref, dts):
            c.step(x)
            c.step(x)
        for i, (c0, c1) in enumerate(zip(ref, bat)):
            _assert_same(_state(c0), _state(c1), ("after eager", i))
        assert _state(bat[5])[4].n_removed >= 50
    finally:
        D.dust_batch_destroy(b)
        for c in ref + bat:
            c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_with_the_gas_predictor_equals_one_context_at_a_time(precision):
    """The gas predictor inside the captured graph (in mixed precision with its
    own sort by the zone at x^n): grains, gas and deposit bit for bit as the
    contexts stepped one at a time, across replays, an odd step count and
    eager steps in between."""
    from paper_1908_10793_gb300 import dust as D
    ws = [I.si2d_instance(k, "small") for k in range(4)] + [I.subsample(I.cyldisk("small"), 3000)]
    ref = [_make(D, w, precision, gas_predictor=1) for w in ws]
    bat = [_make(D, w, precision, gas_predictor=1) for w in ws]
    b = D.dust_batch_create([c.handle for c in bat])
    try:
        dts = [w.dt for w in ws]
        for nsteps in (4, 3):
            D.dust_batch_step(b, dts, nsteps)
            for c, x in zip(ref, dts):
                for _ in range(nsteps):
                    c.step(x)
            for i, (c0, c1) in enumerate(zip(ref, bat)):
                _assert_same(_state(c0), _state(c1), (nsteps, i))
        for c0, c1, x in zip(ref, bat, dts):
            c0.step(x)
            c1.step(x)
        D.dust_batch_step(b, dts, 2)
        for c, x in zip(ref, dts):
            c.step(x)
            c.step(x)
        for i, (c0, c1) in enumerate(zip(ref, bat)):
            _assert_same(_state(c0), _state(c1), ("after eager", i))
    finally:
        D.dust_batch_destroy(b)
        for c in ref + bat:
            c.close()


def test_batch_rejects_bad_arguments():
    from paper_1908_10793_gb300 import dust as D
    w = I.si2d_instance(0, "small")
    c = _make(D, w, 1)
    try:
        with pytest.raises(D.DustError) as e:
            D.dust_batch_create([c.handle, c.handle])
        assert e.value.code == D.DUST_EINVAL
        b = D.dust_batch_create([c.handle])
        try:
            with pytest.raises(D.DustError) as e:
                D.dust_batch_step(b, [float("nan")], 2)
            assert e.value.code == D.DUST_EINVAL
            D.dust_batch_step(b, [w.dt], 0)
        finally:
            D.dust_batch_destroy(b)
        fresh = D.Context(w, precision=1)
        try:
            b = D.dust_batch_create([fresh.handle])
            with pytest.raises(D.DustError) as e:
                D.dust_batch_step(b, [w.dt], 2)
            assert e.value.code == D.DUST_ESTATE
            D.dust_batch_destroy(b)
        finally:
            fresh.close()
    finally:
        c.close()
