"""Batched stepping as one persistent launch: a batch of streaming-instability
boxes (2-D x-z shearing boxes in the orbital-advection frame, mixed
precision) runs each dust_batch_step call as a single cooperative kernel
that takes every instance's sort, step and feedback work items from one
work list, each task waiting for its group's previous task to complete.
The grains, gas, deposit and counters must equal, bit for bit, those of the
same contexts stepped one at a time with dust_step, across calls with even
and odd step counts, a new step length, eager steps in between, and a sort
every second step.  The tasks' bounded wait is checked without a GPU fault:
a testing option makes every wait expect one item more than its task has,
the wait runs out, and every instance reports DUST_ETIMEOUT."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I
from test_batch_gpu import _assert_same, _state

pytestmark = pytest.mark.gpu


def _make(D, w, sort_interval=1, tile=None):
    kw = {} if tile is None else {"tile": tile}
    ctx = D.Context(w, precision=D.DUST_MIXED, sort_interval=sort_interval, **kw)
    ctx.set_gas(w.rho, w.vgas)
    ctx.load(w.q, w.v, w.species, w.param)
    return ctx


def _instances():
    # sizes 32^2 ... 512^2 (small scale: 16^2 ... 64^2) with 1-16 grains per
    # zone and the three Stokes numbers
    return [I.si2d_instance(k, "small") for k in range(11)]


@pytest.mark.parametrize("sort_interval", [1, 2])
def test_persistent_batch_equals_one_context_at_a_time(sort_interval):
    from paper_1908_10793_gb300 import dust as D
    ws = _instances()
    ref = [_make(D, w, sort_interval) for w in ws]
    bat = [_make(D, w, sort_interval) for w in ws]
    opt = D.dust_options(sort_interval=sort_interval)
    b = D.dust_batch_create([c.handle for c in bat], opt)
    try:
        dts = [w.dt for w in ws]
        calls = ((4, 1.0), (2, 1.0), (4, 0.5)) if sort_interval == 2 else \
            ((4, 1.0), (3, 1.0), (2, 0.5), (1, 0.5))
        for nsteps, scale in calls:
            dt = [x * scale for x in dts]
            D.dust_batch_step(b, dt, nsteps)
            for c, x in zip(ref, dt):
                for _ in range(nsteps):
                    c.step(x)
            for i, (c0, c1) in enumerate(zip(ref, bat)):
                _assert_same(_state(c0), _state(c1), (sort_interval, nsteps, scale, i))
        # eager steps in between (a whole sort period), then the batch again
        for c0, c1, x in zip(ref, bat, dts):
            for _ in range(sort_interval):
                c0.step(x)
                c1.step(x)
        D.dust_batch_step(b, dts, 2 * sort_interval)
        for c, x in zip(ref, dts):
            for _ in range(2 * sort_interval):
                c.step(x)
        for i, (c0, c1) in enumerate(zip(ref, bat)):
            _assert_same(_state(c0), _state(c1), ("after eager", i))
            rc, _ = c1.sync(check=False)
            assert rc in (0, D.DUST_ECFL)
    finally:
        D.dust_batch_destroy(b)
        for c in ref + bat:
            c.close()


@pytest.mark.parametrize("tile", [(16, 1, 16), (32, 1, 16)])
def test_persistent_batch_with_a_compiled_tile_shape(tile):
    """Every instance with the same 16 x 16 or 32 x 16 tile: the persistent
    launch runs the copy compiled for that shape, and still gives the
    one-at-a-time results bit for bit."""
    from paper_1908_10793_gb300 import dust as D
    if tile[0] == 16:
        ws = [I.si2d_instance(k, "small") for k in (1, 2, 4, 5, 7, 8)]   # 16^2 and 24^2
    else:
        ws = [I.si2d_instance(k) for k in (0, 5, 10, 15)]               # 32^2, 1-16 per zone
    ref = [_make(D, w, tile=tile) for w in ws]
    bat = [_make(D, w, tile=tile) for w in ws]
    b = D.dust_batch_create([c.handle for c in bat])
    try:
        dts = [w.dt for w in ws]
        for nsteps in (3, 2):
            D.dust_batch_step(b, dts, nsteps)
            for c, x in zip(ref, dts):
                for _ in range(nsteps):
                    c.step(x)
            for i, (c0, c1) in enumerate(zip(ref, bat)):
                _assert_same(_state(c0), _state(c1), (tile, nsteps, i))
    finally:
        D.dust_batch_destroy(b)
        for c in ref + bat:
            c.close()


def test_persistent_batch_task_wait_runs_out_and_is_reported():
    from paper_1908_10793_gb300 import dust as D
    ws = _instances()[:4]
    bat = [_make(D, w) for w in ws]
    try:
        opt = D.dust_options(test_wait_timeout=1)
        b = D.dust_batch_create([c.handle for c in bat], opt)
        try:
            D.dust_batch_step(b, [w.dt for w in ws], 2)
            for c in bat:
                rc, st = c.sync(check=False)
                assert rc == D.DUST_ETIMEOUT, rc
                assert st.flags & D.DUST_FLAG_TIMEOUT
        finally:
            D.dust_batch_destroy(b)
        # the device is still usable: reloaded contexts step through a new
        # batch like contexts stepped alone (at the same time: the failed
        # call advanced the batch contexts' time by two steps)
        ref = [_make(D, w) for w in ws]
        try:
            for c, w in zip(ref, ws):
                c.step(w.dt)
                c.step(w.dt)
            for c, w in zip(bat + ref, ws + ws):
                c.set_gas(w.rho, w.vgas)
                c.load(w.q, w.v, w.species, w.param)
            b = D.dust_batch_create([c.handle for c in bat])
            try:
                D.dust_batch_step(b, [w.dt for w in ws], 2)
                for c, w in zip(ref, ws):
                    c.step(w.dt)
                    c.step(w.dt)
                for i, (c0, c1) in enumerate(zip(ref, bat)):
                    s0, s1 = _state(c0), _state(c1)
                    for d in range(3):
                        assert np.array_equal(s0[0][d], s1[0][d]), (i, d)
                        assert np.array_equal(s0[1][d], s1[1][d]), (i, d)
                    assert np.array_equal(s0[2], s1[2]), i
            finally:
                D.dust_batch_destroy(b)
        finally:
            for c in ref:
                c.close()
    finally:
        for c in bat:
            c.close()
