"""dust_options.host_io_async: host-memory loads and read-backs only enqueue
their copies (two copy streams, double-buffered outputs) and dust_sync waits
for them.  A pipelined loop (load, set gas, step, read back, without waiting)
must give, after dust_sync, exactly the results of the synchronous calls, and
invalid grains must be dropped and reported by dust_sync."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def _loop(w, async_io, steps, precision):
    """Every step: load the grains and the gas from host buffers, step, read
    the grains and the deposit back.  Returns the host outputs of each step."""
    from paper_1908_10793_gb300 import dust as D
    ctx = D.Context(w, precision=precision, host_io_async=async_io, feedback=0)
    n = w.ngrains
    hq = [_pinned(x) for x in w.q]
    hv = [_pinned(x) for x in w.v]
    hs = _pinned(w.species) if w.species is not None else None
    hp = _pinned(w.param) if w.param is not None else None
    hrho = _pinned(w.rho)
    hg = [_pinned(x) for x in w.vgas]
    outs = [([_pinned(np.zeros(n)) for _ in range(6)], _pinned(np.zeros(n, np.int64)),
             _pinned(np.zeros((w.ncell, 4), np.int64))) for _ in range(steps)]
    try:
        for k in range(steps):
            D.dust_load_particles(ctx.handle, *hq, *hv, hs, hp)
            D.dust_set_gas(ctx.handle, hrho, *hg)
            D.dust_step(ctx.handle, w.dt * (1 + k))
            o, ids, dep = outs[k]
            D.dust_get_particles(ctx.handle, n, *o, ids=ids)
            D.dust_get_deposit(ctx.handle, fixed=dep)
        rc, _ = ctx.sync(check=False)
    finally:
        ctx.close()
    assert rc in (0, D.DUST_ECFL)
    return outs


@pytest.mark.parametrize("name", ["box2d", "cyldisk", "sphdisk"])
@pytest.mark.parametrize("precision", [0, 1])
def test_async_host_io_matches_synchronous_calls(name, precision):
    w = {"box2d": I.box2d, "cyldisk": I.cyldisk, "sphdisk": I.sphdisk}[name]("small")
    steps = 3
    sync = _loop(w, 0, steps, precision)
    asyn = _loop(w, 1, steps, precision)
    for k in range(steps):
        (os_, ids_s, dep_s), (oa, ids_a, dep_a) = sync[k], asyn[k]
        assert np.array_equal(ids_s, ids_a), k
        for d in range(6):
            assert np.array_equal(os_[d], oa[d], equal_nan=True), (k, d)
        assert np.array_equal(dep_s, dep_a), k


def test_async_load_drops_invalid_grains_and_reports_at_sync():
    from paper_1908_10793_gb300 import dust as D
    w = I.box2d("small")
    q = [x.copy() for x in w.q]
    q[0][5] = np.nan
    q[1][7] = w.edges[1][-1] + 1.0       # outside the grid
    ctx = D.Context(w, precision=D.DUST_MIXED, host_io_async=1, feedback=0)
    try:
        D.dust_load_particles(ctx.handle, *[_pinned(x) for x in q], *[_pinned(x) for x in w.v])
        ctx.n = w.ngrains
        D.dust_set_gas(ctx.handle, _pinned(w.rho), *[_pinned(x) for x in w.vgas])
        D.dust_step(ctx.handle, w.dt)
        rc, st = ctx.sync(check=False)
        assert rc == D.DUST_EINVAL
        assert st.n_removed >= 2
        # reported once; the context keeps working
        D.dust_step(ctx.handle, w.dt)
        rc2, _ = ctx.sync(check=False)
        assert rc2 in (0, D.DUST_ECFL)
        qo, _, ids = ctx.particles()
        ctx.sync(check=False)              # the read-back is asynchronous too
        assert np.isnan(qo[0][ids == 5][0]) and np.isnan(qo[0][ids == 7][0])
        assert np.isfinite(qo[0][ids == 6][0])
    finally:
        ctx.close()
