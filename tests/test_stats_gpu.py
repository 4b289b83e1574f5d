"""dust_sync's dust time step (Eq. particles_dt, Sec. 3.5): 1.8 over the
largest |v_d^{n+1/2}| / dl_d.  Grains drifting with the gas at a uniform
velocity keep that velocity exactly, so the expected value is known in closed
form; it is checked for both precisions and, with a faster grain added, it
follows the fastest grain."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _drifting_box(u):
    w = I.box2d("small")
    n = w.ngrains
    w.v = [np.full(n, u[0]), np.full(n, u[1]), np.zeros(n)]
    w.vgas = [np.full(w.ncell, u[0]), np.full(w.ncell, u[1]), np.zeros(w.ncell)]
    return w


@pytest.mark.parametrize("precision", [0, 1])
def test_dust_time_step_of_uniform_drift(precision):
    from paper_1908_10793_gb300 import dust as D
    u = (0.3, -0.7)
    w = _drifting_box(u)
    dx = [w.edges[d][1] - w.edges[d][0] for d in range(2)]
    expect = 1.8 / max(abs(u[0]) / dx[0], abs(u[1]) / dx[1])
    ctx = D.Context(w, precision=precision, feedback=0)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v)
        for _ in range(3):
            ctx.step(w.dt)
        rc, st = ctx.sync(check=False)
        assert rc == 0
        # the kernels track the displacement in single precision
        assert abs(st.dt_dust - expect) <= 1e-6 * expect, (st.dt_dust, expect)
        # a faster grain sets the next estimate
        v = [x.copy() for x in w.v]
        v[0][17] = 4.0
        ctx.load(w.q, v)
        ctx.step(w.dt)
        rc, st = ctx.sync(check=False)
        fast = 1.8 / max(4.0 / dx[0], abs(u[1]) / dx[1])
        # the fast grain is slowed by the drag during the step
        assert st.dt_dust < expect and st.dt_dust >= fast, (st.dt_dust, fast)
    finally:
        ctx.close()
