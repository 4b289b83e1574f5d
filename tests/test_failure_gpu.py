"""Failure detection on the GPU without a GPU fault.  The tile kernels wait
for their gas box (a bulk tensor copy completing on a transaction barrier)
with a time limit.  The testing option test_wait_timeout makes that wait run
out: the barrier expects 16 bytes the copy never brings, and the limit drops
to 1 ms.  The blocks give up, dust_sync reports DUST_ETIMEOUT with
DUST_FLAG_TIMEOUT, and the device stays usable: contexts stepped afterwards
give the same results as before."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I
from parity_util import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,kernel,predictor", [(1, 0, 0), (1, 2, 0), (0, 0, 0), (1, 0, 1)])
def test_bounded_gas_wait_runs_out_and_is_reported(precision, kernel, predictor):
    from paper_1908_10793_gb300 import dust as D
    w = I.sbox3d("small")
    before = run_gpu(w, 1, precision, kernel=kernel)
    ctx = D.Context(w, precision=precision, kernel=kernel, gas_predictor=predictor,
                    test_wait_timeout=1, feedback=0)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v)
        ctx.step(w.dt)
        rc, st = ctx.sync(check=False)
        assert rc == D.DUST_ETIMEOUT, rc
        assert st.flags & D.DUST_FLAG_TIMEOUT
        assert "wait" in D.dust_last_error(ctx.handle)
    finally:
        ctx.close()
    after = run_gpu(w, 1, precision, kernel=kernel)
    assert after["rc"] == 0
    for d in range(3):
        assert np.array_equal(before["q"][d], after["q"][d])
        assert np.array_equal(before["v"][d], after["v"][d])
    assert np.array_equal(before["fixed"], after["fixed"])
