"""Particle load and read-back with float32 velocity arrays
(dust_load_particles_v32 / dust_get_particles_v32).

Loading float32 velocities must store exactly what dust_load_particles
stores when given the same values widened to float64, in every geometry and
in both host I/O modes; reading back into float32 must give the float64
read-back rounded to float32.  Two mixed-precision steps are taken between
load and read-back, so the stored state is also checked through the step
(positions, velocities, ids and the deposit integers)."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "sbox3d": lambda: I.sbox3d("small"),
    "cyldisk": lambda: I.cyldisk("small"),
    "sphdisk": lambda: I.sphdisk("small"),
}


def _run(D, w, v, loader, host_io_async, steps=2):
    ctx = D.Context(w, precision=D.DUST_MIXED, host_io_async=host_io_async)
    try:
        ctx.set_gas(w.rho, w.vgas)
        loader(ctx.handle, *w.q, *v, getattr(w, "species", None), getattr(w, "param", None))
        for _ in range(steps):
            ctx.step(w.dt)
        ctx.sync()
        n = w.ngrains
        q = [np.empty(n) for _ in range(3)]
        v64 = [np.empty(n) for _ in range(3)]
        v32 = [np.empty(n, np.float32) for _ in range(3)]
        ids64 = np.empty(n, np.int64)
        ids32 = np.empty(n, np.int64)
        q32 = [np.empty(n) for _ in range(3)]
        D.dust_get_particles(ctx.handle, n, *q, *v64, ids=ids64)
        D.dust_get_particles_v32(ctx.handle, n, *q32, *v32, ids=ids32)
        ctx.sync()
        fixed, _ = ctx.deposit()
        return dict(q=q, v64=v64, v32=v32, q32=q32, ids64=ids64, ids32=ids32, fixed=fixed)
    finally:
        ctx.close()


@pytest.mark.parametrize("host_io_async", [0, 1])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_v32_load_and_read_back_match_float64_calls(name, host_io_async):
    from paper_1908_10793_gb300 import dust as D
    w = WORKLOADS[name]()
    vf = [np.ascontiguousarray(x, dtype=np.float32) for x in w.v]
    vd = [x.astype(np.float64) for x in vf]
    a = _run(D, w, vd, D.dust_load_particles, host_io_async)
    b = _run(D, w, vf, D.dust_load_particles_v32, host_io_async)
    for d in range(3):
        assert np.array_equal(a["q"][d], b["q"][d], equal_nan=True), (name, "q", d)
        assert np.array_equal(a["v64"][d], b["v64"][d], equal_nan=True), (name, "v", d)
        # float32 read-back: the float64 read-back rounded, same order
        assert np.array_equal(b["v32"][d], b["v64"][d].astype(np.float32), equal_nan=True), (name, "v32", d)
        assert np.array_equal(b["q32"][d], b["q"][d], equal_nan=True), (name, "q32", d)
    assert np.array_equal(a["ids64"], b["ids64"])
    assert np.array_equal(b["ids32"], b["ids64"])
    assert np.array_equal(a["fixed"], b["fixed"])


def test_v32_device_arrays():
    """The same calls with CUDA tensors (DUST_MEM_DEVICE)."""
    torch = pytest.importorskip("torch")
    from paper_1908_10793_gb300 import dust as D
    w = I.sbox3d("small")
    n = w.ngrains
    ctx = D.Context(w, precision=D.DUST_MIXED)
    try:
        ctx.set_gas(w.rho, w.vgas)
        qd = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in w.q]
        vd = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in w.v]
        D.dust_load_particles_v32(ctx.handle, *qd, *vd)
        ctx.n = n  # the grain count Context.load would record
        ctx.step(w.dt)
        ctx.sync()
        oq = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3)]
        ov = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        oid = torch.empty(n, dtype=torch.int64, device="cuda")
        D.dust_get_particles_v32(ctx.handle, n, *oq, *ov, ids=oid)
        q, v, ids = ctx.particles()
        for d in range(3):
            assert np.array_equal(oq[d].cpu().numpy(), q[d], equal_nan=True)
            assert np.array_equal(ov[d].cpu().numpy(), v[d].astype(np.float32), equal_nan=True)
        assert np.array_equal(oid.cpu().numpy(), ids)
    finally:
        ctx.close()
