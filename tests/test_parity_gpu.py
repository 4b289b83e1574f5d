"""GPU parity: the CUDA library (through the C interface) against the FP64
oracle on the same seeded inputs, element by element.

Tolerances
* FP64 path: positions and momentum-like variables within 1e-12 of the
  grain's speed (times dt for positions) per step; deposit, every channel
  (the energy channel included), within 1e-12 of the channel's largest value
  plus the fixed-point representation's own error: half a quantum for every
  piece a zone can receive (27 per grain in 3-D, 9 in 2-D, times the grains
  that reach it), doubled because the host zone of a grain or chunk takes
  the rest of its rounded total and so the other pieces' rounding as well.
  The integers themselves are compared with the oracle's fixed-point rule in
  test_fixed_point_gpu.py.
* Mixed path (FP32 push, FP64 positions): momentum-like variables within
  1e-5 relative per step; coordinates within 1e-5 of the step's displacement
  plus one ulp; the deposit is -m (p^{n+1} - p^n - dt a) with p in FP32, so
  each piece carries an absolute error of a few FP32 ulps of m |p| (not of the
  deposit itself): tolerance 16 eps32 m |p|max times the largest number of
  grains that reach one zone, plus quanta.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_10793_gb300 import inputs as I
from parity_util import default_quantum, periodic_diff, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
EPS32 = 2.0 ** -24


def _grains_per_zone_max(w):
    cells = [np.clip(np.searchsorted(w.edges[d], w.q[d], side="right") - 1, 0, len(w.edges[d]) - 2)
             for d in range(3)]
    n = w.n
    lin = cells[0] + n[0] * (cells[1] + n[1] * cells[2])
    return int(np.bincount(lin, minlength=w.ncell).max())


def compare(w, steps, precision, dt=None, feedback=None, extra_v=0.0, predictor=False, **kw):
    dt = w.dt if dt is None else dt
    qo, vo, active, dep_o, pg_o = run_oracle(w, steps, dt, feedback, predictor)
    if predictor:
        kw["gas_predictor"] = 1
    g = run_gpu(w, steps, precision, dt, feedback, **kw)
    check_against_oracle(w, g, (qo, vo, active, dep_o), steps, precision, dt, extra_v)
    return g, (qo, vo, active, dep_o, pg_o)


def check_against_oracle(w, g, oracle_out, steps, precision, dt, extra_v=0.0):
    """Grain states and the last deposit of a GPU run (dict with q, v in id
    order, fixed, quantum, rc) against the oracle's, with the tolerances of
    the module docstring."""
    qo, vo, active, dep_o = oracle_out
    assert g["rc"] in (0, -4), "device status %d" % g["rc"]
    alive = active.astype(bool)
    assert np.array_equal(~np.isnan(g["q"][0]), alive), "removed grains differ"
    if precision == FP64:
        rtol = 1e-12 * max(1, steps)
    else:
        rtol = 1e-5 * max(1, steps)
    # scales: the grain's speed (momentum-like variables can cancel in one
    # component, e.g. v_R on a Keplerian orbit) and the distance it can move
    speed = np.sqrt(sum(vo[d][alive] ** 2 for d in range(3))) + 1e-300
    if w.geom == O.OG_SHEARING_BOX and w.fargo:
        # the y drift also carries the mean shear -q Omega x
        speed = speed + w.qshear * w.omega * np.abs(qo[0][alive])
    for d in range(3):
        dq = np.abs(periodic_diff(w, d, g["q"][d][alive], qo[d][alive]))
        L = w.edges[d][-1] - w.edges[d][0]
        metric = 1.0 if d == 0 or w.geom in (O.OG_CARTESIAN, O.OG_SHEARING_BOX) else \
            1.0 / np.maximum(qo[0][alive], 1e-3) / (np.sin(qo[1][alive]) if (d == 2 and w.geom == O.OG_SPHERICAL) else 1.0)
        disp = speed * metric * abs(dt) * steps
        ulps = (L + np.max(np.abs(w.edges[d]))) * 2.0 ** -52 * 4 * steps
        assert np.all(dq <= rtol * disp + ulps), "coordinate %d: max err %.3e" % (d, dq.max())
        dv = np.abs(g["v"][d][alive] - vo[d][alive])
        assert np.all(dv <= rtol * speed + extra_v), "velocity %d: max rel err %.3e" % (
            d, (dv / speed).max())
    # deposit of the last step
    dep_g = g["fixed"] * g["quantum"]
    big = np.abs(dep_o).max(axis=0)
    # a zone collects at most nz pieces, each rounded by half a quantum
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9) * 2
    if precision == FP64:
        tol = 1e-12 * big + 0.5 * nz * g["quantum"]
    else:
        from parity_util import to_momentum
        p = to_momentum(w, w.q, w.v)
        m = np.max(w.species_mass)
        pmax = max(np.abs(x).max() for x in p)
        tol = 16 * EPS32 * m * pmax * nz * np.array([1, 1, 1, 2.0 * pmax]) + 1e-5 * big + \
            (0.5 * nz + 4) * g["quantum"]
    err = np.abs(dep_g - dep_o).max(axis=0)
    assert np.all(err <= tol), "deposit err %s tol %s" % (err, tol)


WORKLOADS = {
    "box2d": lambda: I.box2d("small"),
    "sbox3d": lambda: I.sbox3d("small"),
    "cyldisk": lambda: I.cyldisk("small"),
    "sphdisk": lambda: I.sphdisk("small"),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_parity_one_step(name, precision):
    compare(WORKLOADS[name](), 1, precision)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_parity_fp64_several_steps_with_feedback(name):
    """Four steps with the deposit applied to the gas.  The gas update uses the
    fixed-point deposit, so each zone's gas velocity differs from the oracle's
    dense sum by at most (pieces per zone) * quantum / 2 / (rho dV) per step;
    the grains see that difference through the drag term."""
    w = WORKLOADS[name]()
    steps = 4
    qo, vo, active, dep_o, pg_o = run_oracle(w, steps, feedback=1)
    g = run_gpu(w, steps, FP64, feedback=1)
    from test_oracle_push import _zone_volumes
    prob = O.Problem(geom=w.geom, edges=w.edges)
    dV = _zone_volumes(prob)
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9)
    dgas = steps * nz * 0.5 * g["quantum"] / (w.rho * dV)
    compare(w, steps, FP64, feedback=1, extra_v=2 * steps * dgas.max())
    ref_v = pg_o
    if w.geom == O.OG_CYLINDRICAL:
        R, _, _ = I._grid3(w.edges)
        ref_v = [pg_o[0], pg_o[1] / R, pg_o[2]]
        dgas = [dgas, dgas / R, dgas]
    elif w.geom == O.OG_SPHERICAL:
        r, th, _ = I._grid3(w.edges)
        ref_v = [pg_o[0], pg_o[1] / r, pg_o[2] / (r * np.sin(th))]
        dgas = [dgas, dgas / r, dgas / (r * np.sin(th))]
    else:
        dgas = [dgas] * 3
    for d in range(3):
        scale = np.abs(ref_v[d]).max() + 1e-300
        assert np.all(np.abs(g["vgas"][d] - ref_v[d]) <= 1e-12 * scale + dgas[d])


@pytest.mark.parametrize("weight", [I.CIC, I.TSC])
@pytest.mark.parametrize("name", ["box2d", "cyldisk", "sphdisk"])
def test_parity_weights(name, weight):
    w = WORKLOADS[name]()
    w.weight = weight
    compare(w, 2, FP64)
    compare(w, 1, MIXED)


@pytest.mark.parametrize("fargo,vgrav", [(0, 1), (1, 1), (0, 0)])
def test_parity_shearing_box_frames(fargo, vgrav):
    w = I.sbox3d("small")
    w.fargo, w.vertical_gravity = fargo, vgrav
    w.v = [x * 30.0 for x in w.v]   # cross zone and x boundaries more often
    compare(w, 3, FP64)
    compare(w, 1, MIXED)


def test_parity_shear_periodic_wrap():
    w = I.sbox3d("small")
    w = I.subsample(w, 3000)
    # push grains out through both radial boundaries during the step
    L = w.edges[0][-1] - w.edges[0][0]
    w.q[0] = np.where(np.arange(w.ngrains) % 2 == 0, w.edges[0][-1] - 1e-4 * L, w.edges[0][0] + 1e-4 * L)
    w.v[0] = np.where(np.arange(w.ngrains) % 2 == 0, 0.05, -0.05)
    compare(w, 2, FP64, dt=w.dt, feedback=0)
    w.fargo = 0
    compare(w, 2, FP64, dt=w.dt, feedback=0)


def test_parity_outflow_removal_cylindrical():
    w = I.cyldisk("small")
    w = I.subsample(w, 5000)
    # grains close to the inner radius falling inward leave through outflow
    w.q[0] = np.where(np.arange(w.ngrains) % 3 == 0, w.edges[0][0] + 1e-5, w.q[0])
    w.v[0] = np.where(np.arange(w.ngrains) % 3 == 0, -0.5, w.v[0])
    g, (qo, vo, active, dep_o, _) = compare(w, 2, FP64, feedback=0)
    assert (active == 0).sum() > 100
    assert g["stats"].n_removed == (active == 0).sum()


def test_slab_kernel_outflow_removal_over_sorts():
    """Mixed precision, slab kernel, a sort before every step: the step before
    each sort predicts its keys, grains removed earlier sit after every zone's
    group and must keep the removed-grain key."""
    from paper_1908_10793_gb300 import dust as D
    w = I.cyldisk("small")
    w = I.subsample(w, 6000)
    w.q[0] = np.where(np.arange(w.ngrains) % 3 == 0, w.edges[0][0] + 1e-5, w.q[0])
    w.v[0] = np.where(np.arange(w.ngrains) % 3 == 0, -0.5, w.v[0])
    for steps in (1, 3):
        g, (qo, vo, active, dep_o, _) = compare(w, steps, MIXED, feedback=0,
                                                kernel=D.DUST_KERNEL_SLAB, sort_interval=1)
        assert (active == 0).sum() > 100
    # a change of step length: the keys predicted for the old length are
    # dropped and the sort computes its own; grain states match the
    # one-thread-per-grain kernel's
    dts = [w.dt, 0.5 * w.dt, 0.5 * w.dt, w.dt]
    a = run_gpu(w, 4, MIXED, dts, 0, kernel=D.DUST_KERNEL_SLAB, sort_interval=1)
    b = run_gpu(w, 4, MIXED, dts, 0, kernel=D.DUST_KERNEL_PER_GRAIN)
    assert np.array_equal(np.isnan(a["q"][0]), np.isnan(b["q"][0]))
    alive = ~np.isnan(b["q"][0])
    for d in range(3):
        scale = np.abs(b["v"][d][alive]).max() + 1.0
        assert np.abs(a["v"][d][alive] - b["v"][d][alive]).max() <= 256 * EPS32 * scale


def test_slab_kernel_dense_zones_split_into_chunks():
    """Zones holding more than 128 grains: the slab kernel quantises each
    zone's run in chunks of 128 grains (by rank in id order).  Parity with the
    oracle, and the integers do not depend on the tile shape."""
    from paper_1908_10793_gb300 import dust as D
    w = I.box2d("small")
    rng = np.random.default_rng(11)
    n = w.ngrains
    # 600 grains in one zone, 300 in another, the rest spread out
    dx = w.edges[0][1] - w.edges[0][0]
    for sel, (cx, cy) in ((slice(0, 600), (3, 5)), (slice(600, 900), (10, 12))):
        k = sel.stop - sel.start
        w.q[0][sel] = w.edges[0][cx] + dx * rng.uniform(0.05, 0.95, k)
        w.q[1][sel] = w.edges[1][cy] + dx * rng.uniform(0.05, 0.95, k)
    assert _grains_per_zone_max(w) >= 600 and n == 1024
    compare(w, 2, MIXED, kernel=D.DUST_KERNEL_SLAB, sort_interval=1)
    first = None
    for tile in ((0, 0, 0), (4, 4, 1), (8, 2, 1)):
        got = run_gpu(w, 2, MIXED, kernel=D.DUST_KERNEL_SLAB, tile=tile, sort_interval=1)
        if first is None:
            first = got
        assert np.array_equal(got["fixed"], first["fixed"]), tile


def test_gas_predictor_dense_zones_and_tile_independent():
    """The gas predictor with zones of 600 and 300 grains (several chunks of
    the slab step): parity with the oracle's predictor-corrector, and results
    that do not depend on the tile shape (the predictor's per-grain rule is
    independent of the grains' order)."""
    from paper_1908_10793_gb300 import dust as D
    from parity_util import zone_volumes
    w = I.box2d("small")
    rng = np.random.default_rng(11)
    dx = w.edges[0][1] - w.edges[0][0]
    for sel, (cx, cy) in ((slice(0, 600), (3, 5)), (slice(600, 900), (10, 12))):
        k = sel.stop - sel.start
        w.q[0][sel] = w.edges[0][cx] + dx * rng.uniform(0.05, 0.95, k)
        w.q[1][sel] = w.edges[1][cy] + dx * rng.uniform(0.05, 0.95, k)
    steps = 2
    nz = _grains_per_zone_max(w) * 9
    quantum = default_quantum(w, MIXED)
    dgas = (nz * 0.5 * quantum / (w.rho * zone_volumes(w))).max()
    compare(w, steps, MIXED, feedback=1, predictor=True, extra_v=4 * steps * dgas,
            kernel=D.DUST_KERNEL_SLAB, sort_interval=1)
    first = None
    for tile in ((0, 0, 0), (4, 4, 1), (8, 2, 1)):
        got = run_gpu(w, steps, MIXED, feedback=1, kernel=D.DUST_KERNEL_SLAB, tile=tile,
                      sort_interval=1, gas_predictor=1)
        if first is None:
            first = got
        assert np.array_equal(got["fixed"], first["fixed"]), tile
        for d in range(3):
            assert np.array_equal(got["v"][d], first["v"][d], equal_nan=True), (tile, d)


@pytest.mark.parametrize("name,fargo", [("box2d", None), ("sbox3d", 0), ("sbox3d", 1)])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_parity_semi_implicit_pusher(name, fargo, precision):
    """The semi-implicit pusher (Sec. 3.2.1) on the GPU against the oracle's,
    Cartesian and shearing box in both frames, with stiff grains mixed in
    (per-grain St down to 1e-3, where the scheme oscillates)."""
    w = WORKLOADS[name]()
    w.pusher = 1
    if fargo is not None:
        w.fargo = fargo
    rng = np.random.default_rng(3)
    w.param = np.where(rng.uniform(size=w.ngrains) < 0.5, 1e-3, 0.3) * (
        1.0 if w.geom == O.OG_SHEARING_BOX else 0.1)
    # For stiff grains the kick's result is a small difference of terms of
    # size dt |a_tot| (drag (|v| + |v_g|)/tau, Coriolis, tidal), so rounding is
    # relative to that, not to the grain's speed: allow 64 ulps of it.
    tau_min = w.param.min() / (w.omega if w.geom == O.OG_SHEARING_BOX else 1.0)
    vmax = max(np.abs(x).max() for x in w.v) + max(np.abs(x).max() for x in w.vgas)
    a_scale = vmax / tau_min
    if w.geom == O.OG_SHEARING_BOX:
        xmax = np.abs(w.edges[0]).max()
        a_scale += 2 * w.qshear * w.omega ** 2 * xmax + 2 * w.omega * vmax
    eps = 2.0 ** -52 if precision == FP64 else 2.0 ** -23
    compare(w, 2 if precision == FP64 else 1, precision, extra_v=64 * eps * w.dt * a_scale)


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_parity_gas_predictor(name, precision):
    """Two steps with the gas half-step drag predictor and the feedback
    corrector against the oracle's.  The predictor's impulse is deposited in
    fixed point: each zone's predicted gas velocity may differ from the
    oracle's dense sum by (pieces per zone) quanta / 2 / (rho dV), which the
    drag passes on to the grains; the corrector adds the same per step."""
    from parity_util import zone_volumes
    w = WORKLOADS[name]()
    steps = 2
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9)
    quantum = default_quantum(w, precision)
    dgas = (nz * 0.5 * quantum / (w.rho * zone_volumes(w))).max()
    compare(w, steps, precision, feedback=1, predictor=True, extra_v=4 * steps * dgas)


def test_parity_epstein_tau_mode():
    w = I.box2d("small")
    w.species_tau_mode = [I.TAU_EPSTEIN]
    w.species_tau = [0.05]
    rng = np.random.default_rng(5)
    w.rho = rng.uniform(0.5, 2.0, w.ncell)
    compare(w, 2, FP64)
    compare(w, 1, MIXED)


def test_parity_negative_dt_and_infinite_tau():
    w = I.sphdisk("small")
    # reverse-time drag amplifies by exp(|dt|/tau): keep the grains non-stiff
    w.param = np.where(np.arange(w.ngrains) % 2 == 0, np.inf, np.maximum(w.param, 0.5))
    compare(w, 2, FP64, dt=-w.dt, feedback=0)


def test_single_grain_and_empty():
    w = I.subsample(I.box2d("small"), 1)
    compare(w, 3, FP64)
    w0 = I.subsample(I.box2d("small"), 0)
    g = run_gpu(w0, 2, FP64)
    assert g["rc"] == 0 and np.all(g["fixed"] == 0)


def test_deposit_bitwise_reproducible_and_sort_independent():
    # per-grain kernel: every grain quantises its own pieces, so the integer
    # grid does not depend on the store order at all
    from paper_1908_10793_gb300 import dust as D
    w = I.sbox3d("small")
    K = D.DUST_KERNEL_PER_GRAIN
    a = run_gpu(w, 3, MIXED, sort_interval=1, kernel=K)
    b = run_gpu(w, 3, MIXED, sort_interval=1, kernel=K)
    c = run_gpu(w, 3, MIXED, sort_interval=2, kernel=K)
    assert np.array_equal(a["fixed"], b["fixed"])
    assert np.array_equal(a["fixed"], c["fixed"])
    for d in range(3):
        assert np.array_equal(a["q"][d], c["q"][d]) and np.array_equal(a["v"][d], c["v"][d])


def test_fixed_point_sum_equals_momentum_change():
    # Cartesian, no forces: sum over zones of the deposit = -m sum(dv) to one
    # quantum per grain and channel (per-grain remainder rule)
    w = I.box2d("full")
    g = run_gpu(w, 1, FP64, feedback=0)
    m = w.species_mass[0]
    for d in range(2):
        total = g["fixed"][:, d].sum() * g["quantum"]
        ref = -m * (g["v"][d] - w.v[d]).sum()
        assert abs(total - ref) <= 0.5 * w.ngrains * g["quantum"] + 1e-14 * m * np.abs(w.v[d]).sum()


def test_invalid_inputs_rejected():
    from paper_1908_10793_gb300 import dust as D
    w = I.subsample(I.box2d("small"), 10)
    ctx = D.Context(w, precision=FP64)
    try:
        with pytest.raises(D.DustError):
            ctx.step(0.01)                      # no data yet
        bad = [x.copy() for x in w.q]
        bad[0][3] = np.nan
        with pytest.raises(D.DustError):
            ctx.load(bad, w.v)
        bad[0][3] = 2.0                         # outside the grid
        with pytest.raises(D.DustError):
            ctx.load(bad, w.v)
        with pytest.raises(D.DustError):
            ctx.set_gas(-w.rho, w.vgas)
    finally:
        ctx.close()


def test_full_size_shearing_box_sampled_against_oracle():
    """128^3 shearing box, 16.8M grains, mixed precision, one step in the
    configuration the benchmark times: sampled grains against the oracle
    computed one by one, and the deposit of a slab of zones against the oracle
    run on every grain that can reach it."""
    from paper_1908_10793_gb300 import dust as D
    w = I.sbox3d("full")
    g = run_gpu(w, 1, MIXED, feedback=1)
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(w.ngrains, 4000, replace=False))
    s = I.subsample(w, w.ngrains)  # copy
    s.q = [x[idx] for x in w.q]
    s.v = [x[idx] for x in w.v]
    qo, vo, active, _, _ = run_oracle(s, 1, feedback=0)
    for d in range(3):
        dq = np.abs(periodic_diff(w, d, g["q"][d][idx], qo[d]))
        assert dq.max() <= 1e-5 * (np.abs(w.v[d]).max() + 0.15) * w.dt + 1e-16
        dv = np.abs(g["v"][d][idx] - vo[d])
        assert dv.max() <= 1e-5 * np.abs(vo[d]).max()
    # slab of zones k in [k0, k0+3]: every grain starting in zones k0-2..k0+5
    n = w.n[2]
    k0 = 40
    zc = np.clip(np.searchsorted(w.edges[2], w.q[2], side="right") - 1, 0, n - 1)
    sel = np.nonzero((zc >= k0 - 2) & (zc <= k0 + 5))[0]
    s.q = [x[sel] for x in w.q]
    s.v = [x[sel] for x in w.v]
    _, _, _, dep_o, _ = run_oracle(s, 1, feedback=0)
    nx, ny = w.n[0], w.n[1]
    cells = np.arange(k0 * nx * ny, (k0 + 4) * nx * ny)
    dep_g = g["fixed"][cells] * g["quantum"]
    p = w.v
    m = w.species_mass[0]
    pmax = max(np.abs(x).max() for x in p) + 0.2
    tol = 16 * EPS32 * m * pmax * 27 * 16 + 1e-5 * np.abs(dep_o[cells]).max(axis=0) + 64 * g["quantum"]
    assert np.all(np.abs(dep_g - dep_o[cells]).max(axis=0) <= tol)
    del D


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_tiled_kernel_against_per_grain_kernel(name, precision, kernel):
    """The tiled kernel pushes grains with the same arithmetic as the
    one-thread-per-grain kernel (grain states identical in mixed precision,
    equal to rounding in FP64) but quantises the deposit once per run of grains
    sharing a sort key and host zone: the integer deposit is reproducible bit
    for bit and does not depend on the tile shape, and it matches the
    per-grain kernel's deposit within the fixed-point and summation rounding."""
    from paper_1908_10793_gb300 import dust as D
    w = WORKLOADS[name]()
    ref = run_gpu(w, 3, precision, kernel=D.DUST_KERNEL_PER_GRAIN)
    first = None
    for tile in ((0, 0, 0), (4, 4, 2), (8, 2, 4), (0, 0, 0)):
        got = run_gpu(w, 3, precision, kernel=kernel, tile=tile, sort_interval=1)
        if first is None:
            first = got
        else:
            assert np.array_equal(got["fixed"], first["fixed"]), tile
        for d in range(3):
            a, b = got["q"][d], ref["q"][d]
            assert np.array_equal(np.isnan(a), np.isnan(b))
            # same arithmetic; the compiler may contract multiply-adds
            # differently in the two kernels
            eps = 2.0 ** -23 if precision == MIXED else 2.0 ** -52
            # scale: the largest velocity-like term entering the kick
            vs = max(np.nanmax(np.abs(ref["v"][d])), np.abs(w.vgas[d]).max(),
                     max(np.abs(x).max() for x in w.v), 0.2 if w.geom == O.OG_SHEARING_BOX else 0.0)
            assert np.nanmax(np.abs(got["v"][d] - ref["v"][d])) <= 64 * eps * vs, (tile, d)
            assert np.nanmax(np.abs(a - b)) <= 64 * eps * vs * 3 * w.dt + \
                8 * 2.0 ** -52 * (1 + np.nanmax(np.abs(b))), (tile, d)
    big = np.abs(ref["fixed"]).max(axis=0).astype(np.float64)
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9) * 2
    if precision == MIXED:
        # pieces carry FP32 rounding of m |p| (see the module docstring)
        from parity_util import to_momentum
        pmax = max(np.abs(x).max() for x in to_momentum(w, w.q, w.v)) + 1e-3
        m = np.max(w.species_mass) / ref["quantum"]
        tol = 32 * EPS32 * m * pmax * nz * np.array([1, 1, 1, 2.0 * pmax]) + 1e-5 * big + nz
    else:
        tol = 1e-12 * big + nz
    assert np.all(np.abs(first["fixed"] - ref["fixed"]).max(axis=0) <= tol)


def test_tiled_deposit_independent_of_sort_scatter_order():
    """The zone sort scatters with atomics (arbitrary order inside a zone);
    runs are summed in grain-id order, so repeated runs give the same integers."""
    from paper_1908_10793_gb300 import dust as D
    w = I.cyldisk("small")
    a = run_gpu(w, 4, MIXED, kernel=D.DUST_KERNEL_TILED, sort_interval=2)
    for _ in range(3):
        b = run_gpu(w, 4, MIXED, kernel=D.DUST_KERNEL_TILED, sort_interval=2)
        assert np.array_equal(a["fixed"], b["fixed"])


def _near_axis_cyl():
    """Cylindrical grid whose inner edge is 0.04 zones from the axis (the
    ghost centre of the volume weights lies across it), outflow in R."""
    r = np.random.default_rng(11)
    edges = [0.002 + 0.05 * np.arange(21), np.linspace(0.0, 2 * np.pi, 17), np.linspace(-0.1, 0.1, 5)]
    ncell = 20 * 16 * 4
    ng = 3000
    return I.Workload(
        name="near_axis", geom=I.CYLINDRICAL, edges=edges, bc=[I.OUTFLOW, I.PERIODIC, I.PERIODIC],
        weight=I.VOLUME, species_mass=[1e-3], species_tau_mode=[I.TAU_CONST], species_tau=[0.1],
        rho=r.uniform(0.5, 2.0, ncell),
        vgas=[0.1 * r.standard_normal(ncell) for _ in range(3)],
        q=[r.uniform(0.002, 1.002, ng), r.uniform(0, 2 * np.pi, ng), r.uniform(-0.1, 0.1, ng)],
        v=[0.1 * r.standard_normal(ng) for _ in range(3)], dt=1e-3, steps=2, feedback=0)


def _near_pole_sph():
    """Spherical grid whose polar-angle range ends 0.05 zones from each pole
    (ghost centres across the poles), outflow in r and theta."""
    r = np.random.default_rng(12)
    dth = (np.pi - 0.02) / 16
    edges = [np.linspace(0.5, 1.5, 9), 0.01 + dth * np.arange(17), np.linspace(0.0, 2 * np.pi, 9)]
    ncell = 8 * 16 * 8
    ng = 3000
    return I.Workload(
        name="near_pole", geom=I.SPHERICAL, edges=edges, bc=[I.OUTFLOW, I.OUTFLOW, I.PERIODIC],
        weight=I.VOLUME, species_mass=[1e-3], species_tau_mode=[I.TAU_CONST], species_tau=[0.1],
        rho=r.uniform(0.5, 2.0, ncell),
        vgas=[0.1 * r.standard_normal(ncell) for _ in range(3)],
        q=[r.uniform(0.5, 1.5, ng), r.uniform(edges[1][0], edges[1][-1], ng),
           r.uniform(0, 2 * np.pi, ng)],
        v=[0.1 * r.standard_normal(ng) for _ in range(3)], dt=1e-3, steps=2, feedback=0)


VOLUME_WORKLOADS = {
    "cyldisk": lambda: WORKLOADS["cyldisk"](),
    "sphdisk": lambda: WORKLOADS["sphdisk"](),
    "near_axis": _near_axis_cyl,
    "near_pole": _near_pole_sph,
}


@pytest.mark.parametrize("name", list(VOLUME_WORKLOADS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_parity_volume_weighting(name, precision):
    """Traditional volume weighting (Eq. CIC_vol) against the oracle's: the
    default kernel (two steps; the slab kernel with single-precision volume
    weights in mixed precision, the tiled kernel in FP64) and the
    one-thread-per-grain kernel (one step)."""
    from paper_1908_10793_gb300 import dust as D
    w = VOLUME_WORKLOADS[name]()
    w.weight = I.VOLUME
    compare(w, 2, precision)
    compare(w, 1, precision, kernel=D.DUST_KERNEL_PER_GRAIN)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_parity_volume_weighting_with_gas_predictor(precision):
    from parity_util import zone_volumes
    w = WORKLOADS["cyldisk"]()
    w.weight = I.VOLUME
    steps = 2
    nz = _grains_per_zone_max(w) * 27
    quantum = default_quantum(w, precision)
    dgas = (nz * 0.5 * quantum / (w.rho * zone_volumes(w))).max()
    compare(w, steps, precision, feedback=1, predictor=True, extra_v=4 * steps * dgas)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_volume_weighting_equals_cic_in_cartesian_geometries(precision):
    """Cartesian and shearing-box directions have the coordinate itself as
    volume coordinate: the library must give the CIC results bit for bit."""
    for name in ("box2d", "sbox3d"):
        w = WORKLOADS[name]()
        w.weight = I.CIC
        a = run_gpu(w, 2, precision)
        w.weight = I.VOLUME
        b = run_gpu(w, 2, precision)
        for key in ("q", "v"):
            for d in range(3):
                assert np.array_equal(a[key][d], b[key][d], equal_nan=True), (name, key, d)
        assert np.array_equal(a["fixed"], b["fixed"])


MASS_CASES = [("box2d", I.TSC), ("box2d", I.CIC), ("sbox3d", I.TSC), ("cyldisk", I.TSC),
              ("cyldisk", I.VOLUME), ("sphdisk", I.TSC), ("sphdisk", I.CIC), ("sphdisk", I.VOLUME)]


@pytest.mark.parametrize("name,weight", MASS_CASES)
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_mass_deposit_matches_oracle(name, weight, precision):
    """dust_get_mass_deposit after two steps against the oracle's mass
    deposit of the GPU's own grain positions: each zone within half a
    quantum per piece it can receive (plus the weights' rounding), and the
    zone sum equal to the grain sum of rint(m / quantum) exactly."""
    from paper_1908_10793_gb300 import dust as D
    w = WORKLOADS[name]()
    w.weight = weight
    ctx = D.Context(w, precision=precision, feedback=0)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v, w.species, w.param)
        for _ in range(2):
            ctx.step(w.dt)
        ctx.sync(check=False)
        fixed, quantum = ctx.mass_deposit()
        q, _, ids = ctx.particles()
    finally:
        ctx.close()
    alive = ~np.isnan(q[0])
    sp = w.species[ids] if w.species is not None else None
    prob = O.Problem(geom=w.geom, edges=w.edges, bc=w.bc, weight=weight,
                     species_mass=w.species_mass, species_tau_mode=w.species_tau_mode,
                     species_tau=w.species_tau)
    dense = O.deposit_mass(prob, q, alive.astype(np.uint8), sp)
    m = np.asarray(w.species_mass)[sp if sp is not None else np.zeros(len(ids), int)]
    assert fixed.sum() == int(np.rint(m[alive] / quantum).sum())
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9)
    tol = (0.5 * nz + 1) * quantum + 1e-12 * dense.max()
    assert np.abs(fixed * quantum - dense).max() <= tol


def _take(w, idx):
    import copy
    s = copy.copy(w)
    s.q = [x[idx] for x in w.q]
    s.v = [x[idx] for x in w.v]
    s.species = None if w.species is None else w.species[idx]
    s.param = None if w.param is None else w.param[idx]
    return s


@pytest.mark.parametrize("name", ["cyldisk", "sphdisk"])
def test_full_size_disks_sampled_against_oracle(name):
    """The cylindrical (384 x 1024 x 64, 50M grains, feedback on) and
    spherical (256 x 128 x 512, 33M grains) disks at full size, mixed
    precision, one step in the configuration the benchmark times: 4000
    sampled grains against the oracle run on them alone (a grain's push does
    not depend on the others within a step), and the deposit of a slab of
    four zone layers in the last direction against the oracle run on every
    grain that can reach it."""
    from parity_util import to_momentum
    w = {"cyldisk": I.cyldisk, "sphdisk": I.sphdisk}[name]("full")
    feedback = 1 if name == "cyldisk" else 0
    g = run_gpu(w, 1, MIXED, feedback=feedback)
    assert g["rc"] in (0, -4)
    rng = np.random.default_rng(12)
    idx = np.sort(rng.choice(w.ngrains, 4000, replace=False))
    qo, vo, active, _, _ = run_oracle(_take(w, idx), 1, feedback=0)
    alive = active.astype(bool)
    assert np.array_equal(~np.isnan(g["q"][0][idx]), alive)
    speed = np.sqrt(sum(vo[d][alive] ** 2 for d in range(3)))
    for d in range(3):
        metric = 1.0
        if d > 0:
            metric = 1.0 / qo[0][alive]
            if d == 2 and w.geom == O.OG_SPHERICAL:
                metric = metric / np.sin(qo[1][alive])
        L = w.edges[d][-1] - w.edges[d][0]
        ulps = (L + np.max(np.abs(w.edges[d]))) * 2.0 ** -52 * 4
        dq = np.abs(periodic_diff(w, d, g["q"][d][idx][alive], qo[d][alive]))
        assert np.all(dq <= 1e-5 * speed * metric * w.dt + ulps), d
        dv = np.abs(g["v"][d][idx][alive] - vo[d][alive])
        assert np.all(dv <= 1e-5 * speed), d
    # deposit of zone layers k0 .. k0+3 of the last direction: every grain
    # starting within two layers of them
    n = w.n
    k0 = n[2] // 2
    kz = np.clip(np.searchsorted(w.edges[2], w.q[2], side="right") - 1, 0, n[2] - 1)
    sel = np.nonzero((kz >= k0 - 2) & (kz <= k0 + 5))[0]
    _, _, _, dep_o, _ = run_oracle(_take(w, sel), 1, feedback=0)
    cells = np.arange(k0 * n[0] * n[1], (k0 + 4) * n[0] * n[1])
    dep_g = g["fixed"][cells] * g["quantum"]
    big = np.abs(dep_o[cells]).max(axis=0)
    nz = _grains_per_zone_max(_take(w, sel)) * 27 * 2
    p = to_momentum(w, w.q, w.v)
    m = np.max(w.species_mass)
    pmax = max(np.abs(x).max() for x in p)
    tol = 16 * EPS32 * m * pmax * nz * np.array([1, 1, 1, 2.0 * pmax]) + 1e-5 * big + \
        (0.5 * nz + 4) * g["quantum"]
    err = np.abs(dep_g - dep_o[cells]).max(axis=0)
    assert np.all(err <= tol), (err, tol)


def test_full_size_batch_against_oracle():
    """The 64 streaming-instability boxes at full size (36M grains) advanced
    by one graph replay of two steps (the batch launch configuration the
    benchmark times, mixed precision, feedback on); instances 0-4 (32^2 to
    512^2 zones), 20 and 63 compared grain by grain, and their last deposit,
    with the oracle run on the whole instance."""
    from paper_1908_10793_gb300 import dust as D
    ws = I.si2d_batch("full")
    ctxs = []
    try:
        for w in ws:
            c = D.Context(w, precision=MIXED, sort_interval=1)
            c.set_gas(w.rho, w.vgas)
            c.load(w.q, w.v, w.species, w.param)
            ctxs.append(c)
        b = D.dust_batch_create([c.handle for c in ctxs])
        try:
            D.dust_batch_step(b, [w.dt for w in ws], 2)
        finally:
            D.dust_batch_destroy(b)
        for k in (0, 1, 2, 3, 4, 20, 63):
            w, c = ws[k], ctxs[k]
            q, v, ids = c.particles()
            o = np.argsort(ids)
            fixed, quantum = c.deposit()
            rc, _ = c.sync(check=False)
            g = {"q": [x[o] for x in q], "v": [x[o] for x in v], "fixed": fixed,
                 "quantum": quantum, "rc": rc}
            qo, vo, active, dep_o, _ = run_oracle(w, 2, feedback=1)
            # the gas of step 2 carries step 1's fixed-point feedback
            from test_oracle_push import _zone_volumes
            dV = _zone_volumes(O.Problem(geom=w.geom, edges=w.edges))
            nz = _grains_per_zone_max(w) * 9
            dgas = (nz * 0.5 * quantum / (w.rho * dV)).max()
            check_against_oracle(w, g, (qo, vo, active, dep_o), 2, MIXED, w.dt, extra_v=4 * dgas)
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n", [13, 21])
def test_parity_ragged_tiles(n, precision):
    """Shearing box of n^3 zones, n not a multiple of the 8^3 tile: partial
    tiles on every axis (the slab kernel's gas box then reaches past the grid
    at the high end as well as the low one), two steps with feedback."""
    w = I.sbox3d(str(n))
    compare(w, 2, precision, feedback=1, extra_v=_feedback_extra_v(w, 2, precision))


def _feedback_extra_v(w, steps, precision):
    from test_oracle_push import _zone_volumes
    dV = _zone_volumes(O.Problem(geom=w.geom, edges=w.edges))
    nz = _grains_per_zone_max(w) * (27 if w.n[2] > 1 else 9)
    quantum = default_quantum(w, precision)
    return 2 * steps * (steps * nz * 0.5 * quantum / (w.rho * dV)).max()
