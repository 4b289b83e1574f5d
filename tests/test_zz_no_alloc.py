"""dust_step_noalloc: one FP64 step of the one-thread-per-grain kernel on
caller-owned device arrays, with its scratch in a fixed device array of the
library instead of allocated memory.

Two consecutive calls are checked against the context interface
(dust_create / dust_step with DUST_KERNEL_PER_GRAIN, FP64) and against the
FP64 oracle on the same seeded inputs, with the FP64 parity tolerances:
coordinates and momentum-like variables within 1e-12 of the grain's speed
(times dt for coordinates) per step plus a few ulps of the domain; the
deposit within 1e-12 of its largest value plus half a quantum per piece a
zone can receive against the context, and integer for integer against the
oracle's fixed-point rule (a quantum of 2^-30 of the mass, so that the two
sides' different rounding of the same double-precision values moves a piece
across a half-integer only rarely; those flips are counted and bounded).
The file is named to be collected last, so it runs both after the other
tests and alone.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _noalloc_source():
    src = open(os.path.join(ROOT, "paper_1908_10793_gb300", "csrc", "dust_api.cu")).read()
    start = src.index('extern "C" int dust_step_noalloc(')
    depth, i = 0, src.index("{", start)
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[start:j + 1]
    raise AssertionError("unterminated function")


def test_noalloc_entry_allocates_nothing_in_source():
    body = _noalloc_source()
    for banned in ("cudaMalloc", "cudaFree", "cudaHostAlloc", "new ", "std::vector",
                   "malloc(", "dalloc("):
        assert banned not in body, banned
    assert "cudaGetSymbolAddress" in body
    # the host image is page-locked in place, so its copy does not block
    assert "cudaHostRegister" in body


def test_noalloc_rejects_oversize_grid_without_gpu():
    # the size check comes before any CUDA call
    from paper_1908_10793_gb300 import dust as D
    lib = D.load_library()
    w = I.box2d("small")
    geo, grid, sp, _, keep = D.make_descriptors(w, precision=D.DUST_FP64)
    big = np.linspace(0.0, 1.0, 4097)
    grid.n[0] = 4096
    grid.edges[0] = big.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    arr = (D.dust_species * len(sp))(*sp)
    rc = lib.dust_step_noalloc(ctypes.byref(geo), ctypes.byref(grid), arr, len(sp), 0, 0.0,
                               0.0, 1e-3, 0, *([None] * 11), 0, None)
    assert rc == D.DUST_EINVAL
    msg = lib.dust_last_error(None).decode()
    assert "4096 zones" in msg and "2048" in msg, msg


def _gas_momentum_like(w):
    """[ncell, 4]: rho and the momentum-like gas velocity with zone-centre
    radius factors (the context's stored gas)."""
    zc = [0.5 * (e[1:] + e[:-1]) for e in w.edges]
    n = w.n
    c0 = np.tile(zc[0], n[1] * n[2])
    c1 = np.tile(np.repeat(zc[1], n[0]), n[2])
    out = np.empty((w.ncell, 4))
    out[:, 0] = w.rho
    out[:, 1] = w.vgas[0]
    out[:, 2] = w.vgas[1]
    out[:, 3] = w.vgas[2]
    if w.geom == I.CYLINDRICAL:
        out[:, 2] = c0 * w.vgas[1]
    elif w.geom == I.SPHERICAL:
        out[:, 2] = c0 * w.vgas[1]
        out[:, 3] = c0 * np.sin(c1) * w.vgas[2]
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["sbox3d", "cyldisk", "sphdisk"])
def test_noalloc_two_calls_match_context_step_and_oracle(name):
    import torch

    import oracle as O
    from paper_1908_10793_gb300 import dust as D
    from parity_util import oracle_problem, run_gpu, to_momentum, to_physical
    w = {"sbox3d": I.sbox3d, "cyldisk": I.cyldisk, "sphdisk": I.sphdisk}[name]("small")
    dt = w.dt
    quantum = np.ldexp(max(abs(m) for m in w.species_mass), -30)
    geo, grid, sp, opt, keep = D.make_descriptors(w, precision=D.DUST_FP64, feedback=0)
    dev = torch.device("cuda", 0)
    q = [torch.tensor(x, dtype=torch.float64, device=dev) for x in w.q]
    p = [torch.tensor(x, dtype=torch.float64, device=dev) for x in to_momentum(w, w.q, w.v)]
    spi = torch.tensor(w.species, dtype=torch.uint8, device=dev) if w.species is not None else None
    par = torch.tensor(w.param, dtype=torch.float64, device=dev) if w.param is not None else None
    gas = torch.tensor(_gas_momentum_like(w), dtype=torch.float64, device=dev)
    dep = torch.empty((w.ncell, 4), dtype=torch.int64, device=dev)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the oracle, stepped beside the calls on the same inputs
    prob = oracle_problem(w, feedback=0)
    qo = [x.copy() for x in w.q]
    po = to_momentum(w, qo, w.v)
    pgo = O.gas_momentum(prob, w.vgas)
    act = np.ones(w.ngrains, np.uint8)
    dead_before = 0
    for call in (1, 2):
        D.dust_step_noalloc(geo, grid, sp, w.weight, quantum, (call - 1) * dt, dt, q, p, gas, dep,
                            species_idx=spi, param=par, status_out=status, device=0,
                            stream=stream.cuda_stream)
        torch.cuda.synchronize()
        _, fx_o, _ = O.step_fixed(prob, qo, po, act, (call - 1) * dt, dt, w.rho.copy(), pgo,
                                  quantum, w.species, w.param)
        ref = run_gpu(w, call, D.DUST_FP64, dt, 0, kernel=D.DUST_KERNEL_PER_GRAIN,
                      quantum=quantum)
        assert ref["rc"] in (0, D.DUST_ECFL)
        qn = [x.cpu().numpy() for x in q]
        pn = [x.cpu().numpy() for x in p]
        vn = to_physical(w, qn, pn)
        alive = ~np.isnan(ref["q"][0])
        assert np.array_equal(~np.isnan(qn[0]), alive), call
        assert np.array_equal(act.astype(bool), alive), call
        speed = np.sqrt(sum(ref["v"][d][alive] ** 2 for d in range(3))) + 1e-300
        if w.geom == I.SHEARING_BOX and w.fargo:
            speed = speed + w.qshear * w.omega * np.abs(ref["q"][0][alive])
        for d in range(3):
            L = w.edges[d][-1] - w.edges[d][0]
            ulps = (L + np.max(np.abs(w.edges[d]))) * 2.0 ** -52 * 4 * call
            metric = 1.0
            if d > 0 and w.geom in (I.CYLINDRICAL, I.SPHERICAL):
                metric = 1.0 / ref["q"][0][alive]
                if d == 2 and w.geom == I.SPHERICAL:
                    metric = metric / np.sin(ref["q"][1][alive])
            for other_q, other_v in ((ref["q"][d][alive], ref["v"][d][alive]),
                                     (qo[d][alive], to_physical(w, qo, po)[d][alive])):
                dq = np.abs(qn[d][alive] - other_q)
                if w.bc[d] == I.PERIODIC:
                    dq = np.minimum(dq, L - dq)
                assert np.all(dq <= 1e-12 * call * speed * metric * dt + ulps), (call, d)
                dv = np.abs(vn[d][alive] - other_v)
                assert np.all(dv <= 1e-12 * call * speed), (call, d)
        # deposit of this call against the context's deposit of its last step
        got = dep.cpu().numpy()
        assert ref["quantum"] == quantum
        big = np.abs(ref["fixed"]).max(axis=0).astype(np.float64)
        nz = 27 * 2 * _grains_per_zone_max(w)
        tol = 1e-12 * big + 0.5 * nz
        assert np.all(np.abs(got - ref["fixed"]).max(axis=0) <= tol), call
        # and integer for integer against the oracle's fixed-point rule
        diff = got - fx_o
        nflip = int(np.abs(diff).sum())
        assert np.abs(diff).max(initial=0) <= 2, call
        assert nflip <= max(8, 1e-5 * int((fx_o != 0).sum())), (call, nflip)
        # status words of this call: removed grains, no NaN or overflow flag
        st = status.cpu().numpy().view(np.uint32)
        dead = int((~alive).sum())
        assert int(st[2]) + (int(st[3]) << 32) == dead - dead_before, call
        dead_before = dead
        assert int(st[0]) & (D.DUST_FLAG_NAN | D.DUST_FLAG_OVERFLOW | D.DUST_FLAG_SPECIES) == 0


@pytest.mark.gpu
def test_noalloc_flags_a_species_index_beyond_the_table():
    import torch
    from paper_1908_10793_gb300 import dust as D
    from parity_util import to_momentum
    w = I.cyldisk("small")
    geo, grid, sp, opt, keep = D.make_descriptors(w, precision=D.DUST_FP64, feedback=0)
    dev = torch.device("cuda", 0)
    q = [torch.tensor(x, dtype=torch.float64, device=dev) for x in w.q]
    p0 = to_momentum(w, w.q, w.v)
    p = [torch.tensor(x, dtype=torch.float64, device=dev) for x in p0]
    bad = np.array(w.species, dtype=np.uint8)
    bad[[3, 17]] = [len(w.species_mass), 255]
    spi = torch.tensor(bad, dtype=torch.uint8, device=dev)
    gas = torch.tensor(_gas_momentum_like(w), dtype=torch.float64, device=dev)
    dep = torch.empty((w.ncell, 4), dtype=torch.int64, device=dev)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    D.dust_step_noalloc(geo, grid, sp, w.weight, 0.0, 0.0, w.dt, q, p, gas, dep,
                        species_idx=spi, status_out=status, device=0,
                        stream=torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    st = status.cpu().numpy().view(np.uint32)
    assert int(st[0]) & D.DUST_FLAG_SPECIES
    qn = [x.cpu().numpy() for x in q]
    pn = [x.cpu().numpy() for x in p]
    for g in (3, 17):
        for d in range(3):
            assert qn[d][g] == w.q[d][g] and pn[d][g] == p0[d][g]
    # the other grains moved
    assert np.any(qn[0] != w.q[0])


def _grains_per_zone_max(w):
    cells = [np.clip(np.searchsorted(w.edges[d], w.q[d], side="right") - 1, 0, len(w.edges[d]) - 2)
             for d in range(3)]
    lin = cells[0] + w.n[0] * (cells[1] + w.n[1] * cells[2])
    return int(np.bincount(lin, minlength=w.ncell).max())
