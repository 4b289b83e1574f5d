"""Python binding of the dust C interface (include/dust.h).

Argument marshalling only: every step of the method runs in libdust.so.
Functions carry the C names.  Arrays may be numpy arrays (host memory) or
torch tensors; CUDA tensors are passed as device pointers (DUST_MEM_DEVICE).
There is no fallback: if the compiled library is missing, importing the
binding's loader raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdust.so")

DUST_OK = 0
DUST_EINVAL, DUST_ENOMEM, DUST_ECUDA, DUST_ECFL, DUST_EOVERFLOW, DUST_ENAN = -1, -2, -3, -4, -5, -6
DUST_ETIMEOUT, DUST_ESTATE = -7, -8
DUST_CARTESIAN, DUST_SHEARING_BOX, DUST_CYLINDRICAL, DUST_SPHERICAL = 0, 1, 2, 3
DUST_BC_PERIODIC, DUST_BC_OUTFLOW = 0, 1
DUST_WEIGHT_CIC, DUST_WEIGHT_TSC, DUST_WEIGHT_VOLUME = 0, 1, 2
DUST_TAU_CONST, DUST_TAU_STOKES, DUST_TAU_EPSTEIN = 0, 1, 2
DUST_FP64, DUST_MIXED = 0, 1
DUST_PUSHER_EM, DUST_PUSHER_SEMI_IMPLICIT = 0, 1
DUST_MEM_HOST, DUST_MEM_DEVICE = 0, 1
DUST_KERNEL_AUTO, DUST_KERNEL_PER_GRAIN, DUST_KERNEL_TILED, DUST_KERNEL_SLAB = 0, 1, 2, 3
DUST_FLAG_NAN, DUST_FLAG_OVERFLOW, DUST_FLAG_CFL, DUST_FLAG_WRAP, DUST_FLAG_TIMEOUT = 1, 2, 4, 8, 16
DUST_FLAG_SPECIES = 32


class DustError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dust error %d: %s" % (code, msg))
        self.code = code


class dust_geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("fargo", ctypes.c_int), ("omega", ctypes.c_double),
                ("q", ctypes.c_double), ("gm", ctypes.c_double),
                ("vertical_gravity", ctypes.c_int)]


class dust_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("edges", ctypes.POINTER(ctypes.c_double) * 3),
                ("bc", ctypes.c_int * 3)]


class dust_species(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("tau_mode", ctypes.c_int),
                ("tau_value", ctypes.c_double)]


class dust_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weight", ctypes.c_int),
                ("feedback_apply", ctypes.c_int), ("quantum", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("sort_interval", ctypes.c_int),
                ("kernel", ctypes.c_int), ("device", ctypes.c_int), ("timing", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("pusher", ctypes.c_int),
                ("gas_predictor", ctypes.c_int), ("host_io_async", ctypes.c_int),
                ("test_wait_timeout", ctypes.c_int), ("batch_mode", ctypes.c_int)]


class dust_kernel_times(ctypes.Structure):
    _fields_ = [("step_ms", ctypes.c_double), ("sort_ms", ctypes.c_double),
                ("other_ms", ctypes.c_double), ("step_launches", ctypes.c_int64),
                ("sort_launches", ctypes.c_int64), ("other_launches", ctypes.c_int64),
                ("steps", ctypes.c_int64)]


class dust_stats(ctypes.Structure):
    _fields_ = [("n_stored", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_removed", ctypes.c_int64), ("max_cells_moved", ctypes.c_double),
                ("flags", ctypes.c_int), ("steps", ctypes.c_int64), ("time", ctypes.c_double),
                ("dt_dust", ctypes.c_double)]


_lib = None


def load_library():
    """Load libdust.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdust.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sigs = {
        "dust_create": (I, [ctypes.POINTER(P), ctypes.POINTER(dust_geometry),
                            ctypes.POINTER(dust_grid), ctypes.POINTER(dust_species), I,
                            ctypes.POINTER(dust_options)]),
        "dust_set_gas": (I, [P, P, P, P, P, I]),
        "dust_get_gas": (I, [P, P, P, P, P, I]),
        "dust_load_particles": (I, [P, I64, P, P, P, P, P, P, P, P, I]),
        "dust_load_particles_v32": (I, [P, I64, P, P, P, P, P, P, P, P, I]),
        "dust_step": (I, [P, D]),
        "dust_sync": (I, [P, ctypes.POINTER(dust_stats)]),
        "dust_get_deposit": (I, [P, P, P, ctypes.POINTER(D), I]),
        "dust_get_mass_deposit": (I, [P, P, P, ctypes.POINTER(D), I]),
        "dust_get_particles": (I, [P, I64, P, P, P, P, P, P, P, ctypes.POINTER(I64), I]),
        "dust_get_particles_v32": (I, [P, I64, P, P, P, P, P, P, P, ctypes.POINTER(I64), I]),
        "dust_get_kernel_times": (I, [P, ctypes.POINTER(dust_kernel_times), I]),
        "dust_step_noalloc": (I, [ctypes.POINTER(dust_geometry), ctypes.POINTER(dust_grid),
                                  ctypes.POINTER(dust_species), I, I, D, D, D, I64,
                                  P, P, P, P, P, P, P, P, P, P, P, I, P]),
        "dust_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I,
                                  ctypes.POINTER(dust_options)]),
        "dust_batch_step": (I, [P, ctypes.POINTER(D), I]),
        "dust_batch_last_error": (ctypes.c_char_p, [P]),
        "dust_batch_destroy": (None, [P]),
        "dust_last_error": (ctypes.c_char_p, [P]),
        "dust_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, mem) of a numpy array or torch tensor; None -> (None, None)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, DUST_MEM_HOST
    # torch tensor
    assert a.is_contiguous()
    return a.data_ptr(), (DUST_MEM_DEVICE if a.is_cuda else DUST_MEM_HOST)


def _mem_of(*arrays):
    mems = {m for _, m in (_ptr(a) for a in arrays if a is not None)}
    if len(mems) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return mems.pop() if mems else DUST_MEM_HOST


def _check(ctx, rc):
    if rc != DUST_OK:
        msg = load_library().dust_last_error(ctx)
        raise DustError(rc, msg.decode() if msg else "")
    return rc


# ------------------------------------------------------------- C names ----
def dust_create(geometry, grid, species, options):
    """geometry: dust_geometry; grid: dust_grid; species: list of
    dust_species; options: dust_options.  Returns an opaque context handle."""
    lib = load_library()
    out = ctypes.c_void_p()
    arr = (dust_species * len(species))(*species)
    rc = lib.dust_create(ctypes.byref(out), ctypes.byref(geometry), ctypes.byref(grid), arr,
                         len(species), ctypes.byref(options))
    if rc != DUST_OK:
        raise DustError(rc, lib.dust_last_error(None).decode())
    return out.value


def dust_set_gas(ctx, rho, v0, v1, v2):
    mem = _mem_of(rho, v0, v1, v2)
    return _check(ctx, load_library().dust_set_gas(ctx, _ptr(rho)[0], _ptr(v0)[0], _ptr(v1)[0],
                                                   _ptr(v2)[0], mem))


def dust_get_gas(ctx, rho, v0, v1, v2):
    mem = _mem_of(rho, v0, v1, v2)
    return _check(ctx, load_library().dust_get_gas(ctx, _ptr(rho)[0], _ptr(v0)[0], _ptr(v1)[0],
                                                   _ptr(v2)[0], mem))


def dust_load_particles(ctx, q0, q1, q2, v0, v1, v2, species=None, param=None):
    mem = _mem_of(q0, q1, q2, v0, v1, v2, species, param)
    n = len(q0)
    return _check(ctx, load_library().dust_load_particles(
        ctx, n, _ptr(q0)[0], _ptr(q1)[0], _ptr(q2)[0], _ptr(v0)[0], _ptr(v1)[0], _ptr(v2)[0],
        _ptr(species)[0], _ptr(param)[0], mem))


def dust_load_particles_v32(ctx, q0, q1, q2, v0, v1, v2, species=None, param=None):
    """Velocities as float32 arrays (coordinates float64)."""
    mem = _mem_of(q0, q1, q2, v0, v1, v2, species, param)
    n = len(q0)
    return _check(ctx, load_library().dust_load_particles_v32(
        ctx, n, _ptr(q0)[0], _ptr(q1)[0], _ptr(q2)[0], _ptr(v0)[0], _ptr(v1)[0], _ptr(v2)[0],
        _ptr(species)[0], _ptr(param)[0], mem))


def dust_step(ctx, dt):
    return _check(ctx, load_library().dust_step(ctx, float(dt)))


def dust_sync(ctx, stats=None, check=True):
    st = dust_stats() if stats is None else stats
    rc = load_library().dust_sync(ctx, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return rc, st


def dust_get_deposit(ctx, fixed=None, as_double=None):
    mem = _mem_of(fixed, as_double)
    qo = ctypes.c_double()
    _check(ctx, load_library().dust_get_deposit(ctx, _ptr(fixed)[0], _ptr(as_double)[0],
                                                ctypes.byref(qo), mem))
    return qo.value


def dust_get_mass_deposit(ctx, fixed=None, as_double=None):
    mem = _mem_of(fixed, as_double)
    qo = ctypes.c_double()
    _check(ctx, load_library().dust_get_mass_deposit(ctx, _ptr(fixed)[0], _ptr(as_double)[0],
                                                     ctypes.byref(qo), mem))
    return qo.value


def dust_get_particles(ctx, cap, q0=None, q1=None, q2=None, v0=None, v1=None, v2=None, ids=None):
    mem = _mem_of(q0, q1, q2, v0, v1, v2, ids)
    n = ctypes.c_int64()
    _check(ctx, load_library().dust_get_particles(
        ctx, int(cap), _ptr(q0)[0], _ptr(q1)[0], _ptr(q2)[0], _ptr(v0)[0], _ptr(v1)[0],
        _ptr(v2)[0], _ptr(ids)[0], ctypes.byref(n), mem))
    return n.value


def dust_get_particles_v32(ctx, cap, q0=None, q1=None, q2=None, v0=None, v1=None, v2=None, ids=None):
    """Velocities into float32 arrays (coordinates float64)."""
    mem = _mem_of(q0, q1, q2, v0, v1, v2, ids)
    n = ctypes.c_int64()
    _check(ctx, load_library().dust_get_particles_v32(
        ctx, int(cap), _ptr(q0)[0], _ptr(q1)[0], _ptr(q2)[0], _ptr(v0)[0], _ptr(v1)[0],
        _ptr(v2)[0], _ptr(ids)[0], ctypes.byref(n), mem))
    return n.value


def dust_get_kernel_times(ctx, reset=False):
    t = dust_kernel_times()
    _check(ctx, load_library().dust_get_kernel_times(ctx, ctypes.byref(t), int(bool(reset))))
    return t


def dust_step_noalloc(geometry, grid, species, weight, quantum, t, dt, q, p, gas, dep,
                      species_idx=None, param=None, status_out=None, device=0, stream=None):
    """q, p: three CUDA float64 tensors each (updated in place); gas: CUDA
    float64 [ncell, 4]; dep: CUDA int64 [ncell, 4] (overwritten);
    species_idx / param / status_out: CUDA tensors or None; stream: a
    cudaStream_t handle (int) or None."""
    for a in list(q) + list(p) + [gas, dep, species_idx, param, status_out]:
        if a is not None and _ptr(a)[1] != DUST_MEM_DEVICE:
            raise ValueError("dust_step_noalloc takes device arrays only")
    lib = load_library()
    arr = (dust_species * len(species))(*species)
    rc = lib.dust_step_noalloc(ctypes.byref(geometry), ctypes.byref(grid), arr, len(species),
                               int(weight), float(quantum), float(t), float(dt), len(q[0]),
                               _ptr(q[0])[0], _ptr(q[1])[0], _ptr(q[2])[0],
                               _ptr(p[0])[0], _ptr(p[1])[0], _ptr(p[2])[0],
                               _ptr(species_idx)[0], _ptr(param)[0], _ptr(gas)[0], _ptr(dep)[0],
                               _ptr(status_out)[0], int(device), stream)
    if rc != DUST_OK:
        raise DustError(rc, lib.dust_last_error(None).decode())
    return rc


def dust_batch_create(ctxs, options=None):
    """ctxs: context handles.  Returns an opaque batch handle."""
    lib = load_library()
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    rc = lib.dust_batch_create(ctypes.byref(out), arr, len(ctxs),
                               ctypes.byref(options) if options is not None else None)
    if rc != DUST_OK:
        raise DustError(rc, lib.dust_batch_last_error(None).decode())
    return out.value


def dust_batch_step(batch, dt, nsteps):
    """dt: one step length per instance."""
    lib = load_library()
    arr = (ctypes.c_double * len(dt))(*[float(x) for x in dt])
    rc = lib.dust_batch_step(batch, arr, int(nsteps))
    if rc != DUST_OK:
        raise DustError(rc, lib.dust_batch_last_error(batch).decode())
    return rc


def dust_batch_last_error(batch):
    m = load_library().dust_batch_last_error(batch)
    return m.decode() if m else ""


def dust_batch_destroy(batch):
    load_library().dust_batch_destroy(batch)


def dust_last_error(ctx):
    m = load_library().dust_last_error(ctx)
    return m.decode() if m else ""


def dust_destroy(ctx):
    load_library().dust_destroy(ctx)


# ------------------------------------------------- descriptor helpers ----
def make_descriptors(w, precision=DUST_MIXED, feedback=None, stream=None, sort_interval=0,
                     kernel=DUST_KERNEL_AUTO, quantum=0.0, device=0, timing=0, tile=(0, 0, 0),
                     pusher=None, gas_predictor=0, host_io_async=0, test_wait_timeout=0):
    """C descriptors for a workload from paper_1908_10793_gb300.inputs.
    Returns (geometry, grid, species list, options, keepalive)."""
    geo = dust_geometry(kind=w.geom, fargo=w.fargo, omega=w.omega, q=w.qshear, gm=w.gm,
                        vertical_gravity=w.vertical_gravity)
    edges = [np.ascontiguousarray(e, dtype=np.float64) for e in w.edges]
    grid = dust_grid()
    for d in range(3):
        grid.n[d] = len(edges[d]) - 1
        grid.edges[d] = edges[d].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        grid.bc[d] = w.bc[d]
    sp = [dust_species(mass=m, tau_mode=k, tau_value=t)
          for m, k, t in zip(w.species_mass, w.species_tau_mode, w.species_tau)]
    opt = dust_options(precision=precision, weight=w.weight,
                       feedback_apply=w.feedback if feedback is None else feedback,
                       quantum=quantum, stream=stream, sort_interval=sort_interval,
                       kernel=kernel, device=device, timing=timing,
                       pusher=getattr(w, "pusher", DUST_PUSHER_EM) if pusher is None else pusher,
                       gas_predictor=gas_predictor, host_io_async=host_io_async,
                       test_wait_timeout=test_wait_timeout)
    for d in range(3):
        opt.tile[d] = int(tile[d])
    return geo, grid, sp, opt, edges


class Context:
    """Owns one dust context; thin convenience over the C names."""

    def __init__(self, w, **kw):
        geo, grid, sp, opt, self._keep = make_descriptors(w, **kw)
        self.handle = dust_create(geo, grid, sp, opt)
        self.ncell = w.ncell

    def set_gas(self, rho, v):
        dust_set_gas(self.handle, rho, v[0], v[1], v[2])

    def load(self, q, v, species=None, param=None):
        self.n = len(q[0])
        dust_load_particles(self.handle, q[0], q[1], q[2], v[0], v[1], v[2], species, param)

    def step(self, dt):
        dust_step(self.handle, dt)

    def sync(self, check=True):
        return dust_sync(self.handle, check=check)

    def deposit(self):
        fixed = np.zeros((self.ncell, 4), np.int64)
        quantum = dust_get_deposit(self.handle, fixed=fixed)
        return fixed, quantum

    def mass_deposit(self):
        """Dust mass per zone (int64 in units of the quantum) and the quantum."""
        fixed = np.zeros(self.ncell, np.int64)
        quantum = dust_get_mass_deposit(self.handle, fixed=fixed)
        return fixed, quantum

    def particles(self):
        n = self.n
        out = [np.empty(n) for _ in range(6)]
        ids = np.empty(n, np.int64)
        dust_get_particles(self.handle, n, *out, ids=ids)
        return out[:3], out[3:], ids

    def gas(self):
        out = [np.empty(self.ncell) for _ in range(4)]
        dust_get_gas(self.handle, *out)
        return out[0], out[1:]

    def kernel_times(self, reset=False):
        return dust_get_kernel_times(self.handle, reset)

    def close(self):
        if self.handle:
            dust_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
