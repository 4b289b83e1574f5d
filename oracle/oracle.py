"""ctypes wrapper around dust_oracle.c (test infrastructure only).

The C file is compiled with gcc -O2 -ffp-contract=off (no FMA contraction, no
fast-math) into oracle/_build/liboracle.so.  Arrays are numpy float64 /
uint8, passed by pointer; the oracle updates them in place.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

OG_CARTESIAN, OG_SHEARING_BOX, OG_CYLINDRICAL, OG_SPHERICAL = 0, 1, 2, 3
OB_PERIODIC, OB_OUTFLOW = 0, 1
OW_CIC, OW_TSC, OW_VOLUME = 0, 1, 2
OT_CONST, OT_STOKES, OT_EPSTEIN = 0, 1, 2
OP_EM, OP_SEMI_IMPLICIT = 0, 1
(W1_CART_CIC, W1_CART_TSC, W1_CYL_R_CIC, W1_CYL_R_TSC, W1_SPH_R_CIC,
 W1_SPH_R_TSC, W1_SPH_TH_CIC, W1_SPH_TH_TSC, W1_CYL_R_VOL, W1_SPH_R_VOL,
 W1_SPH_TH_VOL) = range(11)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dust_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library (gcc, plain C, FP64).  The mutation
    tests point DUST_ORACLE_LIB at a deliberately broken build instead."""
    planted = os.environ.get("DUST_ORACLE_LIB")
    if planted:
        return planted
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


class _ProblemC(ctypes.Structure):
    _fields_ = [
        ("geom", ctypes.c_int), ("fargo", ctypes.c_int),
        ("omega", ctypes.c_double), ("q", ctypes.c_double), ("gm", ctypes.c_double),
        ("vertical_gravity", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("edges", ctypes.POINTER(ctypes.c_double) * 3),
        ("bc", ctypes.c_int * 3),
        ("weight", ctypes.c_int),
        ("n_species", ctypes.c_int),
        ("sp_mass", ctypes.POINTER(ctypes.c_double)),
        ("sp_tau_mode", ctypes.POINTER(ctypes.c_int)),
        ("sp_tau", ctypes.POINTER(ctypes.c_double)),
        ("feedback_apply", ctypes.c_int),
        ("pusher", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_weights_1d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, dp]
            lib.oracle_weights_1d.restype = None
            lib.oracle_weights_vol.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int,
                                               ctypes.c_int, dp]
            lib.oracle_weights_vol.restype = None
            lib.oracle_locate.argtypes = [dp, ctypes.c_int, ctypes.c_double]
            lib.oracle_locate.restype = ctypes.c_int
            lib.oracle_step.argtypes = [ctypes.POINTER(_ProblemC)] + [dp] * 6 + [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_double, ctypes.c_double, dp, dp, dp, dp, dp]
            lib.oracle_step.restype = ctypes.c_int64
            lib.oracle_step_fixed.argtypes = lib.oracle_step.argtypes + [ctypes.c_void_p,
                                                                         ctypes.c_double]
            lib.oracle_step_fixed.restype = ctypes.c_int64
            lib.oracle_gas_momentum.argtypes = [ctypes.POINTER(_ProblemC)] + [dp] * 6
            lib.oracle_gas_momentum.restype = None
            lib.oracle_gas_predictor.argtypes = [ctypes.POINTER(_ProblemC)] + [dp] * 6 + [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_double] + [dp] * 8
            lib.oracle_gas_predictor.restype = None
            lib.oracle_deposit_mass.argtypes = [ctypes.POINTER(_ProblemC)] + [dp] * 3 + [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, dp]
            lib.oracle_deposit_mass.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def weights_1d(kind, x, lo, hi):
    """Weights of zones (i-1, i, i+1) for a grain at x hosted by zone [lo, hi)."""
    w = np.zeros(3)
    _load().oracle_weights_1d(int(kind), float(x), float(lo), float(hi), _dp(w))
    return w


def weights_vol(kind, x, edges, i):
    """Volume weights (Eq. CIC_vol) of zones (i-1, i, i+1) for a grain at x
    hosted by zone i of the grid with the given edges."""
    e = _f64(edges)
    w = np.zeros(3)
    _load().oracle_weights_vol(int(kind), float(x), _dp(e), len(e) - 1, int(i), _dp(w))
    return w


def locate(edges, x):
    e = _f64(edges)
    return _load().oracle_locate(_dp(e), len(e) - 1, float(x))


class Problem:
    """Geometry, grid, species and options of one oracle instance."""

    def __init__(self, geom, edges, bc=(OB_PERIODIC,) * 3, weight=OW_TSC,
                 species_mass=(1.0,), species_tau_mode=(OT_CONST,), species_tau=(1.0,),
                 fargo=0, omega=1.0, q=1.5, gm=0.0, vertical_gravity=0, feedback_apply=0,
                 pusher=OP_EM):
        if pusher == OP_SEMI_IMPLICIT and geom not in (OG_CARTESIAN, OG_SHEARING_BOX):
            raise ValueError("the semi-implicit pusher is defined for Cartesian and "
                             "shearing-box geometries (Sec. 3.2.1)")
        self.edges = [_f64(e) for e in edges]
        self.n = [len(e) - 1 for e in self.edges]
        self.sp_mass = _f64(species_mass)
        self.sp_tau = _f64(species_tau)
        self.sp_mode = np.ascontiguousarray(species_tau_mode, dtype=np.int32)
        c = _ProblemC()
        c.geom, c.fargo = int(geom), int(fargo)
        c.omega, c.q, c.gm = float(omega), float(q), float(gm)
        c.vertical_gravity = int(vertical_gravity)
        for d in range(3):
            c.n[d] = self.n[d]
            c.edges[d] = _dp(self.edges[d])
            c.bc[d] = int(bc[d])
        c.weight = int(weight)
        c.n_species = len(self.sp_mass)
        c.sp_mass = _dp(self.sp_mass)
        c.sp_tau_mode = self.sp_mode.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        c.sp_tau = _dp(self.sp_tau)
        c.feedback_apply = int(feedback_apply)
        c.pusher = int(pusher)
        self.c = c
        self.geom = int(geom)

    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]


def step(prob, q, p, active, t, dt, rho, pg, species=None, param=None):
    """One step in place.  q, p: lists of three float64 arrays; active: uint8
    array; rho: float64 [ncell]; pg: list of three float64 [ncell] arrays.
    Returns (dense deposit [ncell, 4], number removed)."""
    lib = _load()
    for a in list(q) + list(p) + [rho] + list(pg):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    assert active.dtype == np.uint8
    n = len(q[0])
    dep = np.zeros((prob.ncell, 4))
    sp = None if species is None else np.ascontiguousarray(species, dtype=np.uint8)
    pa = None if param is None else _f64(param)
    removed = lib.oracle_step(ctypes.byref(prob.c), _dp(q[0]), _dp(q[1]), _dp(q[2]),
                              _dp(p[0]), _dp(p[1]), _dp(p[2]),
                              None if sp is None else sp.ctypes.data,
                              None if pa is None else pa.ctypes.data,
                              active.ctypes.data, n, float(t), float(dt),
                              _dp(rho), _dp(pg[0]), _dp(pg[1]), _dp(pg[2]), _dp(dep))
    return dep, removed


def step_fixed(prob, q, p, active, t, dt, rho, pg, quantum, species=None, param=None):
    """One step in place, like step(), with the deposit also given by the
    fixed-point rule (per grain: the non-host nodes get the nearest integer
    of W D / quantum, the host zone the rest of the nearest integer of
    D / quantum).  Returns (dense deposit [ncell, 4], int64 deposit
    [ncell, 4] in units of quantum, number removed)."""
    lib = _load()
    for a in list(q) + list(p) + [rho] + list(pg):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    assert active.dtype == np.uint8
    n = len(q[0])
    dep = np.zeros((prob.ncell, 4))
    fixed = np.zeros((prob.ncell, 4), np.int64)
    sp = None if species is None else np.ascontiguousarray(species, dtype=np.uint8)
    pa = None if param is None else _f64(param)
    removed = lib.oracle_step_fixed(ctypes.byref(prob.c), _dp(q[0]), _dp(q[1]), _dp(q[2]),
                                    _dp(p[0]), _dp(p[1]), _dp(p[2]),
                                    None if sp is None else sp.ctypes.data,
                                    None if pa is None else pa.ctypes.data,
                                    active.ctypes.data, n, float(t), float(dt),
                                    _dp(rho), _dp(pg[0]), _dp(pg[1]), _dp(pg[2]), _dp(dep),
                                    fixed.ctypes.data, float(quantum))
    return dep, fixed, removed


def gas_predictor(prob, q, p, active, dt, rho, pg, species=None, param=None):
    """Half-step gas prediction from the drag of the grains at x^n.  Returns
    (impulse per zone [ncell, 3], half-step momentum-like gas velocity list)."""
    lib = _load()
    imp = np.zeros((prob.ncell, 3))
    ph = [np.zeros(prob.ncell) for _ in range(3)]
    qq = [_f64(x) for x in q]
    pp = [_f64(x) for x in p]
    rr = _f64(rho)
    gg = [_f64(x) for x in pg]
    sp = None if species is None else np.ascontiguousarray(species, dtype=np.uint8)
    pa = None if param is None else _f64(param)
    act = np.ascontiguousarray(active, dtype=np.uint8)
    lib.oracle_gas_predictor(ctypes.byref(prob.c), _dp(qq[0]), _dp(qq[1]), _dp(qq[2]),
                             _dp(pp[0]), _dp(pp[1]), _dp(pp[2]),
                             None if sp is None else sp.ctypes.data,
                             None if pa is None else pa.ctypes.data,
                             act.ctypes.data, len(qq[0]), float(dt), _dp(rr),
                             _dp(gg[0]), _dp(gg[1]), _dp(gg[2]), _dp(imp),
                             _dp(ph[0]), _dp(ph[1]), _dp(ph[2]))
    return imp, ph


def deposit_mass(prob, q, active=None, species=None):
    """Dust mass per zone (Eq. deposition with q_p = m_p) of the grains at
    positions q (active ones only), with the problem's weighting."""
    q = [_f64(x) for x in q]
    n = len(q[0])
    active = np.ones(n, np.uint8) if active is None else np.ascontiguousarray(active, np.uint8)
    sp = None if species is None else np.ascontiguousarray(species, np.uint8)
    out = np.zeros(prob.ncell)
    _load().oracle_deposit_mass(ctypes.byref(prob.c), _dp(q[0]), _dp(q[1]), _dp(q[2]),
                                None if sp is None else sp.ctypes.data, active.ctypes.data, n,
                                _dp(out))
    return out


def gas_momentum(prob, v):
    """Momentum-like gas velocity per zone from physical components v[0..2]."""
    v = [_f64(x) for x in v]
    pg = [np.zeros(prob.ncell) for _ in range(3)]
    _load().oracle_gas_momentum(ctypes.byref(prob.c), _dp(v[0]), _dp(v[1]), _dp(v[2]),
                                _dp(pg[0]), _dp(pg[1]), _dp(pg[2]))
    return pg
