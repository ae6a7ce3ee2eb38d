"""ctypes binding of the plain FP64 CPU oracle (``turret_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the correctness reference for the
CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may load it.  It imports nothing from the CUDA package and the
CUDA package imports nothing from here.

Every function mirrors one C entry point; the C file cites the passage of the
paper (arXiv 2408.15115) each one follows.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "turret_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i32p = C.POINTER(C.c_int32)


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc_x", C.c_int), ("bc_y", C.c_int),
        ("bc_bottom", C.c_int), ("bc_top", C.c_int),
        ("sponge", C.c_int), ("slide", C.c_int),
        ("anchor_frac", C.c_double), ("tau0", C.c_double),
        ("force_scheme", C.c_int), ("rot_form", C.c_int), ("gravity", C.c_int),
        ("renorm", C.c_int), ("ibm_cycles", C.c_int),
        ("kappa", C.c_double), ("g", C.c_double * 3),
        ("fixed_position", C.c_int), ("uw_bottom", C.c_double * 3), ("uw_top", C.c_double * 3),
        ("reinject_trigger", C.c_int), ("reinject_target", C.c_int), ("reinject_below", C.c_int),
        ("reinject_above", C.c_int), ("force_eval", C.c_int),
        ("predictor", C.c_int), ("pred_warm", C.c_int), ("pred_eps", C.c_double),
    ]


class OrcGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("per_x", C.c_int), ("per_y", C.c_int), ("per_z", C.c_int)]


def build(force=False):
    """Compile the oracle with gcc (-O2, OpenMP); returns the library path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
            subprocess.check_call(cmd)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_peskin.restype = C.c_double
        L.orc_hermite.restype = C.c_double
        L.orc_a1.restype = C.c_double
        L.orc_new.restype = C.c_void_p
        L.orc_new.argtypes = [C.POINTER(OrcParams)]
        L.orc_free.argtypes = [C.c_void_p]
        for name in ("orc_init_fields", "orc_set_force", "orc_get_f", "orc_get_fpost", "orc_set_f",
                     "orc_get_velocity", "orc_get_stress", "orc_get_force_field", "orc_get_utop",
                     "orc_particle_state", "orc_markers", "orc_set_particle_dyn",
                     "orc_advance_particle_only", "orc_fluid_step", "orc_step", "orc_load_particle"):
            getattr(L, name).restype = C.c_int if name in ("orc_step", "orc_load_particle") else None
        L.orc_get_threads.restype = C.c_int
        L.orc_ibm_warm.restype = C.c_int
        L.orc_ibm_cycles.restype = C.c_int64
        L.orc_ibm_cycles.argtypes = [C.c_void_p]
        L.orc_predictor_step.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


def lattice():
    xi = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().orc_lattice(xi.ctypes.data_as(_ip), _p(w))
    return xi, w


def hermite(i, idx):
    a = np.array(idx, dtype=np.int32)
    return lib().orc_hermite(int(i), len(idx), a.ctypes.data_as(_ip))


def feq(rho, u):
    out = np.zeros(27)
    lib().orc_feq(C.c_double(rho), _p(_c(u)), _p(out))
    return out


def a1(idx, P, u):
    a = np.array(idx, dtype=np.int32)
    return lib().orc_a1(len(idx), a.ctypes.data_as(_ip), _p(_c(P)), _p(_c(u)))


def fone(P, u):
    out = np.zeros(27)
    lib().orc_fone(_p(_c(P)), _p(_c(u)), _p(out))
    return out


def moments(f):
    rho = C.c_double()
    u = np.zeros(3)
    P = np.zeros(9)
    lib().orc_moments(_p(_c(f)), C.byref(rho), _p(u), _p(P))
    return rho.value, u, P.reshape(3, 3)


def collide_cell(f, h, tau, force_scheme=0):
    out = np.zeros(27)
    lib().orc_collide_cell(_p(_c(f)), _p(_c(h)), C.c_double(tau), C.c_int(force_scheme), _p(out))
    return out


def stress(f, tau):
    sig = np.zeros(9)
    u = np.zeros(3)
    lib().orc_stress(_p(_c(f)), C.c_double(tau), _p(sig), _p(u))
    return sig.reshape(3, 3), u


def peskin(r):
    return lib().orc_peskin(C.c_double(r))


def mesh_props(verts, tris):
    V = _c(verts)
    T = _c(tris, np.int32)
    nv, nt = V.shape[0], T.shape[0]
    dS = np.zeros(nv)
    nrm = np.zeros((nv, 3))
    vol = C.c_double()
    com = np.zeros(3)
    Jm = np.zeros(9)
    area = C.c_double()
    rc = lib().orc_mesh_props(_p(V), C.c_int64(nv), T.ctypes.data_as(_i32p), C.c_int64(nt), _p(dS), _p(nrm),
                              C.byref(vol), _p(com), _p(Jm), C.byref(area))
    if rc != 0:
        raise ValueError("mesh is not a closed, outward-oriented two-manifold")
    return dict(dS=dS, normals=nrm, volume=vol.value, com=com, J_over_m=Jm.reshape(3, 3), area=area.value)


def _grid(shape, periodic):
    nz, ny, nx = shape
    return OrcGrid(nx, ny, nz, int(periodic[0]), int(periodic[1]), int(periodic[2]))


def interp(field, X, periodic=(True, True, True)):
    """field: (nz, ny, nx, ncomp); X: (nm, 3) in (x, y, z) cell coordinates."""
    field = _c(field)
    nz, ny, nx, nc = field.shape
    X = _c(X)
    out = np.zeros((X.shape[0], nc))
    g = _grid((nz, ny, nx), periodic)
    lib().orc_interp(C.byref(g), _p(field), C.c_int(nc), _p(X), C.c_int64(X.shape[0]), _p(out))
    return out


def spread(hk, X, dS, shape, periodic=(True, True, True)):
    X = _c(X)
    out = np.zeros(tuple(shape) + (3,))
    g = _grid(shape, periodic)
    lib().orc_spread(C.byref(g), _p(_c(hk)), _p(X), _p(_c(dS)), C.c_int64(X.shape[0]), _p(out))
    return out


def ibm(ustar, X, U, dS, ncycles=4, periodic=(True, True, True)):
    ustar = _c(ustar)
    shape = ustar.shape[:3]
    X = _c(X)
    himm = np.zeros(tuple(shape) + (3,))
    hl = np.zeros((X.shape[0], 3))
    g = _grid(shape, periodic)
    lib().orc_ibm(C.byref(g), _p(ustar), _p(X), _p(_c(U)), _p(_c(dS)), C.c_int64(X.shape[0]), C.c_int(ncycles),
                  _p(himm), _p(hl))
    return himm, hl


def ibm_warm(ustar, X, U, dS, h0, ncycles=4, eps=0.0, periodic=(True, True, True)):
    """IBM cycles warm-started from the Lagrangian force h0 (predictor option):
    returns (h_imm dense, h, cycles run)."""
    ustar = _c(ustar)
    shape = ustar.shape[:3]
    X = _c(X)
    himm = np.zeros(tuple(shape) + (3,))
    hl = _c(h0).copy()
    g = _grid(shape, periodic)
    run = lib().orc_ibm_warm(C.byref(g), _p(ustar), _p(X), _p(_c(U)), _p(_c(dS)), C.c_int64(X.shape[0]),
                             C.c_int(ncycles), C.c_double(eps), _p(himm), _p(hl))
    return himm, hl, run


class Sim:
    """Dense FP64 window simulation (fluid + optional particle), Table 1 order.

    Boundary codes: bc_x/bc_y 0 periodic, 1 no-slip; bc_bottom/bc_top 0 periodic,
    1 no-slip, 2 constant pressure (top only), 3 no-slip wall moving in its plane
    with velocity uw_bottom / uw_top.  fixed_position 1 holds the particle's
    centre (v = 0) and leaves its rotation free.  reinject = (trigger, target,
    below, above): the re-injection copy of Sec. 2.5 (slide 0 only; trigger 0
    off).  force_eval 0: force and torque from the stress on the surface
    offset by 2 cells along the normals (outside the diffuse interface); 1: the
    stress interpolated at the markers, as printed in Sec. 2.2.  predictor 1:
    markers move with the body's motion at t + 1 estimated from a linear
    extrapolation of F, T (not in the paper); pred_warm 1 with it: IBM cycles
    warm-started from the previous step's h, skipped once the slip is below
    pred_eps.  Arrays are (nz, ny, nx, ...)."""

    STATE_FIELDS = 45

    def __init__(self, nx, ny, nz, tau, bc_x=0, bc_y=0, bc_bottom=0, bc_top=0, sponge=0, slide=0,
                 anchor_frac=0.25, force_scheme=0, rot_form=0, gravity=0, renorm=0, ibm_cycles=4,
                 kappa=1.0, g=(0.0, 0.0, 0.0), fixed_position=0, uw_bottom=(0.0, 0.0, 0.0), uw_top=(0.0, 0.0, 0.0),
                 reinject=(0, 0, 0, 0), force_eval=0, predictor=0, pred_warm=0, pred_eps=0.0):
        self.shape = (nz, ny, nx)
        p = OrcParams(nx, ny, nz, bc_x, bc_y, bc_bottom, bc_top, sponge, slide, float(anchor_frac), float(tau),
                      force_scheme, rot_form, gravity, renorm, ibm_cycles, float(kappa), (C.c_double * 3)(*g),
                      int(fixed_position), (C.c_double * 3)(*uw_bottom), (C.c_double * 3)(*uw_top),
                      *[int(v) for v in reinject], int(force_eval), int(predictor), int(pred_warm),
                      float(pred_eps))
        self._params = p
        self._s = lib().orc_new(C.byref(p))

    def __del__(self):
        if getattr(self, "_s", None) and _lib is not None:
            _lib.orc_free(C.c_void_p(self._s))
            self._s = None

    def init_fields(self, rho=None, u=None):
        L = lib()
        rp = _p(_c(rho)) if rho is not None else None
        up = _p(_c(u)) if u is not None else None
        L.orc_init_fields(C.c_void_p(self._s), rp, up)

    def set_force(self, h):
        lib().orc_set_force(C.c_void_p(self._s), _p(_c(h)))

    def fluid_step(self, n=1):
        lib().orc_fluid_step(C.c_void_p(self._s), C.c_int(n))

    def load_particle(self, verts, tris, r0, v0=(0, 0, 0), w0=(0, 0, 0)):
        V = _c(verts)
        T = _c(tris, np.int32)
        rc = lib().orc_load_particle(C.c_void_p(self._s), _p(V), C.c_int64(V.shape[0]), T.ctypes.data_as(_i32p),
                                     C.c_int64(T.shape[0]), _p(_c(r0)), _p(_c(v0)), _p(_c(w0)))
        if rc != 0:
            raise ValueError("orc_load_particle failed (%d)" % rc)

    def step(self, n=1):
        rc = lib().orc_step(C.c_void_p(self._s), C.c_int(n))
        if rc != 0:
            raise RuntimeError("orc_step failed (%d)" % rc)

    def _get(self, fn, ncomp):
        out = np.zeros(self.shape + (ncomp,))
        getattr(lib(), fn)(C.c_void_p(self._s), _p(out))
        return out

    def f(self):
        return self._get("orc_get_f", 27)

    def fpost(self):
        return self._get("orc_get_fpost", 27)

    def set_f(self, f):
        lib().orc_set_f(C.c_void_p(self._s), _p(_c(f)))

    def velocity(self):
        return self._get("orc_get_velocity", 3)

    def stress(self):
        return self._get("orc_get_stress", 9).reshape(self.shape + (3, 3))

    def force_field(self):
        return self._get("orc_get_force_field", 3)

    def utop(self):
        nz, ny, nx = self.shape
        out = np.zeros((ny, nx, 3))
        lib().orc_get_utop(C.c_void_p(self._s), _p(out))
        return out

    def state(self):
        o = np.zeros(self.STATE_FIELDS)
        lib().orc_particle_state(C.c_void_p(self._s), _p(o))
        return dict(r=o[0:3].copy(), d=o[3:12].reshape(3, 3).copy(), v=o[12:15].copy(), w=o[15:18].copy(),
                    F=o[18:21].copy(), T=o[21:24].copy(), L=o[24:27].copy(), origin=o[27:30].copy(),
                    step=int(o[30]), volume=o[31], J_over_m=o[32:41].reshape(3, 3).copy(), area=o[41],
                    Fp=o[42:45].copy())

    def markers(self, nm):
        X = np.zeros((nm, 3)); n = np.zeros((nm, 3)); U = np.zeros((nm, 3)); dS = np.zeros(nm); hl = np.zeros((nm, 3))
        lib().orc_markers(C.c_void_p(self._s), _p(X), _p(n), _p(U), _p(dS), _p(hl))
        return dict(X=X, n=n, U=U, dS=dS, hl=hl)

    def set_particle_dyn(self, r, d, v, w, L, F, T):
        lib().orc_set_particle_dyn(C.c_void_p(self._s), *[_p(_c(a)) for a in (r, d, v, w, L, F, T)])

    def advance_particle_only(self, n=1):
        lib().orc_advance_particle_only(C.c_void_p(self._s), C.c_int(n))

    def ibm_cycles(self):
        """IBM cycles run so far."""
        return int(lib().orc_ibm_cycles(C.c_void_p(self._s)))

    def predictor_step(self, F, T):
        """Predictor and 6DOF update alone: enter F, T as the current force
        evaluation, predict, advance; returns the (v, omega) the markers move with."""
        vel, om = np.zeros(3), np.zeros(3)
        lib().orc_predictor_step(C.c_void_p(self._s), _p(_c(F)), _p(_c(T)), _p(vel), _p(om))
        return vel, om
