"""ctypes binding of libturret.so (declared in include/turret.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides the device workspaces and the CUDA stream.
The library is built in-tree (``paper_2408_15115_gb300/libturret.so``); if it
is missing this module raises instead of falling back to anything else.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libturret.so")

STATUS = {0: "TURRET_OK", 1: "TURRET_EINVAL", 2: "TURRET_ENOMEM", 3: "TURRET_ECUDA", 4: "TURRET_ESTATE",
          5: "TURRET_EDIVERGED", 6: "TURRET_ETIMEOUT", 7: "TURRET_EDOMAIN", 8: "TURRET_EOVERFLOW"}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
PERIODIC, NOSLIP, PRESSURE = 0, 1, 2


class Window(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("bc_bottom", C.c_int32), ("bc_top", C.c_int32),
                ("sponge_cells", C.c_int32), ("slide", C.c_int32), ("pad0", C.c_int32),
                ("anchor_frac", C.c_double)]


class Flags(C.Structure):
    _fields_ = [("force_scheme", C.c_int32), ("rot_form", C.c_int32), ("gravity", C.c_int32),
                ("renorm_orientation", C.c_int32), ("ibm_cycles", C.c_int32), ("no_graph", C.c_int32),
                ("stochastic_rounding", C.c_int32), ("fixed_position", C.c_int32), ("force_eval", C.c_int32),
                ("staged_loads", C.c_int32)]


class ParticleState(C.Structure):
    _fields_ = [("r", C.c_double * 3), ("d", C.c_double * 9), ("v", C.c_double * 3), ("w", C.c_double * 3),
                ("F", C.c_double * 3), ("T", C.c_double * 3), ("L", C.c_double * 3),
                ("origin", C.c_int64 * 3), ("step", C.c_int64), ("status", C.c_int32), ("n_markers", C.c_int32),
                ("volume", C.c_double), ("area", C.c_double), ("kernels_per_step", C.c_int32),
                ("pad0", C.c_int32), ("Fp", C.c_double * 3)]


class TurretError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class PredictorStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("net_steps", C.c_int64), ("fallbacks", C.c_int64), ("cycles", C.c_int64),
                ("logged", C.c_int64), ("resid", C.c_double), ("slip", C.c_double * 8), ("hist_n", C.c_int32),
                ("fallback", C.c_int32)]


class AdamW(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float)]


_lib = None
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


def lib():
    """Load libturret.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libturret.so is not built; run paper_2408_15115_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.lbm_workspace_bytes.restype = C.c_size_t
        L.lbm_workspace_bytes.argtypes = [C.POINTER(Window), C.c_int]
        L.lbm_init.restype = C.c_int
        L.lbm_init.argtypes = [C.POINTER(vp), C.POINTER(Window), C.c_int, C.c_double, C.c_double, _dp, C.c_int,
                               vp, C.c_size_t, vp]
        L.lbm_set_flags.restype = C.c_int
        L.lbm_set_flags.argtypes = [vp, C.POINTER(Flags)]
        L.lbm_set_wall_velocity.restype = C.c_int
        L.lbm_set_wall_velocity.argtypes = [vp, _dp, _dp]
        L.lbm_set_fields.restype = C.c_int
        L.lbm_set_fields.argtypes = [vp, _dp, _dp]
        L.ibm_workspace_bytes.restype = C.c_size_t
        L.ibm_workspace_bytes.argtypes = [vp, _dp, C.c_int64, C.POINTER(C.c_int32), C.c_int64]
        L.ibm_load_surface.restype = C.c_int
        L.ibm_load_surface.argtypes = [vp, _dp, C.c_int64, C.POINTER(C.c_int32), C.c_int64, _dp, _dp, _dp, vp,
                                       C.c_size_t]
        L.step.restype = C.c_int
        L.step.argtypes = [vp, C.c_int64]
        L.lbm_fluid_step.restype = C.c_int
        L.lbm_fluid_step.argtypes = [vp, C.c_int64]
        L.query_particle_state.restype = C.c_int
        L.query_particle_state.argtypes = [vp, C.POINTER(ParticleState)]
        L.lbm_copy_macro.restype = C.c_int
        L.lbm_copy_macro.argtypes = [vp, vp]
        L.lbm_copy_populations.restype = C.c_int
        L.lbm_copy_populations.argtypes = [vp, vp]
        L.lbm_destroy.restype = C.c_int
        L.lbm_destroy.argtypes = [vp]
        L.ibm_spread_workspace_bytes.restype = C.c_size_t
        L.ibm_spread_workspace_bytes.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int64]
        L.ibm_spread.restype = C.c_int
        L.ibm_spread.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_size_t, vp]
        L.ibm_spread_noalloc.restype = C.c_int
        L.ibm_spread_noalloc.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32, vp, vp]
        L.turret_last_error.restype = C.c_char_p
        L.turret_last_error.argtypes = [vp]
        L.turret_batch_workspace_bytes.restype = C.c_size_t
        L.turret_batch_workspace_bytes.argtypes = [C.c_int32]
        L.turret_batch_init.restype = C.c_int
        L.turret_batch_init.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int32, vp, C.c_size_t, vp]
        L.turret_batch_set_tiles.restype = C.c_int
        L.turret_batch_set_tiles.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
        L.turret_batch_step.restype = C.c_int
        L.turret_batch_step.argtypes = [vp, C.c_int64]
        L.turret_batch_destroy.restype = C.c_int
        L.turret_batch_destroy.argtypes = [vp]
        L.turret_batch_last_error.restype = C.c_char_p
        L.turret_batch_last_error.argtypes = [vp]
        L.mlp_workspace_bytes.restype = C.c_size_t
        L.mlp_workspace_bytes.argtypes = [C.c_int32]
        L.mlp_init.restype = C.c_int
        L.mlp_init.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32, _fp, vp, C.c_size_t, vp]
        for name in ("mlp_set_params", "mlp_get_params"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [vp, _fp]
        L.mlp_set_norm.restype = C.c_int
        L.mlp_set_norm.argtypes = [vp, _fp, _fp, _fp, _fp]
        for name in ("mlp_forward", "mlp_infer"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [vp, vp, C.c_int32, vp]
        L.mlp_loss_grad.restype = C.c_int
        L.mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int32, _fp, vp]
        L.mlp_train_step.restype = C.c_int
        L.mlp_train_step.argtypes = [vp, vp, vp, C.c_int32, C.POINTER(AdamW), _fp]
        L.mlp_destroy.restype = C.c_int
        L.mlp_destroy.argtypes = [vp]
        L.mlp_last_error.restype = C.c_char_p
        L.mlp_last_error.argtypes = [vp]
        L.turret_set_predictor.restype = C.c_int
        L.turret_set_predictor.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_double, C.c_double]
        L.turret_set_log.restype = C.c_int
        L.turret_set_log.argtypes = [vp, vp, C.c_int64]
        L.turret_set_reinjection.restype = C.c_int
        L.turret_set_reinjection.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.turret_query_predictor.restype = C.c_int
        L.turret_query_predictor.argtypes = [vp, C.POINTER(PredictorStats)]
        L.mlp_build_samples.restype = C.c_int
        L.mlp_build_samples.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
        for name in ("turret_save", "turret_load"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [vp, C.c_char_p]
        L.turret_time_collide.restype = C.c_int
        L.turret_time_collide.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_float)]
        _lib = L
    return _lib


def _arr(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _aligned_workspace(torch, nbytes, device):
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


def ibm_spread(X, h, dS, shape, stream=None):
    """S[h](x) = sum_k h_k W(x - X_k) dS_k on a (nz, ny, nx) grid (Sec. 2.2, step l = 1).

    X, h: float32 CUDA tensors (3, n); dS: (n,); returns a (3, nz, ny, nx) tensor."""
    import torch
    L = lib()
    nz, ny, nx = shape
    n = X.shape[1]
    dev = X.device
    out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=dev)
    nb = L.ibm_spread_workspace_bytes(nx, ny, nz, n)
    if nb == 0:
        raise TurretError(1, "invalid spread sizes")
    ws, ptr = _aligned_workspace(torch, nb, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = L.ibm_spread(C.c_void_p(X.data_ptr()), C.c_void_p(h.data_ptr()), C.c_void_p(dS.data_ptr()), n, nx, ny, nz,
                      C.c_void_p(out.data_ptr()), C.c_void_p(ptr), C.c_size_t(nb), C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise TurretError(rc, "ibm_spread failed")
    return out


class Turret:
    """One simulation window (+ optional particle) on one GPU.

    bc codes: PERIODIC, NOSLIP (halfway bounce-back), PRESSURE (top only)."""

    def __init__(self, nx, ny, nz, nu, kappa=1.0, g=(0.0, 0.0, 0.0), bc_x=PERIODIC, bc_y=PERIODIC,
                 bc_bottom=PERIODIC, bc_top=PERIODIC, sponge=0, slide=0, anchor_frac=0.25, storage="f32",
                 flags=None, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.shape = (nz, ny, nx)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._L = lib()
        self.win = Window(nx, ny, nz, bc_x, bc_y, bc_bottom, bc_top, sponge, slide, 0, float(anchor_frac))
        st = STORAGE[storage]
        self.storage = storage
        nb = self._L.lbm_workspace_bytes(C.byref(self.win), st)
        if nb == 0:
            raise TurretError(1, "invalid window")
        self._ws, ptr = _aligned_workspace(torch, nb, self.device)
        self._ibm_ws = None
        g3 = (C.c_double * 3)(*g)
        ctx = C.c_void_p()
        rc = self._L.lbm_init(C.byref(ctx), C.byref(self.win), 27, float(nu), float(kappa), g3, st,
                              C.c_void_p(ptr), C.c_size_t(nb), C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise TurretError(rc, self._L.turret_last_error(None).decode())
        self.ctx = ctx
        if flags:
            f = Flags(0, 0, 0, 0, 4, 0, 0, 0, 0, 0)
            for k, v in flags.items():
                setattr(f, k, int(v))
            self._check(self._L.lbm_set_flags(self.ctx, C.byref(f)))

    def _check(self, rc):
        if rc != 0:
            raise TurretError(rc, self._L.turret_last_error(self.ctx).decode())

    def set_wall_velocity(self, u_bottom=(0.0, 0.0, 0.0), u_top=(0.0, 0.0, 0.0)):
        """Velocities of moving bottom / top walls (window bc 3), in their plane."""
        ub = (C.c_double * 3)(*u_bottom)
        ut = (C.c_double * 3)(*u_top)
        self._check(self._L.lbm_set_wall_velocity(self.ctx, ub, ut))

    def set_fields(self, rho=None, u=None):
        rp = _arr(rho).ctypes.data_as(_dp) if rho is not None else None
        ua = _arr(u) if u is not None else None
        up = ua.ctypes.data_as(_dp) if ua is not None else None
        self._check(self._L.lbm_set_fields(self.ctx, rp, up))

    def load_surface(self, verts, tris, r0, v0=(0, 0, 0), w0=(0, 0, 0)):
        V = _arr(verts)
        T = _arr(tris, np.int32)
        vp, tp = V.ctypes.data_as(_dp), T.ctypes.data_as(C.POINTER(C.c_int32))
        nb = self._L.ibm_workspace_bytes(self.ctx, vp, V.shape[0], tp, T.shape[0])
        if nb == 0:
            raise TurretError(1, "invalid surface mesh")
        self._ibm_ws, ptr = _aligned_workspace(self.torch, nb, self.device)
        r0 = (C.c_double * 3)(*r0)
        v0 = (C.c_double * 3)(*v0)
        w0 = (C.c_double * 3)(*w0)
        self._check(self._L.ibm_load_surface(self.ctx, vp, V.shape[0], tp, T.shape[0], r0, v0, w0,
                                             C.c_void_p(ptr), C.c_size_t(nb)))

    def step(self, n=1):
        self._check(self._L.step(self.ctx, int(n)))

    def fluid_step(self, n=1):
        self._check(self._L.lbm_fluid_step(self.ctx, int(n)))

    def state(self, check=True):
        s = ParticleState()
        rc = self._L.query_particle_state(self.ctx, C.byref(s))
        if check:
            self._check(rc)
        return dict(r=np.array(s.r), d=np.array(s.d).reshape(3, 3), v=np.array(s.v), w=np.array(s.w),
                    F=np.array(s.F), T=np.array(s.T), L=np.array(s.L), origin=np.array(s.origin),
                    step=int(s.step), status=int(s.status), n_markers=int(s.n_markers), volume=s.volume,
                    area=s.area, kernels_per_step=int(s.kernels_per_step), Fp=np.array(s.Fp), rc=rc)

    def macro(self):
        """(4, nz, ny, nx) float32 tensor: rho, u_x, u_y, u_z of f(t)."""
        out = self.torch.empty((4,) + self.shape, dtype=self.torch.float32, device=self.device)
        self._check(self._L.lbm_copy_macro(self.ctx, C.c_void_p(out.data_ptr())))
        return out

    def populations(self):
        """(27, nz, ny, nx) float32 tensor: deviations f_i(t) - w_i."""
        out = self.torch.empty((27,) + self.shape, dtype=self.torch.float32, device=self.device)
        self._check(self._L.lbm_copy_populations(self.ctx, C.c_void_p(out.data_ptr())))
        return out

    def save(self, path):
        """Checkpoint of the current time level (see turret_save)."""
        self._check(self._L.turret_save(self.ctx, os.fsencode(path)))

    def load(self, path):
        """Restore a checkpoint into this identically configured context."""
        self._check(self._L.turret_load(self.ctx, os.fsencode(path)))

    def time_collide(self, threads, tx, minb, reps=20):
        """Mean microseconds of one collide+stream launch with the given launch
        shape (the context's state is left unchanged)."""
        us = C.c_float()
        self._check(self._L.turret_time_collide(self.ctx, int(threads), int(tx), int(minb), int(reps), C.byref(us)))
        return float(us.value)

    PREDICTORS = {"paper": 0, "linear": 1, "mlp": 2}
    LOG_REC = 32

    def set_predictor(self, mode="paper", net=None, warm=False, velocity=True, slip_eps=1e-4, resid_theta=0.5,
                      relative=False):
        """Force/torque predictor: 'paper' (the method as published), 'linear'
        or 'mlp' (with the MLP object `net`); warm: warm-started adaptive IBM
        cycles; velocity: marker velocities at t + 1; relative: resid_theta is
        a ratio to linear extrapolation's running error.  See turret_set_predictor."""
        self._net = net
        opts = (1 if warm else 0) | (2 if velocity else 0) | (4 if relative else 0)
        self._check(self._L.turret_set_predictor(self.ctx, self.PREDICTORS[mode], net.m if net is not None else None,
                                                 opts, float(slip_eps), float(resid_theta)))

    def set_reinjection(self, trigger, target, below, above):
        """The re-injection copy of Sec. 2.5 (see turret_set_reinjection); trigger 0 = off."""
        self._check(self._L.turret_set_reinjection(self.ctx, int(trigger), int(target), int(below), int(above)))

    def set_log(self, capacity):
        """Attach a device trajectory log of `capacity` records (0 detaches)."""
        if capacity > 0:
            self._log = self.torch.zeros((int(capacity), self.LOG_REC), dtype=self.torch.float64, device=self.device)
            self._check(self._L.turret_set_log(self.ctx, C.c_void_p(self._log.data_ptr()), int(capacity)))
        else:
            self._check(self._L.turret_set_log(self.ctx, None, 0))
            self._log = None

    def log_records(self):
        """The logged records in time order (float64 CUDA tensor [n][32])."""
        n = self.predictor_stats()["logged"]
        cap = self._log.shape[0]
        if n <= cap:
            return self._log[:n].clone()
        k = n % cap
        return self.torch.cat([self._log[k:], self._log[:k]]).clone()

    def predictor_stats(self):
        s = PredictorStats()
        self._check(self._L.turret_query_predictor(self.ctx, C.byref(s)))
        return dict(steps=int(s.steps), net_steps=int(s.net_steps), fallbacks=int(s.fallbacks),
                    cycles=int(s.cycles), logged=int(s.logged), resid=float(s.resid), slip=list(s.slip),
                    hist_n=int(s.hist_n), fallback=int(s.fallback))

    @property
    def cells(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def close(self):
        if getattr(self, "ctx", None) is not None:
            self._L.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent runs (Turret objects with a loaded surface) advanced together:
    one launch per phase of the step for all runs, one CUDA graph per step.
    Every run evolves bit for bit as it would alone."""

    def __init__(self, turrets, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.runs = list(turrets)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._L = lib()
        n = len(self.runs)
        nb = self._L.turret_batch_workspace_bytes(n)
        if nb == 0:
            raise TurretError(1, "empty batch")
        self._ws, ptr = _aligned_workspace(torch, nb, self.device)
        arr = (C.c_void_p * n)(*[t.ctx.value for t in self.runs])
        b = C.c_void_p()
        rc = self._L.turret_batch_init(C.byref(b), arr, n, C.c_void_p(ptr), C.c_size_t(nb),
                                       C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise TurretError(rc, self._L.turret_batch_last_error(None).decode())
        self.b = b
        self.tiles = (128, 2, [32] * n)

    def _check(self, rc):
        if rc != 0:
            raise TurretError(rc, self._L.turret_batch_last_error(self.b).decode())

    def set_tiles(self, threads, minb, tx):
        if len(tx) != len(self.runs):
            raise ValueError("one tile width per run")
        arr = (C.c_int32 * len(self.runs))(*[int(t) for t in tx])
        self._check(self._L.turret_batch_set_tiles(self.b, int(threads), int(minb), arr))
        self.tiles = (int(threads), int(minb), [int(t) for t in tx])

    def autotune(self, cache_path=None, reps=20, candidates=None):
        """Choose the collide+stream launch shape by timing candidates on one
        run per (nx, storage) class; timings are cached in a JSON file."""
        from . import autotune as AT
        choice = AT.tune([AT.RunInfo(t.shape[2], t.storage, t.cells, t) for t in self.runs],
                         timer=lambda t, th, tx, mb: t.time_collide(th, tx, mb, reps),
                         cache_path=cache_path, device_name=self.torch.cuda.get_device_name(self.device),
                         candidates=candidates)
        self.set_tiles(choice.threads, choice.minb, choice.tx)
        return choice

    def step(self, n=1):
        self._check(self._L.turret_batch_step(self.b, int(n)))

    def close(self):
        if getattr(self, "b", None) is not None:
            self._L.turret_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_IN, MLP_OUT, MLP_NPARAM = 34, 6, 38278


class MLP:
    """The force/torque surrogate network (34 -> 3 x 128 GELU -> 6) on the GPU.

    precision "bf16": tensor-core matrix products with BF16 operands and FP32
    accumulation; "fp32": FP32 throughout (check mode)."""

    def __init__(self, params, batch_cap=4096, precision="bf16", device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._L = lib()
        self.cap = int(batch_cap)
        nb = self._L.mlp_workspace_bytes(self.cap)
        if nb == 0:
            raise TurretError(1, "invalid batch capacity")
        self._ws, ptr = _aligned_workspace(torch, nb, self.device)
        p = _arr(params, np.float32)
        m = C.c_void_p()
        rc = self._L.mlp_init(C.byref(m), self.cap, {"bf16": 0, "fp32": 1}[precision], p.ctypes.data_as(_fp),
                              C.c_void_p(ptr), C.c_size_t(nb), C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise TurretError(rc, self._L.mlp_last_error(None).decode())
        self.m = m
        self.precision = precision

    def _check(self, rc):
        if rc != 0:
            raise TurretError(rc, self._L.mlp_last_error(self.m).decode())

    def _dev(self, a, shape):
        t = a if isinstance(a, self.torch.Tensor) else self.torch.as_tensor(np.asarray(a, dtype=np.float32))
        t = t.to(device=self.device, dtype=self.torch.float32).contiguous()
        assert tuple(t.shape) == shape, (t.shape, shape)
        return t

    def set_params(self, params):
        p = _arr(params, np.float32)
        self._check(self._L.mlp_set_params(self.m, p.ctypes.data_as(_fp)))

    def params(self):
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(self._L.mlp_get_params(self.m, p.ctypes.data_as(_fp)))
        return p

    def set_norm(self, mean_x, std_x, mean_y, std_y):
        a = [_arr(v, np.float32) for v in (mean_x, std_x, mean_y, std_y)]
        self._check(self._L.mlp_set_norm(self.m, *[v.ctypes.data_as(_fp) for v in a]))
        self.norm = tuple(np.array(v) for v in a)

    def _run(self, fn, x):
        n = x.shape[0]
        xt = self._dev(x, (n, MLP_IN))
        y = self.torch.empty((n, MLP_OUT), dtype=self.torch.float32, device=self.device)
        self.torch.cuda.current_stream(self.device).synchronize()
        self._check(fn(self.m, C.c_void_p(xt.data_ptr()), n, C.c_void_p(y.data_ptr())))
        self.stream.synchronize()
        return y

    def forward(self, x):
        """Outputs [n][6] of rows x [n][34] through the training kernels."""
        return self._run(self._L.mlp_forward, x)

    def infer(self, x):
        """Outputs [n][6] through the fused inference kernel of the predictor."""
        return self._run(self._L.mlp_infer, x)

    def loss_grad(self, x, y):
        n = x.shape[0]
        xt, yt = self._dev(x, (n, MLP_IN)), self._dev(y, (n, MLP_OUT))
        g = self.torch.empty(MLP_NPARAM, dtype=self.torch.float32, device=self.device)
        L = C.c_float()
        self.torch.cuda.current_stream(self.device).synchronize()
        self._check(self._L.mlp_loss_grad(self.m, C.c_void_p(xt.data_ptr()), C.c_void_p(yt.data_ptr()), n,
                                          C.byref(L), C.c_void_p(g.data_ptr())))
        return float(L.value), g

    def train_step(self, x, y, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, want_loss=True):
        """One AdamW step; x, y float32 CUDA tensors [n][34], [n][6] (n <= batch_cap)."""
        n = x.shape[0]
        opt = AdamW(lr, beta1, beta2, eps, weight_decay)
        L = C.c_float()
        self._check(self._L.mlp_train_step(self.m, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), n,
                                           C.byref(opt), C.byref(L) if want_loss else None))
        return float(L.value) if want_loss else None

    def close(self):
        if getattr(self, "m", None) is not None:
            self._L.mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_samples(records):
    """Training pairs (x [n-4][34], y [n-4][6]) from consecutive trajectory
    records (float64 CUDA tensor [n][32]), built on the GPU."""
    import torch
    n = records.shape[0]
    if n < 5:
        raise TurretError(1, "at least five records are needed")
    dev = records.device
    x = torch.empty((n - 4, MLP_IN), dtype=torch.float32, device=dev)
    y = torch.empty((n - 4, MLP_OUT), dtype=torch.float32, device=dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    rc = lib().mlp_build_samples(C.c_void_p(records.contiguous().data_ptr()), n, C.c_void_p(x.data_ptr()),
                                 C.c_void_p(y.data_ptr()), C.c_void_p(bad.data_ptr()), C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise TurretError(rc, "mlp_build_samples failed")
    if int(bad.item()) != 0:
        raise TurretError(1, "%d samples span non-consecutive time levels" % int(bad.item()))
    return x, y
