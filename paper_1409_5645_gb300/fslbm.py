"""Python binding of the C interface in ``include/fslbm.h`` (argument
marshalling only; every step of the method runs in the CUDA library).

Arrays may be host NumPy arrays or CUDA ``torch.Tensor`` objects; device
tensors are passed to the library as device pointers on the tensor's GPU,
so no host round trip is made.  There is no fallback: if the CUDA library is
not built or cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# FSLBM_CHECKED=1: the bounds-checked variant of the library (build.build(checked=True))
LIB_PATH = os.path.join(_PKG, "_build", *(["checked"] if os.environ.get("FSLBM_CHECKED") == "1" else []),
                        "libfslbm.so")

FSK, FSL = 0, 1
F64, F32, F16 = 0, 1, 2
HOST, DEVICE = 0, 1
FIELD_FLAGS, FIELD_F, FIELD_MASS, FIELD_PHI, FIELD_RHO, FIELD_U = 1, 2, 4, 8, 16, 32
PRECISIONS = {"f64": F64, "f32": F32, "f16": F16}
LOADS = {"plain": 0, "async": 1, "tma": 2, "pairs": 3}  # fslbm_loads
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_STATE", -5: "ERR_UNSTABLE",
          -6: "ERR_OVERFLOW", -7: "ERR_TIMEOUT", -8: "ERR_TOO_LARGE"}


class FslbmError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("tau", C.c_double), ("magic", C.c_double), ("g", C.c_double * 3),
                ("rho_G", C.c_double), ("sigma", C.c_double), ("rule", C.c_int), ("compressible", C.c_int),
                ("linear_eq", C.c_int), ("eps", C.c_double), ("periodic", C.c_int * 3), ("zshift", C.c_int),
                ("freeze", C.c_int), ("cleanup", C.c_int), ("keep_f0", C.c_int), ("delta_min", C.c_double),
                ("stress", C.c_int), ("shear_b", C.c_double * 6), ("wall_u", C.c_double * 3),
                ("ub_extrap", C.c_int), ("recon_nc", C.c_int), ("excess_split", C.c_int),
                ("bulk_loads", C.c_int), ("precision", C.c_int),
                ("stream", C.c_void_p), ("elvira", C.c_int), ("adjoint_fp32", C.c_int),
                ("u_max", C.c_double)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libfslbm.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            vp, ip, dp, u8p = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p
            L.fslbm_default_params.argtypes = [C.POINTER(Params)]
            L.fslbm_default_params.restype = None
            L.fslbm_create.argtypes = [C.POINTER(C.c_int), C.c_double, dp, C.c_double, C.c_double, ip,
                                       C.POINTER(vp)]
            L.fslbm_create_ex.argtypes = [C.POINTER(Params), C.POINTER(vp)]
            L.fslbm_tau_of_viscosity.argtypes = [C.c_double, dp]
            L.fslbm_fp64_rate.argtypes = [dp, vp]
            box = C.POINTER(C.c_int)
            L.fslbm_set_owned.argtypes = [vp, box, box]
            L.fslbm_halo_bytes.argtypes = [vp, box, box]
            L.fslbm_halo_bytes.restype = C.c_longlong
            L.fslbm_halo_pack.argtypes = [vp, box, box, vp]
            L.fslbm_halo_unpack.argtypes = [vp, box, box, vp]
            L.fslbm_set_state.argtypes = [vp, u8p, vp, vp, vp, ip]
            L.fslbm_init_equilibrium.argtypes = [vp, u8p, vp, vp, vp, vp, vp, ip]
            L.fslbm_set_state_post.argtypes = [vp, u8p, vp, vp, vp, vp, ip]
            L.fslbm_step.argtypes = [vp, ip]
            L.fslbm_sync.argtypes = [vp]
            L.fslbm_get_fields.argtypes = [vp, C.c_uint, C.POINTER(vp), ip]
            L.fslbm_total_mass.argtypes = [vp, dp, dp]
            L.fslbm_step_mass.argtypes = [vp, dp]
            L.fslbm_counters.argtypes = [vp, C.POINTER(C.c_longlong)]
            L.fslbm_timing.argtypes = [vp, ip]
            L.fslbm_timing_read.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
            L.fslbm_adjoint_forward.argtypes = [vp, ip, ip, ip, dp]
            L.fslbm_adjoint_backward.argtypes = [vp, dp, dp, C.c_void_p, ip]
            L.fslbm_adjoint_stats.argtypes = [vp, dp, dp, C.POINTER(C.c_size_t)]
            L.fslbm_time.argtypes = [vp]
            L.fslbm_time.restype = C.c_longlong
            L.fslbm_bulk_loads.argtypes = [vp]
            L.fslbm_bulk_loads.restype = C.c_int
            L.fslbm_set_overlap.argtypes = [vp, C.c_int]
            L.fslbm_set_overlap.restype = C.c_int
            L.fslbm_launches_per_step.argtypes = [vp]
            L.fslbm_launches_per_step.restype = C.c_int
            L.fslbm_check_grid_barrier.argtypes = [ip, vp]
            L.fslbm_check_grid_barrier.restype = C.c_int
            L.fslbm_build_info.argtypes = []
            L.fslbm_build_info.restype = C.c_int
            L.fslbm_device_bytes.argtypes = [vp]
            L.fslbm_device_bytes.restype = C.c_size_t
            L.fslbm_last_error.argtypes = [vp]
            L.fslbm_last_error.restype = C.c_char_p
            L.fslbm_destroy.argtypes = [vp]
            L.fslbm_destroy.restype = None
            _lib = L
    return _lib


def tau_of_viscosity(nu: float) -> float:
    """Relaxation time tau of the kinematic viscosity nu (the library's
    map of Sec. 2.1)."""
    tau = C.c_double()
    rc = lib().fslbm_tau_of_viscosity(float(nu), C.byref(tau))
    if rc:
        raise FslbmError(rc, f"viscosity {nu}")
    return tau.value


def fp64_rate(stream=None) -> float:
    """The current device's FP64 arithmetic rate, TFLOP/s (measured)."""
    t = C.c_double()
    rc = lib().fslbm_fp64_rate(C.byref(t), stream)
    if rc:
        raise FslbmError(rc, "fp64 rate")
    return t.value


def check_grid_barrier(expire: bool, stream=None) -> str:
    """Self-check of the conversion kernel's grid barrier (one cooperative
    launch): 'ok' when it completed, 'timeout' when its bounded wait ran out
    (expire=True makes it wait for a block that does not exist)."""
    rc = lib().fslbm_check_grid_barrier(1 if expire else 0, stream)
    if rc == 0:
        return "ok"
    if rc == -7:
        return "timeout"
    raise FslbmError(rc, "grid barrier self-check")


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


class _Arg:
    """Keeps the buffers alive and yields (pointer, where)."""

    def __init__(self):
        self.keep = []
        self.where = None

    def __call__(self, a, dtype):
        if a is None:
            return None
        if _is_torch_cuda(a):
            import torch
            tdt = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
            t = a.contiguous()
            if t.dtype != tdt:
                raise TypeError(f"expected {tdt}, got {t.dtype}")
            self._where(DEVICE)
            self.keep.append(t)
            return C.c_void_p(t.data_ptr())
        arr = np.ascontiguousarray(a, dtype=dtype)
        self._where(HOST)
        self.keep.append(arr)
        return C.c_void_p(arr.ctypes.data)

    def _where(self, w):
        if self.where is None:
            self.where = w
        elif self.where != w:
            raise ValueError("mixing host arrays and device tensors in one call")


def params_struct(dims, params: dict, precision=F64, stream=None) -> Params:
    P = Params()
    lib().fslbm_default_params(C.byref(P))
    for a in range(3):
        P.dims[a] = int(dims[a])
    P.tau = params.get("tau", P.tau)
    P.magic = params.get("magic", P.magic)
    g = params.get("g", (0.0, 0.0, 0.0))
    per = params.get("periodic", (0, 0, 0))
    for a in range(3):
        P.g[a] = g[a]
        P.periodic[a] = int(per[a])
    P.rho_G = params.get("rho_G", P.rho_G)
    P.sigma = params.get("sigma", P.sigma)
    P.rule = int(params.get("rule", P.rule))
    P.compressible = int(params.get("compressible", 0))
    P.linear_eq = int(params.get("linear_eq", 0))
    P.eps = params.get("eps", P.eps)
    P.zshift = int(params.get("zshift", 0))
    P.freeze = int(params.get("freeze", 0))
    P.cleanup = int(params.get("cleanup", P.cleanup))
    P.keep_f0 = int(params.get("keep_f0", 0))
    P.delta_min = params.get("delta_min", P.delta_min)
    P.stress = int(params.get("stress", 0))
    for k, val in enumerate(params.get("shear_b", (0.0,) * 6)):
        P.shear_b[k] = float(val)
    for k, val in enumerate(params.get("wall_u", (0.0,) * 3)):
        P.wall_u[k] = float(val)
    P.ub_extrap = int(params.get("ub_extrap", 0))
    P.recon_nc = int(params.get("recon_nc", 0))
    P.excess_split = int(params.get("excess_split", 0))
    P.bulk_loads = LOADS[params.get("bulk_loads", "plain")]
    P.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    P.stream = stream
    P.elvira = int(params.get("elvira", 0))
    P.adjoint_fp32 = int(params.get("adjoint_fp32", 0))
    P.u_max = float(params.get("u_max", 0.4))
    return P


class Lattice:
    """One lattice on the current CUDA device (a handle of the C library)."""

    def __init__(self, dims, params: dict, precision="f64", stream=None):
        self.L = lib()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        self.params = dict(params)
        self.precision = precision
        self._P = params_struct(self.dims, self.params, precision, stream)
        h = C.c_void_p()
        rc = self.L.fslbm_create_ex(C.byref(self._P), C.byref(h))
        if rc != 0:
            raise FslbmError(rc, "fslbm_create_ex")
        self.h = h

    @classmethod
    def create(cls, dims, tau, g, rho_G=1.0, sigma=0.0, rule=FSL):
        """A lattice from the paper's problem data alone (fslbm_create): every
        other parameter at the library's default."""
        self = cls.__new__(cls)
        self.L = lib()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        self.params = dict(tau=tau, g=tuple(g), rho_G=rho_G, sigma=sigma, rule=rule)
        self.precision = "f64"
        d = (C.c_int * 3)(*self.dims)
        gv = (C.c_double * 3)(*[float(v) for v in g])
        h = C.c_void_p()
        rc = self.L.fslbm_create(d, float(tau), gv, float(rho_G), float(sigma), int(rule), C.byref(h))
        if rc != 0:
            raise FslbmError(rc, "fslbm_create")
        self.h = h
        return self

    @classmethod
    def from_case(cls, case, precision="f64", stream=None, **override):
        p = dict(case["params"])
        p.update(override)
        lat = cls(case["dims"], p, precision, stream)
        lat.init_equilibrium(case["flags"], case["rho"], case["u"], case["phi"], case.get("noise"),
                             case.get("wall_delta"))
        return lat

    def _check(self, rc, what):
        if rc != 0:
            raise FslbmError(rc, f"{what}: {self.L.fslbm_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.L.fslbm_destroy(self.h)
            self.h = None

    __del__ = close

    def init_equilibrium(self, flags, rho, u, phi, noise=None, wall_delta=None):
        A = _Arg()
        args = (A(flags, np.uint8), A(rho, np.float64), A(u, np.float64), A(phi, np.float64),
                A(noise, np.float64), A(wall_delta, np.float64))
        self._check(self.L.fslbm_init_equilibrium(self.h, *args, A.where), "init_equilibrium")

    def set_state(self, flags, f, phi, wall_delta=None):
        A = _Arg()
        args = (A(flags, np.uint8), A(f, np.float64), A(phi, np.float64), A(wall_delta, np.float64))
        self._check(self.L.fslbm_set_state(self.h, *args, A.where), "set_state")

    def set_state_post(self, flags, f_post, m, phi, wall_delta=None):
        A = _Arg()
        args = (A(flags, np.uint8), A(f_post, np.float64), A(m, np.float64), A(phi, np.float64),
                A(wall_delta, np.float64))
        self._check(self.L.fslbm_set_state_post(self.h, *args, A.where), "set_state_post")

    def step(self, n: int = 1):
        self._check(self.L.fslbm_step(self.h, int(n)), "step")

    def sync(self):
        self._check(self.L.fslbm_sync(self.h), "sync")

    def get(self, mask: int = 63, device=None) -> dict:
        """Fields as NumPy arrays (or CUDA tensors when ``device`` is given)."""
        N = self.N
        spec = [(FIELD_FLAGS, "flags", (N,), np.uint8), (FIELD_F, "f", (19, N), np.float64),
                (FIELD_MASS, "m", (N,), np.float64), (FIELD_PHI, "phi", (N,), np.float64),
                (FIELD_RHO, "rho", (N,), np.float64), (FIELD_U, "u", (N, 3), np.float64)]
        out, ptrs = {}, []
        for bit, name, shape, dt in spec:
            if not mask & bit:
                continue
            if device is not None:
                import torch
                t = torch.empty(shape, dtype=torch.uint8 if dt == np.uint8 else torch.float64, device=device)
                out[name] = t
                ptrs.append(t.data_ptr())
            else:
                a = np.empty(shape, dtype=dt)
                out[name] = a
                ptrs.append(a.ctypes.data)
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        self._check(self.L.fslbm_get_fields(self.h, mask, arr, DEVICE if device is not None else HOST), "get_fields")
        return out

    def get_into(self, mask: int, out: dict):
        """Fields into caller-owned host arrays (``out`` keyed like get())."""
        names = [(FIELD_FLAGS, "flags"), (FIELD_F, "f"), (FIELD_MASS, "m"), (FIELD_PHI, "phi"), (FIELD_RHO, "rho"),
                 (FIELD_U, "u")]
        ptrs = [out[n].ctypes.data for bit, n in names if mask & bit]
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        self._check(self.L.fslbm_get_fields(self.h, mask, arr, HOST), "get_fields")

    def total_mass(self):
        M, L = C.c_double(), C.c_double()
        self._check(self.L.fslbm_total_mass(self.h, C.byref(M), C.byref(L)), "total_mass")
        return M.value, L.value

    def step_mass(self) -> float:
        M = C.c_double()
        self._check(self.L.fslbm_step_mass(self.h, C.byref(M)), "step_mass")
        return M.value

    def counters(self):
        c = (C.c_longlong * 5)()
        self._check(self.L.fslbm_counters(self.h, c), "counters")
        return list(c)

    def timing(self, on: bool = True):
        self._check(self.L.fslbm_timing(self.h, 1 if on else 0), "timing")

    def timing_read(self):
        """Average ms per step of (bulk, interface, reduction, conversions)."""
        ms = (C.c_double * 4)()
        n = C.c_longlong()
        self._check(self.L.fslbm_timing_read(self.h, ms, C.byref(n)), "timing_read")
        return list(ms), n.value

    # -- slab decomposition ---------------------------------------------------
    @staticmethod
    def _box(lo, hi):
        return (C.c_int * 3)(*[int(v) for v in lo]), (C.c_int * 3)(*[int(v) for v in hi])

    def set_owned(self, lo, hi):
        """Cells of [lo, hi) are this handle's own (mass balance, lost ledger)."""
        self._check(self.L.fslbm_set_owned(self.h, *self._box(lo, hi)), "set_owned")

    def halo_bytes(self, lo, hi) -> int:
        n = int(self.L.fslbm_halo_bytes(self.h, *self._box(lo, hi)))
        if n < 0:
            raise FslbmError(n, "halo_bytes")
        return n

    def halo_pack(self, lo, hi, buf):
        """Pack the box's state into ``buf`` (a CUDA uint8 tensor of
        halo_bytes(lo, hi)); asynchronous on the handle's stream."""
        self._check(self.L.fslbm_halo_pack(self.h, *self._box(lo, hi), C.c_void_p(buf.data_ptr())), "halo_pack")

    def halo_unpack(self, lo, hi, buf):
        self._check(self.L.fslbm_halo_unpack(self.h, *self._box(lo, hi), C.c_void_p(buf.data_ptr())), "halo_unpack")

    # -- differentiation ------------------------------------------------------
    def adjoint_forward(self, nsteps: int, K: int = 200, objective: int = 0) -> float:
        J = C.c_double()
        self._check(self.L.fslbm_adjoint_forward(self.h, int(nsteps), int(K), int(objective), C.byref(J)),
                    "adjoint_forward")
        return J.value

    def adjoint_backward(self, device=None):
        """(dJ/dnu, dJ/dg[3], dJ/dphi0[N]) as NumPy (or a CUDA tensor for phi0)."""
        dnu = C.c_double()
        dg = (C.c_double * 3)()
        if device is not None:
            import torch
            dphi = torch.empty(self.N, dtype=torch.float64, device=device)
            ptr, where = C.c_void_p(dphi.data_ptr()), DEVICE
        else:
            dphi = np.empty(self.N, dtype=np.float64)
            ptr, where = C.c_void_p(dphi.ctypes.data), HOST
        self._check(self.L.fslbm_adjoint_backward(self.h, C.byref(dnu), dg, ptr, where), "adjoint_backward")
        return dnu.value, np.array(list(dg)), dphi

    def adjoint_stats(self):
        f, a, b = C.c_double(), C.c_double(), C.c_size_t()
        self._check(self.L.fslbm_adjoint_stats(self.h, C.byref(f), C.byref(a), C.byref(b)), "adjoint_stats")
        return f.value, a.value, b.value

    @property
    def time(self) -> int:
        return int(self.L.fslbm_time(self.h))

    @property
    def bulk_loads(self) -> str:
        """How the bulk kernel reaches its pulled values: 'async' (cp.async into
        shared memory), 'plain' (global loads), 'tma' (tensor-map row copies)
        or 'pairs' (two cells per lane)."""
        return {v: k for k, v in LOADS.items()}[self.L.fslbm_bulk_loads(self.h)]

    def set_overlap(self, on: bool):
        """Interface kernels on a second stream beside the bulk kernel (True,
        the default) or every kernel in order on the handle's stream."""
        self._check(self.L.fslbm_set_overlap(self.h, int(bool(on))), "set_overlap")

    @property
    def launches_per_step(self) -> int:
        """Kernel launches one time step makes on this lattice."""
        return int(self.L.fslbm_launches_per_step(self.h))

    @property
    def device_bytes(self) -> int:
        return int(self.L.fslbm_device_bytes(self.h))
