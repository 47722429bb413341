"""ctypes wrapper of the FP64 CPU oracle (fslbm_oracle.cpp).

Test infrastructure only: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product library.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fslbm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liborc_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

F_PRE, F_POST, MASS, PHI, RHO, VEL = 0, 1, 2, 3, 4, 5


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction); ``omp=True`` builds
    the OpenMP variant of the same source (all-core CPU timing only)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if omp else _LIB_PATH
    stamp = os.path.join(_BUILD, "STAMP_omp" if omp else "STAMP")
    try:
        same_machine = open(stamp).read().strip() == platform.machine()
    except OSError:
        same_machine = False
    if (force or not same_machine or not os.path.exists(path)
            or os.path.getmtime(path) < os.path.getmtime(_SRC)):
        tmp = path + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC"]
                              + (["-fopenmp"] if omp else []) + [_SRC, "-o", tmp])
        os.replace(tmp, path)
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    return path


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("magic", C.c_double), ("g", C.c_double * 3),
                ("rho_G", C.c_double), ("sigma", C.c_double), ("rule", C.c_int),
                ("compressible", C.c_int), ("linear_eq", C.c_int), ("eps", C.c_double),
                ("periodic", C.c_int * 3), ("zshift", C.c_int), ("freeze", C.c_int),
                ("cleanup", C.c_int), ("delta_min", C.c_double), ("stress", C.c_int),
                ("shear_b", C.c_double * 6), ("wall_u", C.c_double * 3),
                ("ub_extrap", C.c_int), ("recon_nc", C.c_int),
                ("excess_split", C.c_int), ("elvira", C.c_int)]


def lib(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            L = C.CDLL(build(omp=omp))
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
            u8p = C.POINTER(C.c_uint8)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [C.POINTER(Params), ip]
            L.orc_destroy.argtypes = [vp]
            L.orc_init.argtypes = [vp, u8p, dp, dp, dp, dp, dp]
            L.orc_set_state.argtypes = [vp, u8p, dp, dp, dp]
            L.orc_step.argtypes = [vp, ip]
            L.orc_get.argtypes = [vp, ip, ip, dp]
            L.orc_get_flags.argtypes = [vp, u8p]
            L.orc_total_mass.restype = C.c_double
            L.orc_total_mass.argtypes = [vp, dp]
            L.orc_geometry.argtypes = [vp, dp, dp, dp, dp, u8p]
            L.orc_cube_volume.restype = C.c_double
            L.orc_cube_volume.argtypes = [dp, C.c_double]
            L.orc_plic_offset.restype = C.c_double
            L.orc_plic_offset.argtypes = [dp, C.c_double]
            L.orc_counters.argtypes = [vp, C.POINTER(C.c_long), C.POINTER(C.c_long)]
            L.orc_seed.argtypes = [vp, C.c_double, dp, dp]
            L.orc_step_from_post.argtypes = [vp, u8p, dp, dp, dp]
            L.orc_threads.restype = C.c_int
            L.orc_threads.argtypes = [ip]
            if omp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if omp else _lib


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build (n > 0 sets them); returns the count in use."""
    return int(lib(omp=True).orc_threads(int(n)))


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def make_params(dims, p) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = (int(v) for v in dims)
    P.tau = p["tau"]
    P.magic = p["magic"]
    for a in range(3):
        P.g[a] = p["g"][a]
        P.periodic[a] = int(p["periodic"][a])
    P.rho_G = p["rho_G"]
    P.sigma = p["sigma"]
    P.rule = int(p["rule"])
    P.compressible = int(p["compressible"])
    P.linear_eq = int(p["linear_eq"])
    P.eps = p["eps"]
    P.zshift = int(p["zshift"])
    P.freeze = int(p["freeze"])
    P.cleanup = int(p.get("cleanup", 3))
    P.delta_min = p["delta_min"]
    P.stress = int(p.get("stress", 0))
    for k, v in enumerate(p.get("shear_b", (0.0,) * 6)):
        P.shear_b[k] = float(v)
    for k, v in enumerate(p.get("wall_u", (0.0,) * 3)):
        P.wall_u[k] = float(v)
    P.ub_extrap = int(p.get("ub_extrap", 0))
    P.recon_nc = int(p.get("recon_nc", 0))
    P.excess_split = int(p.get("excess_split", 0))
    P.elvira = int(p.get("elvira", 0))
    return P


class Oracle:
    """One lattice in the oracle.  ``dual=True`` carries one tangent;
    ``omp=True`` runs it on the OpenMP build (same results)."""

    def __init__(self, dims, params, dual: bool = False, omp: bool = False):
        self.L = lib(omp)
        self.dims = tuple(int(v) for v in dims)
        self.N = int(np.prod(self.dims))
        self.params = dict(params)
        self._P = make_params(self.dims, self.params)
        self.h = self.L.orc_create(C.byref(self._P), 1 if dual else 0)
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.dual = dual

    @classmethod
    def from_case(cls, case, dual: bool = False, omp: bool = False, **override):
        p = dict(case["params"])
        p.update(override)
        o = cls(case["dims"], p, dual=dual, omp=omp)
        o.init(case)
        return o

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    def init(self, case):
        """Populations = equilibrium(rho, u) + noise; m = phi * rho."""
        flags = np.ascontiguousarray(case["flags"], dtype=np.uint8)
        rho, u, phi = _f64(case["rho"]), _f64(case["u"]), _f64(case["phi"])
        noise, wd = _f64(case.get("noise")), _f64(case.get("wall_delta"))
        self._keep = (flags, rho, u, phi, noise, wd)
        return self.L.orc_init(self.h, flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(rho), _dp(u),
                               _dp(phi), _dp(noise), _dp(wd))

    def set_state(self, flags, f, phi, wall_delta=None):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        f, phi, wd = _f64(f), _f64(phi), _f64(wall_delta)
        return self.L.orc_set_state(self.h, flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(f),
                                    _dp(phi), _dp(wd))

    def step(self, n: int = 1) -> int:
        return self.L.orc_step(self.h, int(n))

    def step_from_post(self, flags, f_post, m, phi) -> int:
        """One step from a post-collision state (FP64 handles)."""
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        f_post, m, phi = _f64(f_post), _f64(m), _f64(phi)
        self._keep_post = (flags, f_post, m, phi)
        return self.L.orc_step_from_post(self.h, flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(f_post),
                                         _dp(m), _dp(phi))

    def get(self, field: int, tangent: bool = False) -> np.ndarray:
        size = {F_PRE: 19 * self.N, F_POST: 19 * self.N, VEL: 3 * self.N}.get(field, self.N)
        out = np.empty(size, dtype=np.float64)
        rc = self.L.orc_get(self.h, field, 1 if tangent else 0, _dp(out))
        if rc != 0:
            raise ValueError(f"oracle get({field}) -> {rc}")
        if field in (F_PRE, F_POST):
            return out.reshape(19, self.N)
        if field == VEL:
            return out.reshape(self.N, 3)
        return out

    def flags(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.uint8)
        self.L.orc_get_flags(self.h, out.ctypes.data_as(C.POINTER(C.c_uint8)))
        return out

    def total_mass(self):
        lost = C.c_double()
        M = self.L.orc_total_mass(self.h, C.byref(lost))
        return M, lost.value

    def geometry(self):
        N = self.N
        n = np.empty(3 * N)
        d = np.empty(N)
        k = np.empty(N)
        dl = np.empty(19 * N)
        ok = np.empty(N, dtype=np.uint8)
        self.L.orc_geometry(self.h, _dp(n), _dp(d), _dp(k), _dp(dl), ok.ctypes.data_as(C.POINTER(C.c_uint8)))
        return n.reshape(N, 3), d, k, dl.reshape(19, N), ok

    def counters(self):
        c = (C.c_long * 4)()
        t = C.c_long()
        self.L.orc_counters(self.h, c, C.byref(t))
        return list(c), t.value

    def seed(self, dtau=0.0, dg=None, dphi=None):
        dg = _f64(dg)
        dphi = _f64(dphi)
        self._seed_keep = (dg, dphi)
        return self.L.orc_seed(self.h, float(dtau), _dp(dg), _dp(dphi))


def cube_volume(n, d) -> float:
    n = np.ascontiguousarray(n, dtype=np.float64)
    return lib().orc_cube_volume(_dp(n), float(d))


def plic_offset(n, phi) -> float:
    n = np.ascontiguousarray(n, dtype=np.float64)
    return lib().orc_plic_offset(_dp(n), float(phi))
