"""Python marshalling for the FP64 CPU oracle (``oracle/sisph_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain restatement of the SISPH
time step (arXiv 1908.01762, Algorithm 1) used by the tests to check the CUDA
library and by the benchmark's CPU-baseline leg.  The product path never
imports this package.  The pins live in ``tests/test_oracle_*.py``; the
oracle's C header lists which functions are pinned by invariants only.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sisph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sisph_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("periodic", C.c_int32 * 3),
        ("h", C.c_double), ("dt", C.c_double), ("rho0", C.c_double), ("nu", C.c_double),
        ("g", C.c_double * 3), ("alpha", C.c_double), ("c0", C.c_double),
        ("eta", C.c_double), ("omega", C.c_double), ("fs_ratio", C.c_double),
        ("min_iter", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
        ("pgrad_symm", C.c_int32), ("free_surface", C.c_int32), ("ustar_slip", C.c_int32),
        ("pref_mode", C.c_int32), ("p_ref", C.c_double), ("gtvf_hfac", C.c_double),
        ("gtvf_K", C.c_int32), ("residual_form", C.c_int32), ("brute_neighbors", C.c_int32),
        ("adaptive_dt", C.c_int32), ("ppe_solver", C.c_int32),
    ]


class Diag(C.Structure):
    _fields_ = [("iters", C.c_int32), ("residual", C.c_double), ("lambda_", C.c_double),
                ("converged", C.c_int32), ("nonfinite", C.c_int32), ("umax", C.c_double),
                ("dt", C.c_double)]


_libs = {}        # mistake number (0: none) -> loaded library
_active = 0       # the library lib() returns (a planted mistake, or 0)


def _declare(L):
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.or_default_params.argtypes = [C.POINTER(Params)]
    L.or_kernel_w.argtypes = [C.c_double, C.c_double, C.c_int32]
    L.or_kernel_w.restype = C.c_double
    L.or_kernel_dwdr.argtypes = [C.c_double, C.c_double, C.c_int32]
    L.or_kernel_dwdr.restype = C.c_double
    L.or_neighbors.argtypes = [C.POINTER(Params), C.c_int64, dp, dp, dp, ip, ip, C.c_int64]
    L.or_neighbors.restype = C.c_int64
    L.or_create.argtypes = [C.POINTER(Params), C.c_int64] + [dp] * 9 + [ip] + [dp] * 3
    L.or_create.restype = C.c_void_p
    L.or_destroy.argtypes = [C.c_void_p]
    L.or_get.argtypes = [C.c_void_p, C.c_char_p, dp]
    L.or_get.restype = C.c_int32
    L.or_set.argtypes = [C.c_void_p, C.c_char_p, dp]
    L.or_set.restype = C.c_int32
    L.or_build_neighbors.argtypes = [C.c_void_p]
    L.or_build_neighbors.restype = C.c_int64
    L.or_neighbor_list.argtypes = [C.c_void_p, ip, ip, C.c_int64]
    L.or_neighbor_list.restype = C.c_int64
    for fn in ("or_density", "or_wall_normals", "or_stage1", "or_ppe_setup",
               "or_pressure_gradient", "or_gtvf", "or_update"):
        getattr(L, fn).argtypes = [C.c_void_p]
    L.or_ghost_velocity.argtypes = [C.c_void_p, C.c_int32]
    L.or_ppe_iterate.argtypes = [C.c_void_p, C.POINTER(Diag)]
    L.or_ppe_apply.argtypes = [C.c_void_p, dp, dp]
    L.or_ppe_export.argtypes = [C.c_void_p, dp, dp, ip, dp, dp, dp, dp]
    L.or_ppe_export.restype = C.c_int64
    L.or_step.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Diag)]
    L.or_step.restype = C.c_int32
    L.or_ppe_solve.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.POINTER(Diag)]
    L.or_ppe_solve.restype = C.c_int32
    L.or_get_pref.argtypes = [C.c_void_p]
    L.or_get_pref.restype = C.c_double
    L.or_get_dt.argtypes = [C.c_void_p]
    L.or_get_dt.restype = C.c_double
    return L


def lib():
    """The oracle library in use: liboracle.so, or a mutant build while a
    test has planted a mistake (plant_mistake)."""
    if _active not in _libs:
        if _active == 0:
            path = build()
        else:
            from . import mutants
            path = mutants.build(_active)
        _libs[_active] = _declare(C.CDLL(path))
    return _libs[_active]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def kernel_w(r, h, dim):
    return lib().or_kernel_w(float(r), float(h), int(dim))


def kernel_dwdr(r, h, dim):
    return lib().or_kernel_dwdr(float(r), float(h), int(dim))


def plant_mistake(which: int):
    """Route the oracle calls that follow (module functions and Sims created
    from now on) to the mutant build with mistake `which` planted, to show
    that a pin catches it; 0 returns to the oracle itself.  The mutants are
    separate builds (oracle/mutants.py): the oracle's own source and library
    have a single arithmetic path."""
    global _active
    which = int(which)
    if which != 0:
        from . import mutants
        if which not in mutants.MUTANTS:
            raise KeyError(f"no planted mistake {which}")
    _active = which


def make_params(case, **over) -> Params:
    """Oracle parameters from a ``workloads`` case plus overrides."""
    P = Params()
    lib().or_default_params(C.byref(P))
    prm = dict(case["params"])
    prm.update(over)
    P.dim = case["dim"]
    for k in range(3):
        P.lo[k] = case["lo"][k]
        P.hi[k] = case["hi"][k]
        P.periodic[k] = case["periodic"][k]
        P.g[k] = prm["g"][k]
    for key in ("h", "dt", "rho0", "nu", "alpha", "c0", "tol", "p_ref", "gtvf_hfac"):
        setattr(P, key, float(prm[key]))
    for key in ("max_iter", "pgrad_symm", "free_surface", "ustar_slip", "pref_mode", "gtvf_K"):
        setattr(P, key, int(prm[key]))
    for key in ("eta", "omega", "fs_ratio"):
        if key in prm:
            setattr(P, key, float(prm[key]))
    for key in ("min_iter", "residual_form", "brute_neighbors", "adaptive_dt", "ppe_solver"):
        if key in prm:
            setattr(P, key, int(prm[key]))
    return P


def neighbors(case, x=None, y=None, z=None, brute=False):
    """Neighbour lists (counts, concatenated ascending indices) of a case."""
    P = make_params(case, brute_neighbors=int(brute))
    x = np.ascontiguousarray(case["x"] if x is None else x, np.float64)
    y = np.ascontiguousarray(case["y"] if y is None else y, np.float64)
    z = np.ascontiguousarray(case["z"] if z is None else z, np.float64)
    n = x.size
    counts = np.zeros(n, np.int32)
    cap = max(1024, n * 64)
    while True:
        idx = np.zeros(cap, np.int32)
        tot = lib().or_neighbors(C.byref(P), n, _dp(x), _dp(y), _dp(z), _ip(counts), _ip(idx), cap)
        if tot >= 0:
            return counts, idx[:tot].copy()
        if tot == -2:
            raise MemoryError("oracle neighbour search failed")
        cap *= 2


class Sim:
    """One oracle simulation (user order, FP64)."""

    def __init__(self, case, **over):
        self.case = case
        self.P = make_params(case, **over)
        c = case
        self.n = c["n"]
        self._keep = [np.ascontiguousarray(c[k], np.float64) for k in
                      ("x", "y", "z", "u", "v", "w", "m", "rho", "p", "wall_u", "wall_v", "wall_w")]
        kind = np.ascontiguousarray(c["kind"], np.int32)
        a = self._keep
        self._L = lib()
        self.h = self._L.or_create(C.byref(self.P), self.n, _dp(a[0]), _dp(a[1]), _dp(a[2]),
                                 _dp(a[3]), _dp(a[4]), _dp(a[5]), _dp(a[6]), _dp(a[7]),
                                 _dp(a[8]), _ip(kind), _dp(a[9]), _dp(a[10]), _dp(a[11]))
        if not self.h:
            raise MemoryError("or_create failed")

    def __del__(self):
        if getattr(self, "h", None):
            self._L.or_destroy(self.h)
            self.h = None

    def get(self, field):
        out = np.zeros(self.n)
        if self._L.or_get(self.h, field.encode(), _dp(out)) != 0:
            raise KeyError(field)
        return out

    def set(self, field, values):
        arr = np.ascontiguousarray(values, np.float64)
        if self._L.or_set(self.h, field.encode(), _dp(arr)) != 0:
            raise KeyError(field)

    def build_neighbors(self):
        if self._L.or_build_neighbors(self.h) < 0:
            raise MemoryError("neighbour search failed")

    def neighbor_list(self):
        counts = np.zeros(self.n, np.int32)
        cap = max(1024, self.n * 64)
        while True:
            idx = np.zeros(cap, np.int32)
            tot = self._L.or_neighbor_list(self.h, _ip(counts), _ip(idx), cap)
            if tot >= 0:
                return counts, idx[:tot].copy()
            cap *= 2

    def density(self):
        self._L.or_density(self.h)

    def wall_normals(self):
        self._L.or_wall_normals(self.h)

    def ghost_velocity(self, slip):
        self._L.or_ghost_velocity(self.h, int(slip))

    def stage1(self):
        self._L.or_stage1(self.h)

    def ppe_setup(self):
        self._L.or_ppe_setup(self.h)

    def ppe_iterate(self):
        d = Diag()
        self._L.or_ppe_iterate(self.h, C.byref(d))
        return d

    def ppe_apply(self, p):
        p = np.ascontiguousarray(p, np.float64)
        out = np.zeros(self.n)
        self._L.or_ppe_apply(self.h, _dp(p), _dp(out))
        return out

    def ppe_export(self):
        n = self.n
        counts, idx = self.neighbor_list()
        tot = idx.size
        diag = np.zeros(n); rhs = np.zeros(n); act = np.zeros(n, np.int32)
        fac = np.zeros(max(tot, 1)); ws = np.zeros(n); wh = np.zeros(n); ww = np.zeros(max(tot, 1))
        self._L.or_ppe_export(self.h, _dp(diag), _dp(rhs), _ip(act), _dp(fac), _dp(ws), _dp(wh), _dp(ww))
        return dict(counts=counts, idx=idx, diag=diag, rhs=rhs, active=act, fac=fac[:tot],
                    wall_s=ws, wall_h=wh)

    def pressure_gradient(self):
        self._L.or_pressure_gradient(self.h)

    def gtvf(self):
        self._L.or_gtvf(self.h)

    def update(self):
        self._L.or_update(self.h)

    def ppe_solve(self, tol, max_iter):
        d = Diag()
        rc = self._L.or_ppe_solve(self.h, float(tol), int(max_iter), C.byref(d))
        return rc, d

    def step(self, nsteps=1):
        ds = (Diag * max(1, nsteps))()
        rc = self._L.or_step(self.h, int(nsteps), ds)
        return rc, [ds[i] for i in range(nsteps)]

    @property
    def dt(self):
        """Time step of the next step."""
        return self._L.or_get_dt(self.h)

    @property
    def p_ref(self):
        return self._L.or_get_pref(self.h)
