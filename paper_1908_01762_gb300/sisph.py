"""Thin ctypes binding of libsisph (include/sisph.h): argument marshalling only.

Every function named ``sisph_*`` here calls the C function of the same name.
All computation runs in the library's CUDA kernels; there is no fallback: if
``libsisph.so`` cannot be loaded the import of a function raises.  The
``Simulation`` class only converts between numpy arrays and the C-ABI.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsisph.so")
CHECKED_LIB_PATH = os.path.join(_PKG, "libsisph_checked.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ENONFINITE, ETIMEOUT, EINTERNAL, ECAPACITY = (
    -1, -2, -3, -4, -5, -6, -7, -8)
KIND_FLUID, KIND_WALL = 0, 1
FP64, MIXED = 0, 1
PREF_FIXED, PREF_TWICE_MAX_FIRST, PREF_EXTERNAL = 0, 1, 2
FIELDS = {"x": 0, "y": 1, "z": 2, "u": 3, "v": 4, "w": 5, "ut": 6, "vt": 7, "wt": 8, "p": 9,
          "rho": 10, "m": 11, "nx": 12, "ny": 13, "nz": 14, "rhs": 15, "diag": 16,
          "dx": 17, "dy": 18, "dz": 19, "nskin": 20, "ncount": 21}
_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
          ENOTCONVERGED: "ENOTCONVERGED", ENONFINITE: "ENONFINITE", ETIMEOUT: "ETIMEOUT",
          EINTERNAL: "EINTERNAL", ECAPACITY: "ECAPACITY"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class sisph_particles(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64),
                ("x", _dp), ("y", _dp), ("z", _dp), ("u", _dp), ("v", _dp), ("w", _dp),
                ("m", _dp), ("rho", _dp), ("p", _dp), ("kind", _ip),
                ("wall_u", _dp), ("wall_v", _dp), ("wall_w", _dp),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int32 * 3)]


class sisph_case_params(C.Structure):
    _fields_ = [("h", C.c_double), ("dt", C.c_double), ("rho0", C.c_double), ("nu", C.c_double),
                ("g", C.c_double * 3), ("alpha", C.c_double), ("c0", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("pgrad_symm", C.c_int32),
                ("free_surface", C.c_int32), ("ustar_slip", C.c_int32), ("pref_mode", C.c_int32),
                ("p_ref", C.c_double), ("gtvf_hfac", C.c_double), ("gtvf_K", C.c_int32),
                ("adaptive_dt", C.c_int32), ("ppe_solver", C.c_int32)]


class sisph_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("omega", C.c_double), ("min_iter", C.c_int32),
                ("eta", C.c_double), ("fs_ratio", C.c_double), ("residual_form", C.c_int32),
                ("nbr_capacity", C.c_int32), ("skin", C.c_double), ("block", C.c_int32),
                ("use_graph", C.c_int32),
                ("barrier_timeout_ms", C.c_double), ("debug_skip_barrier", C.c_int32),
                ("ppe_sync", C.c_int32),
                ("physics", sisph_case_params)]


class sisph_case_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("residual", C.c_double),
                ("lambda_", C.c_double), ("p_ref", C.c_double), ("total_iters", C.c_int64),
                ("solves", C.c_int64), ("rebuilds", C.c_int64), ("dt", C.c_double),
                ("time", C.c_double)]


_lib = None


def load_library(path: str = None):
    """Load libsisph.so -- libsisph_checked.so when the environment sets
    SISPH_CHECKED=1 -- (raises OSError if it is missing: no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = CHECKED_LIB_PATH if os.environ.get("SISPH_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"libsisph.so not built ({path}); run paper_1908_01762_gb300.build()")
    L = C.CDLL(path)
    h = C.c_void_p
    sig = {
        "sisph_default_options": (None, [C.POINTER(sisph_options)]),
        "sisph_default_case": (None, [C.POINTER(sisph_case_params)]),
        "sisph_create": (C.c_int, [C.POINTER(sisph_particles), C.c_double, C.c_double, C.c_double,
                                   C.c_double, _dp, C.POINTER(sisph_options), C.POINTER(h)]),
        "sisph_batch_create": (C.c_int, [C.c_int32, C.POINTER(sisph_particles),
                                         C.POINTER(sisph_case_params), C.POINTER(sisph_options),
                                         C.POINTER(h)]),
        "sisph_destroy": (None, [h]),
        "sisph_build_neighbors": (C.c_int, [h]),
        "sisph_neighbors": (C.c_int, [h, _ip, _ip, C.c_int64, C.POINTER(C.c_int64)]),
        "sisph_compute_density": (C.c_int, [h]),
        "sisph_ppe_solve": (C.c_int, [h, C.c_double, C.c_int32, _ip, _dp]),
        "sisph_step": (C.c_int, [h, C.c_int32]),
        "sisph_batch_step": (C.c_int, [h, C.c_int32, _ip]),
        "sisph_get": (C.c_int, [h, C.c_int32, _dp]),
        "sisph_set": (C.c_int, [h, C.c_int32, _dp]),
        "sisph_get_many": (C.c_int, [h, C.c_int32, _ip, C.POINTER(_dp)]),
        "sisph_set_many": (C.c_int, [h, C.c_int32, _ip, C.POINTER(_dp)]),
        "sisph_stats": (C.c_int, [h, C.POINTER(sisph_case_stats)]),
        "sisph_info": (C.c_int, [h, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _ip, _ip]),
        "sisph_set_stream": (C.c_int, [h, C.c_void_p]),
        "sisph_profile_enable": (C.c_int, [h, C.c_int32, C.c_char_p]),
        "sisph_profile_get": (C.c_int, [h, C.c_char_p, C.POINTER(C.c_int64), _dp, _dp]),
        "sisph_launch_count": (C.c_int64, [h]),
        "sisph_save": (C.c_int, [h, C.c_char_p]),
        "sisph_load": (C.c_int, [h, C.c_char_p]),
        "sisph_last_error": (C.c_char_p, [h]),
        "sisph_version": (C.c_char_p, []),
        "sisph_neighbors_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_double, _dp, _dp, _ip, C.c_int32,
                                              C.c_void_p, C.c_void_p, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class SisphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc, handle=None, allow=()):
    if rc != OK and rc not in allow:
        msg = load_library().sisph_last_error(handle)
        raise SisphError(rc, msg.decode() if msg else "")
    return rc


# --- functions with the C names (marshalling only) ---------------------------

def sisph_default_options():
    o = sisph_options()
    load_library().sisph_default_options(C.byref(o))
    return o


def sisph_default_case():
    q = sisph_case_params()
    load_library().sisph_default_case(C.byref(q))
    return q


def _arr(a, dtype=np.float64):
    return None if a is None else np.ascontiguousarray(a, dtype)


def particles_from_case(case):
    """Build a sisph_particles struct (plus the arrays it points into)."""
    keep = {}
    P = sisph_particles()
    P.dim = int(case["dim"])
    P.n = int(case["n"])
    for key in ("x", "y", "z", "u", "v", "w", "m", "rho", "p", "wall_u", "wall_v", "wall_w"):
        a = _arr(case.get(key))
        keep[key] = a
        setattr(P, key, a.ctypes.data_as(_dp) if a is not None else None)
    kind = _arr(case.get("kind"), np.int32)
    keep["kind"] = kind
    P.kind = kind.ctypes.data_as(_ip) if kind is not None else None
    for k in range(3):
        P.lo[k] = case["lo"][k]
        P.hi[k] = case["hi"][k]
        P.periodic[k] = int(case["periodic"][k])
    return P, keep


def case_params_from_dict(prm):
    q = sisph_default_case()
    for key in ("h", "dt", "rho0", "nu", "alpha", "c0", "tol", "p_ref", "gtvf_hfac"):
        setattr(q, key, float(prm[key]))
    for key in ("max_iter", "pgrad_symm", "free_surface", "ustar_slip", "pref_mode", "gtvf_K"):
        setattr(q, key, int(prm[key]))
    q.adaptive_dt = int(prm.get("adaptive_dt", 0))
    q.ppe_solver = int(prm.get("ppe_solver", 0))
    for k in range(3):
        q.g[k] = float(prm["g"][k])
    return q


def sisph_create(particles, h, dt, rho0, nu, g, opt=None):
    L = load_library()
    out = C.c_void_p()
    garr = (C.c_double * 3)(*[float(v) for v in g])
    rc = L.sisph_create(C.byref(particles), h, dt, rho0, nu, C.cast(garr, _dp),
                        C.byref(opt) if opt is not None else None, C.byref(out))
    _check(rc)
    return out


def sisph_batch_create(particles_list, params_list, opt=None):
    L = load_library()
    n = len(particles_list)
    parr = (sisph_particles * n)(*particles_list)
    qarr = (sisph_case_params * n)(*params_list)
    out = C.c_void_p()
    rc = L.sisph_batch_create(n, parr, qarr, C.byref(opt) if opt is not None else None, C.byref(out))
    _check(rc)
    return out


def sisph_destroy(h):
    load_library().sisph_destroy(h)


def sisph_build_neighbors(h):
    return _check(load_library().sisph_build_neighbors(h), h)


def sisph_compute_density(h):
    return _check(load_library().sisph_compute_density(h), h)


def sisph_ppe_solve(h, tol, max_iter, ncases=1):
    it = np.zeros(ncases, np.int32)
    rs = np.zeros(ncases, np.float64)
    rc = load_library().sisph_ppe_solve(h, float(tol), int(max_iter), it.ctypes.data_as(_ip),
                                        rs.ctypes.data_as(_dp))
    _check(rc, h, allow=(ENOTCONVERGED,))
    return rc, it, rs


def sisph_step(h, nsteps=1):
    rc = load_library().sisph_step(h, int(nsteps))
    return _check(rc, h, allow=(ENOTCONVERGED,))


def sisph_get(h, field, n, out=None):
    out = np.empty(n, np.float64) if out is None else out
    _check(load_library().sisph_get(h, FIELDS[field] if isinstance(field, str) else field,
                                    out.ctypes.data_as(_dp)), h)
    return out


def sisph_set(h, field, values):
    a = np.ascontiguousarray(values, np.float64)
    _check(load_library().sisph_set(h, FIELDS[field] if isinstance(field, str) else field,
                                    a.ctypes.data_as(_dp)), h)


def _field_ids(fields):
    return np.ascontiguousarray([FIELDS[f] if isinstance(f, str) else int(f) for f in fields], np.int32)


def sisph_set_many(h, fields, arrays):
    """Write several fields in one call (arrays: n doubles each, caller's
    order; page-locked arrays copy asynchronously)."""
    ids = _field_ids(fields)
    arrs = [np.ascontiguousarray(a, np.float64) for a in arrays]
    ptrs = (_dp * max(1, len(arrs)))(*[a.ctypes.data_as(_dp) for a in arrs])
    _check(load_library().sisph_set_many(h, len(arrs), ids.ctypes.data_as(_ip), ptrs), h)


def sisph_get_many(h, fields, n, outs=None):
    """Read several fields in one call into `outs` (new arrays if None)."""
    ids = _field_ids(fields)
    outs = [np.empty(n, np.float64) for _ in fields] if outs is None else outs
    ptrs = (_dp * max(1, len(outs)))(*[o.ctypes.data_as(_dp) for o in outs])
    _check(load_library().sisph_get_many(h, len(outs), ids.ctypes.data_as(_ip), ptrs), h)
    return outs


def sisph_neighbors(h, n):
    L = load_library()
    counts = np.zeros(n, np.int32)
    tot = C.c_int64()
    _check(L.sisph_neighbors(h, counts.ctypes.data_as(_ip), None, 0, C.byref(tot)), h)
    idx = np.zeros(max(1, tot.value), np.int32)
    _check(L.sisph_neighbors(h, counts.ctypes.data_as(_ip), idx.ctypes.data_as(_ip), idx.size,
                             C.byref(tot)), h)
    return counts, idx[:tot.value]


def sisph_batch_step(h, nsteps, ncases):
    """Steps every case of a batch handle; returns (code, PPE sweeps per case)."""
    its = np.zeros(ncases, np.int32)
    rc = load_library().sisph_batch_step(h, int(nsteps), its.ctypes.data_as(_ip))
    _check(rc, h, allow=(ENOTCONVERGED,))
    return rc, its


def sisph_stats(h, ncases):
    arr = (sisph_case_stats * ncases)()
    _check(load_library().sisph_stats(h, arr), h)
    return [arr[i] for i in range(ncases)]


def sisph_info(h):
    n, nf = C.c_int64(), C.c_int64()
    nc, cap = C.c_int32(), C.c_int32()
    _check(load_library().sisph_info(h, C.byref(n), C.byref(nf), C.byref(nc), C.byref(cap)), h)
    return dict(n=n.value, n_fluid=nf.value, ncases=nc.value, nbr_capacity=cap.value)


def sisph_set_stream(h, stream_ptr):
    return _check(load_library().sisph_set_stream(h, C.c_void_p(stream_ptr) if stream_ptr else None), h)


def sisph_profile_enable(h, on=True, only=None):
    return _check(load_library().sisph_profile_enable(h, int(on), only.encode() if only else None), h)


def sisph_profile_get(h, kernel):
    n, ms, units = C.c_int64(), C.c_double(), C.c_double()
    _check(load_library().sisph_profile_get(h, kernel.encode(), C.byref(n), C.byref(ms),
                                            C.byref(units)), h)
    return n.value, ms.value, units.value


def sisph_launch_count(h):
    return load_library().sisph_launch_count(h)


def sisph_save(h, path):
    return _check(load_library().sisph_save(h, str(path).encode()), h)


def sisph_load(h, path):
    return _check(load_library().sisph_load(h, str(path).encode()), h)


def sisph_last_error(h=None):
    m = load_library().sisph_last_error(h)
    return m.decode() if m else ""


def sisph_version():
    return load_library().sisph_version().decode()


def sisph_neighbors_noalloc(dim, n, x_ptr, y_ptr, z_ptr, h, lo, hi, periodic, cap,
                            counts_ptr, idx_ptr, stream_ptr=None):
    """Neighbour search without allocation; every pointer is a device address.

    Scratch lives in a fixed device array inside the library, for callers
    that cannot allocate device memory themselves (see include/sisph.h)."""
    lo_a = (C.c_double * 3)(*lo)
    hi_a = (C.c_double * 3)(*hi)
    per_a = (C.c_int32 * 3)(*periodic)
    rc = load_library().sisph_neighbors_noalloc(
        int(dim), int(n), C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.c_void_p(z_ptr or 0), float(h),
        C.cast(lo_a, _dp), C.cast(hi_a, _dp), C.cast(per_a, _ip), int(cap),
        C.c_void_p(counts_ptr), C.c_void_p(idx_ptr), C.c_void_p(stream_ptr or 0))
    return _check(rc, None)


class Simulation:
    """A handle plus numpy marshalling for one case or a batch of cases."""

    def __init__(self, cases, precision=FP64, **options):
        if isinstance(cases, dict):
            cases = [cases]
        self.cases = cases
        opt = sisph_default_options()
        opt.precision = precision
        for k, v in options.items():
            setattr(opt, k, v)
        self._keep = []
        plist, qlist = [], []
        for c in cases:
            P, keep = particles_from_case(c)
            self._keep.append(keep)
            plist.append(P)
            qlist.append(case_params_from_dict(c["params"]))
        self.h = sisph_batch_create(plist, qlist, opt)
        info = sisph_info(self.h)
        self.n = info["n"]
        self.ncases = info["ncases"]
        self.nbr_capacity = info["nbr_capacity"]

    def close(self):
        if getattr(self, "h", None):
            sisph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self, field):
        return sisph_get(self.h, field, self.n)

    def set(self, field, values):
        sisph_set(self.h, field, values)

    def get_many(self, fields, outs=None):
        return sisph_get_many(self.h, fields, self.n, outs)

    def set_many(self, fields, arrays):
        sisph_set_many(self.h, fields, arrays)

    def step(self, nsteps=1):
        return sisph_step(self.h, nsteps)

    def build_neighbors(self):
        return sisph_build_neighbors(self.h)

    def density(self):
        return sisph_compute_density(self.h)

    def ppe_solve(self, tol, max_iter):
        return sisph_ppe_solve(self.h, tol, max_iter, self.ncases)

    def neighbors(self):
        return sisph_neighbors(self.h, self.n)

    def stats(self):
        return sisph_stats(self.h, self.ncases)
