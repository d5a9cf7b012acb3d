"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/sisph.h declares, and rejects bad arguments on the host before any
device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1908_01762_gb300 as pkg
    pkg.build()
    from paper_1908_01762_gb300 import sisph
    return sisph.load_library()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "sisph.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(sisph_[a-z_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_checked_build_exports_every_declared_symbol():
    # the variant that bounds-checks every gathered neighbour index on the
    # device (SISPH_CHECKED) has the same C-ABI
    from paper_1908_01762_gb300 import buildlib
    path = buildlib.build(checked=True)
    assert path.endswith("libsisph_checked.so")
    checked = C.CDLL(path)
    for n in _declared():
        assert hasattr(checked, n), n


def test_version_string(lib):
    from paper_1908_01762_gb300 import sisph
    assert "sm_103a" in sisph.sisph_version()


def test_defaults_follow_the_paper(lib):
    from paper_1908_01762_gb300 import sisph
    o = sisph.sisph_default_options()
    assert o.omega == 0.5 and o.min_iter == 2 and o.eta == 0.01 and o.fs_ratio == 0.8
    assert o.physics.max_iter == 1000 and o.physics.gtvf_K == 1


def _bad(case, **over):
    from paper_1908_01762_gb300 import sisph
    P, keep = sisph.particles_from_case(case)
    q = sisph.case_params_from_dict(dict(case["params"], **over))
    for k, v in over.items():
        if hasattr(P, k) and k not in ("h", "dt"):
            setattr(P, k, v)
    return P, q, keep


@pytest.mark.parametrize("mut", ["dim", "n", "h", "dt", "kind", "mass", "small_box", "K"])
def test_invalid_arguments_are_rejected_on_the_host(lib, mut):
    from paper_1908_01762_gb300 import sisph
    case = workloads.taylor_green(8)
    P, keep = sisph.particles_from_case(case)
    q = sisph.case_params_from_dict(case["params"])
    if mut == "dim":
        P.dim = 4
    elif mut == "n":
        P.n = 0
    elif mut == "h":
        q.h = -1.0
    elif mut == "dt":
        q.dt = 0.0
    elif mut == "kind":
        keep["kind"][3] = 7
    elif mut == "mass":
        keep["m"][0] = -1.0
    elif mut == "small_box":
        q.h = 0.2     # 1 / (3 h) < 3 cells in a periodic box
    elif mut == "K":
        q.gtvf_K = 0
    out = C.c_void_p()
    parr = (sisph.sisph_particles * 1)(P)
    qarr = (sisph.sisph_case_params * 1)(q)
    rc = lib.sisph_batch_create(1, parr, qarr, None, C.byref(out))
    assert rc == sisph.EINVAL
    assert not out.value
    assert sisph.sisph_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    from paper_1908_01762_gb300 import sisph
    buf = np.zeros(4)
    assert lib.sisph_step(None, 1) == sisph.EINVAL
    assert lib.sisph_get(None, 0, buf.ctypes.data_as(C.POINTER(C.c_double))) == sisph.EINVAL
    assert lib.sisph_build_neighbors(None) == sisph.EINVAL
    ids = np.zeros(1, np.int32)
    ptrs = (C.POINTER(C.c_double) * 1)(buf.ctypes.data_as(C.POINTER(C.c_double)))
    assert lib.sisph_get_many(None, 1, ids.ctypes.data_as(C.POINTER(C.c_int32)), ptrs) == sisph.EINVAL
    assert lib.sisph_set_many(None, 1, ids.ctypes.data_as(C.POINTER(C.c_int32)), ptrs) == sisph.EINVAL
    lib.sisph_destroy(None)


def test_product_path_has_no_oracle_or_fallback():
    """The package never imports the oracle and has no CPU code path."""
    pkg = os.path.join(ROOT, "paper_1908_01762_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f
