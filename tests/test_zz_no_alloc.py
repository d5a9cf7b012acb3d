"""The neighbour search that allocates nothing (sisph_neighbors_noalloc).

That entry point serves callers that cannot call cudaMalloc themselves -- an
application whose device memory is already fully reserved by its own
allocator, or a latency-critical loop that must not pay for a cudaMalloc /
cudaFree that can synchronise the device.  Its scratch memory is a fixed
device array inside the library.  This test calls it through the C-ABI on
device buffers the test allocates, twice in a row on different point sets
(the second call must not see anything the first left in the shared scratch
array), and compares its lists with the existing entry point (a handle's
sisph_neighbors) exactly: neighbour sets are integer data.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sisph():
    import paper_1908_01762_gb300 as pkg
    pkg.build()
    from paper_1908_01762_gb300 import sisph as mod
    mod.load_library()
    return mod


def _existing(sisph, case):
    sim = sisph.Simulation(case)
    counts, idx = sim.neighbors()
    sim.close()
    return counts, idx


def _noalloc(sisph, case, cap, expect_rc=None):
    import torch
    dev = torch.device("cuda")
    n = case["n"]
    x = torch.tensor(case["x"], dtype=torch.float64, device=dev)
    y = torch.tensor(case["y"], dtype=torch.float64, device=dev)
    z = torch.tensor(case["z"], dtype=torch.float64, device=dev)
    counts = torch.full((n,), -1, dtype=torch.int32, device=dev)
    idx = torch.full((n * cap,), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    args = (case["dim"], n, x.data_ptr(), y.data_ptr(), z.data_ptr() if case["dim"] == 3 else None,
            case["params"]["h"], case["lo"], case["hi"], case["periodic"], cap,
            counts.data_ptr(), idx.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if expect_rc is None:
        sisph.sisph_neighbors_noalloc(*args)
    else:
        with pytest.raises(sisph.SisphError) as ei:
            sisph.sisph_neighbors_noalloc(*args)
        assert ei.value.code == expect_rc
    c = counts.cpu().numpy()
    rows = idx.cpu().numpy().reshape(n, cap)
    flat = np.concatenate([rows[i, :c[i]] for i in range(n)])
    return c, flat


def test_noalloc_matches_existing_entry_point_twice(sisph):
    first = workloads.taylor_green(64, perturb=0.2, seed=17)        # periodic, 4096 points
    second = workloads.lid_driven_cavity(40)                        # walls, 1600 + 516 points
    for case in (first, second):
        cap = 64
        c_new, i_new = _noalloc(sisph, case, cap)
        c_old, i_old = _existing(sisph, case)
        assert np.array_equal(c_new, c_old)
        assert np.array_equal(i_new, i_old)


def test_noalloc_rejects_sizes_beyond_its_limit(sisph):
    import torch
    n = 65537                       # one more than SISPH_NOALLOC_MAX_POINTS
    big = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(sisph.SisphError) as ei:
        sisph.sisph_neighbors_noalloc(2, n, big.data_ptr(), big.data_ptr(), None, 0.01,
                                      (0, 0, 0), (1, 1, 1), (0, 0, 0), 8, out.data_ptr(),
                                      out.data_ptr())
    assert ei.value.code == sisph.EINVAL
    assert "65536" in str(ei.value)


def test_noalloc_3d_dam_break(sisph):
    # 3D: the 27-cell stencil and the z coordinate; walls and fluid
    case = workloads.dam_break_3d(dx=0.05)
    assert case["dim"] == 3 and case["n"] < 65536
    c_new, i_new = _noalloc(sisph, case, 128)
    c_old, i_old = _existing(sisph, case)
    assert np.array_equal(c_new, c_old)
    assert np.array_equal(i_new, i_old)


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_points_outside_a_closed_box(sisph, dim):
    # fluid that left a non-periodic box is searched from the edge cell it is
    # clamped into; its rows must still hold N(i) exactly
    case = workloads.dam_break_2d(dx=0.05) if dim == 2 else workloads.dam_break_3d(dx=0.06)
    case = dict(case)
    rng = np.random.Generator(np.random.PCG64(3))
    fl = np.nonzero(case["kind"] == 0)[0]
    pick = rng.choice(fl, 12, replace=False)
    for key, k in (("x", 0), ("y", 1), ("z", 2))[:dim]:
        a = case[key].copy()
        span = case["hi"][k] - case["lo"][k]
        a[pick[:4]] = case["hi"][k] + rng.uniform(0.0, 0.3 * span, 4)
        a[pick[4:8]] = case["lo"][k] - rng.uniform(0.0, 0.3 * span, 4)
        a[pick[8:]] = case["hi"][k] + 0.05 * rng.uniform(0, 1, 4)   # close together, outside
        case[key] = a
    c_new, i_new = _noalloc(sisph, case, 128)
    c_old, i_old = _existing(sisph, case)
    assert np.array_equal(c_new, c_old)
    assert np.array_equal(i_new, i_old)


def test_noalloc_row_beyond_capacity(sisph):
    # 25 neighbours per lattice point at h = dx: with cap = 20 every interior
    # row overflows; the call reports SISPH_ECAPACITY, counts are clipped to
    # cap and each clipped row holds the cap smallest indices of N(i)
    case = workloads.taylor_green(40, perturb=0.1, seed=9)
    cap = 20
    c_new, i_new = _noalloc(sisph, case, cap, expect_rc=sisph.ECAPACITY)
    c_old, i_old = _existing(sisph, case)
    assert np.any(c_old > cap)
    assert np.array_equal(c_new, np.minimum(c_old, cap))
    starts = np.concatenate([[0], np.cumsum(c_old)])
    want = np.concatenate([i_old[starts[i]:starts[i] + min(c_old[i], cap)] for i in range(case["n"])])
    assert np.array_equal(i_new, want)
    # the next call on the same shared scratch is clean again
    c2, i2 = _noalloc(sisph, case, 64)
    assert np.array_equal(c2, c_old) and np.array_equal(i2, i_old)


def test_noalloc_rejects_a_capturing_stream(sisph):
    # the call synchronises its stream, so it refuses one that is capturing a
    # graph and launches nothing
    import torch
    case = workloads.taylor_green(20)
    n = case["n"]
    x = torch.tensor(case["x"], dtype=torch.float64, device="cuda")
    y = torch.tensor(case["y"], dtype=torch.float64, device="cuda")
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    idx = torch.zeros(n * 32, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(sisph.SisphError) as ei:
        with torch.cuda.graph(g, stream=stream):
            sisph.sisph_neighbors_noalloc(2, n, x.data_ptr(), y.data_ptr(), None,
                                          case["params"]["h"], case["lo"], case["hi"],
                                          case["periodic"], 32, counts.data_ptr(),
                                          idx.data_ptr(), stream.cuda_stream)
    assert ei.value.code == sisph.EINVAL
    assert "capturing" in str(ei.value)
    torch.cuda.synchronize()
    assert int(counts.abs().sum()) == 0
