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


def _noalloc(sisph, case, cap):
    import torch
    dev = torch.device("cuda")
    n = case["n"]
    x = torch.tensor(case["x"], dtype=torch.float64, device=dev)
    y = torch.tensor(case["y"], dtype=torch.float64, device=dev)
    z = torch.tensor(case["z"], dtype=torch.float64, device=dev)
    counts = torch.full((n,), -1, dtype=torch.int32, device=dev)
    idx = torch.full((n * cap,), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    sisph.sisph_neighbors_noalloc(case["dim"], n, x.data_ptr(), y.data_ptr(),
                                  z.data_ptr() if case["dim"] == 3 else None,
                                  case["params"]["h"], case["lo"], case["hi"], case["periodic"], cap,
                                  counts.data_ptr(), idx.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
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
