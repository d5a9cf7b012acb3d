"""Parity at the benchmark's full size: the perturbed 400 x 400 Taylor-Green
vortex (160,000 particles, dx = 0.0025, +-0.05 dx seeded noise, Re = 100,
PPE tolerance 1e-4), in the launch configuration the benchmark times
(MIXED precision, 256-thread tiles, CUDA-graph replay).  The oracle runs the
whole case (about a second per step on one core)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sisph():
    import paper_1908_01762_gb300 as pkg
    pkg.build()
    oracle.build()
    from paper_1908_01762_gb300 import sisph as mod
    mod.load_library()
    return mod


@pytest.fixture(scope="module")
def c2():
    return workloads.taylor_green(400, perturb=0.05, seed=1908, tol=1e-4)


def test_fullsize_neighbors_bit_exact(sisph, c2):
    sim = sisph.Simulation(c2, precision=sisph.MIXED)
    cg, ig = sim.neighbors()
    co, io = oracle.neighbors(c2)
    assert np.array_equal(cg, co) and np.array_equal(ig, io)
    sim.close()


def test_fullsize_step_fp64(sisph, c2):
    case = dict(c2, params=dict(c2["params"], tol=0.0, max_iter=8))
    sim = sisph.Simulation(case, precision=sisph.FP64)
    ref = oracle.Sim(case)
    sim.step(2)
    ref.step(2)
    for f in ("x", "y", "u", "v", "p", "rho"):
        a, b = sim.get(f), ref.get(f)
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10, f
    sim.close()


def test_fullsize_step_mixed(sisph, c2):
    case = dict(c2, params=dict(c2["params"], tol=0.0, max_iter=8))
    sim = sisph.Simulation(case, precision=sisph.MIXED, use_graph=1)
    ref = oracle.Sim(case)
    sim.step(2)
    ref.step(2)
    p, po = sim.get("p"), ref.get("p")
    assert np.linalg.norm(p - po) / np.linalg.norm(po) < 1e-4
    for f in ("u", "v"):
        a, b = sim.get(f), ref.get(f)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, f
    assert np.max(np.abs(sim.get("x") - ref.get("x"))) < 1e-8
    sim.close()


def test_fullsize_natural_convergence_mixed(sisph, c2):
    # both sides iterate to the same tolerance on their own
    sim = sisph.Simulation(c2, precision=sisph.MIXED, use_graph=1)
    ref = oracle.Sim(c2)
    sim.step(1)
    rc, ds = ref.step(1)
    st = sim.stats()[0]
    assert abs(st.iters - ds[0].iters) <= 1
    p, po = sim.get("p"), ref.get("p")
    assert np.linalg.norm(p - po) / np.linalg.norm(po) < 1e-4
    sim.close()


def test_fullsize_mixed_decay_rate(sisph, c2):
    """MIXED vs FP64 oracle on the TGV decay rate over 10 steps (Eq. tgv)."""
    import math
    sim = sisph.Simulation(c2, precision=sisph.MIXED, use_graph=1)
    ref = oracle.Sim(c2)
    sim.step(10)
    ref.step(10)
    t = 10 * c2["params"]["dt"]
    e0 = np.sum(c2["m"] * (c2["u"] ** 2 + c2["v"] ** 2))
    def rate(s):
        e = np.sum(c2["m"] * (s.get("u") ** 2 + s.get("v") ** 2))
        return math.log(e / e0) / (2 * t)
    bg, bo = rate(sim), rate(ref)
    assert abs(bg - bo) < 1e-4 * abs(bo)
    assert abs(bo + 8 * math.pi ** 2 / 100) < 0.05 * 8 * math.pi ** 2 / 100
    sim.close()


def test_sweep_sync_forms_agree_on_the_batch(sisph):
    """The batch of 64 cases (about 2.5M particles) has more tiles than the
    persistent kernel has blocks, so blocks own several tiles of different
    cases: the point-to-point sweeps must reproduce the grid-barrier form bit
    for bit, sweep counts included."""
    cases = workloads.batch_ensemble(64)
    out = []
    for sync in (2, 1):
        sim = sisph.Simulation(cases, precision=sisph.MIXED, ppe_sync=sync)
        sim.step(2)
        out.append(({f: sim.get(f) for f in ("x", "y", "u", "v", "p")},
                    [s.total_iters for s in sim.stats()]))
        sim.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    for f in a:
        assert np.array_equal(a[f], b[f]), f
