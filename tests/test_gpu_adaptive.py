"""Adaptive time step (Sec. 3.2) on the GPU against the oracle: the step
sequence and the state, in FP64 (1e-10 relative, sweep counts forced equal
as in the other FP64 parity tests), and the closed form of a free fall in
both precisions."""
import math

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


def relerr(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (s if s > 0 else 1.0)


@pytest.mark.parametrize("name", ["tgv", "db2d"])
def test_adaptive_steps_match_oracle_fp64(sisph, name):
    case = {"tgv": lambda: workloads.taylor_green(40, perturb=0.05, seed=3),
            "db2d": lambda: workloads.dam_break_2d(dx=0.04)}[name]()
    case["params"] = dict(case["params"], adaptive_dt=1, tol=0.0, max_iter=6)
    sim = sisph.Simulation(case)
    ref = oracle.Sim(case)
    for step in range(6):
        sim.step(1)
        rc, d = ref.step(1)
        st = sim.stats()[0]
        # dt of the next step and the simulated time
        assert abs(st.dt - ref.dt) <= 1e-12 * ref.dt, (step, st.dt, ref.dt)
    fl = case["kind"] == 0          # a wall's velocity slot holds its ghost velocity
    for f in ("x", "y", "u", "v", "p"):
        g, o = sim.get(f), ref.get(f)
        if f in ("u", "v"):
            g, o = g[fl], o[fl]
        assert relerr(g, o) < 1e-10, f
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_free_fall_closed_form(sisph, prec):
    case = workloads.free_fall_blob()
    h, g = case["params"]["h"], 9.81
    sim = sisph.Simulation(case, precision=prec)
    dt_f = 0.25 * math.sqrt(h / g)
    starts, dts, t = [], [], 0.0
    for _ in range(12):
        starts.append(t)
        dts.append(sim.stats()[0].dt)
        sim.step(1)
        t = sim.stats()[0].time
    assert dts[0] == case["params"]["dt"]
    for k in range(1, len(dts)):
        t_prev = starts[k - 1]
        cfl = 0.25 * h / (g * t_prev) if t_prev > 0 else math.inf
        expect = min(dt_f, cfl)
        assert abs(dts[k] - expect) <= 1e-12 * expect, (k, dts[k], expect)
    assert abs(t - sum(dts)) <= 1e-12 * t
    assert np.allclose(sim.get("y"), case["y"] - 0.5 * g * t * t, rtol=0, atol=1e-12)
    sim.close()


def test_adaptive_checkpoint_resumes_the_time_step(sisph, tmp_path):
    case = workloads.free_fall_blob()
    a = sisph.Simulation(case)
    a.step(5)
    path = tmp_path / "ck.bin"
    sisph.sisph_save(a.h, path)
    b = sisph.Simulation(case)
    sisph.sisph_load(b.h, path)
    assert b.stats()[0].dt == a.stats()[0].dt and b.stats()[0].time == a.stats()[0].time
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get("y"), b.get("y"))
    a.close()
    b.close()
