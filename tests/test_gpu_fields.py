"""Several fields in one call (sisph_get_many / sisph_set_many) against the
single-field calls: the same values in the caller's order, the same step
afterwards, and a bad field rejected before anything is written."""
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


STATE = {2: ["x", "y", "u", "v", "ut", "vt", "p"], 3: ["x", "y", "z", "u", "v", "w", "ut", "vt", "wt", "p"]}


@pytest.mark.parametrize("make", [lambda: workloads.dam_break_2d(dx=0.04),
                                  lambda: workloads.dam_break_3d(dx=0.06)], ids=["2d", "3d"])
def test_many_equals_one_by_one(sisph, make):
    case = make()
    fields = STATE[case["dim"]]
    a = sisph.Simulation(case, precision=sisph.MIXED)
    b = sisph.Simulation(case, precision=sisph.MIXED)
    a.step(3)
    b.step(3)
    got = a.get_many(fields + ["rho", "ncount"])
    for f, g in zip(fields + ["rho", "ncount"], got):
        assert np.array_equal(g, a.get(f)), f
    # write a perturbed state both ways, then step both handles alike
    rng = np.random.Generator(np.random.PCG64(5))
    fl = case["kind"] == 0
    new = []
    for f, g in zip(fields, got):
        v = g.copy()
        if f in ("u", "v", "w"):
            v = v + np.where(fl, rng.normal(0, 1e-3, v.size), 0.0)
        new.append(v)
    a.set_many(fields, new)
    for f, v in zip(fields, new):
        b.set(f, v)
    a.step(2)
    b.step(2)
    for f in fields:
        assert np.array_equal(a.get(f), b.get(f)), f
    a.close()
    b.close()


def test_many_rejects_a_bad_field_before_writing(sisph):
    case = workloads.taylor_green(20)
    sim = sisph.Simulation(case)
    p0 = sim.get("p")
    with pytest.raises(sisph.SisphError) as ei:
        sim.set_many(["p", "m"], [p0 + 1.0, p0])          # mass is read-only
    assert ei.value.code == sisph.EINVAL
    assert np.array_equal(sim.get("p"), p0)
    with pytest.raises(sisph.SisphError) as ei:
        sim.set_many(["p", "z"], [p0 + 1.0, p0])          # no z in 2D
    assert ei.value.code == sisph.EINVAL
    assert np.array_equal(sim.get("p"), p0)
    with pytest.raises(sisph.SisphError):
        sim.get_many(["p", 999])
    sim.close()


def test_many_grows_its_staging_between_calls(sisph):
    """A first call with one field, then calls with more: the staging grows
    and every field still matches its single-field read."""
    case = workloads.dam_break_2d(dx=0.04)
    sim = sisph.Simulation(case, precision=sisph.MIXED)
    sim.step(2)
    (p,) = sim.get_many(["p"])
    assert np.array_equal(p, sim.get("p"))
    fields = STATE[2] + ["rho", "ncount", "nx", "ny"]
    for f, g in zip(fields, sim.get_many(fields)):
        assert np.array_equal(g, sim.get(f)), f
    new = [sim.get(f) + (1e-3 if f in ("u", "v") else 0.0) for f in STATE[2]]
    sim.set_many(STATE[2], new)
    for f, v in zip(STATE[2], new):
        assert np.array_equal(sim.get(f), v), f
    sim.close()
