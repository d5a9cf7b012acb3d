"""BiCGStab PPE (the Krylov alternative of Sec. 3.1) on the GPU against the
oracle's BiCGStab: FP64 to 1e-10 relative with the iteration count fixed
(tol = 0) and after natural convergence (measured: 1e-15 to 1e-13), MIXED
within the stated 1e-4 relative L2 after convergence to 1e-6 (measured
1e-6); the
per-case choice inside a batch (a member equals its solo run bit for bit),
the Jacobi sweeps for singular systems, and fewer iterations than Jacobi at
the same tolerance."""
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


def tank(seed=21):
    c = workloads.still_tank_2d(16, 16, dx=0.05)
    rng = np.random.Generator(np.random.PCG64(seed))
    fl = c["kind"] == 0
    c["u"] = np.where(fl, rng.normal(0, 0.05, c["n"]), 0.0)
    c["v"] = np.where(fl, rng.normal(0, 0.05, c["n"]), 0.0)
    c["params"] = dict(c["params"], ppe_solver=1)
    return c


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_bicgstab_solve_fp64_fixed_iterations(sisph, iters):
    c = tank()
    sim = sisph.Simulation(c)
    sim.density()
    rc, it, res = sim.ppe_solve(0.0, iters)
    ref = oracle.Sim(c)
    ref.density()
    rc2, d = ref.ppe_solve(0.0, iters)
    assert it[0] == d.iters == iters
    assert relerr(sim.get("p"), ref.get("p")) < 1e-10
    sim.close()


def test_bicgstab_solve_fp64_converged(sisph):
    c = tank(5)
    sim = sisph.Simulation(c)
    sim.density()
    rc, it, res = sim.ppe_solve(1e-10, 500)
    ref = oracle.Sim(c)
    ref.density()
    rc2, d = ref.ppe_solve(1e-10, 500)
    assert rc == 0 and d.converged
    assert abs(int(it[0]) - d.iters) <= 1
    assert relerr(sim.get("p"), ref.get("p")) < 1e-10
    sim.close()


def test_bicgstab_steps_fp64(sisph):
    c = workloads.dam_break_2d(dx=0.04)
    c["params"] = dict(c["params"], ppe_solver=1, tol=0.0, max_iter=5)
    sim = sisph.Simulation(c)
    ref = oracle.Sim(c)
    sim.step(3)
    ref.step(3)
    fl = c["kind"] == 0
    for f in ("x", "y", "u", "v", "p"):
        g, o = sim.get(f), ref.get(f)
        if f in ("u", "v"):
            g, o = g[fl], o[fl]
        assert relerr(g, o) < 1e-10, f
    sim.close()


def test_bicgstab_mixed_bound(sisph):
    """MIXED (FP32 vectors, FP64 dot products) against the FP64 oracle, both
    converged to 1e-6: relative L2 of the fluid pressure within the stated
    1e-4 (measured 1e-6).  At a loose tolerance (1e-4) the two stop a few
    iterations apart on different paths and differ by about 1e-3, each within
    its own truncation error of the exact solution.  (The
    outer wall layer of this lattice touches the fluid only at exactly 3h,
    where the FP32 kernel weight is 0: such walls get p = 0; they carry no
    weight in any fluid row, so the fluid is unaffected.)"""
    c = tank(7)
    sim = sisph.Simulation(c, precision=sisph.MIXED)
    sim.density()
    rc, it, res = sim.ppe_solve(1e-6, 500)
    ref = oracle.Sim(c)
    ref.density()
    ref.ppe_solve(1e-6, 500)
    fl = c["kind"] == 0
    g, o = sim.get("p")[fl], ref.get("p")[fl]
    l2 = np.linalg.norm(g - o) / np.linalg.norm(o)
    print("MIXED BiCGStab relative L2", l2)
    assert l2 < 1e-4
    sim.close()


def test_bicgstab_batch_member_equals_solo(sisph):
    cases = [workloads.dam_break_2d(dx=0.05), workloads.taylor_green(24, tol=1e-3),
             workloads.dam_break_2d(dx=0.04)]
    for c in (cases[0], cases[2]):
        c["params"] = dict(c["params"], ppe_solver=1)
    batch = sisph.Simulation(cases, precision=sisph.MIXED)
    batch.step(3)
    offs = np.cumsum([0] + [c["n"] for c in cases])
    for k, c in enumerate(cases):
        solo = sisph.Simulation(c, precision=sisph.MIXED)
        solo.step(3)
        for f in ("x", "y", "p"):
            assert np.array_equal(batch.get(f)[offs[k]:offs[k + 1]], solo.get(f)), (k, f)
        solo.close()
    batch.close()


def test_bicgstab_leaves_singular_systems_to_jacobi(sisph):
    c = workloads.lid_driven_cavity(20)
    a = sisph.Simulation(c)
    cb = dict(c)
    cb["params"] = dict(c["params"], ppe_solver=1)
    b = sisph.Simulation(cb)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get("p"), b.get("p"))
    a.close()
    b.close()


def test_bicgstab_needs_fewer_iterations(sisph):
    c = workloads.dam_break_2d(dx=0.02)
    cb = dict(c)
    cb["params"] = dict(c["params"], ppe_solver=1)
    its = []
    for case in (c, cb):
        sim = sisph.Simulation(case, precision=sisph.MIXED)
        sim.step(2)
        rc, it, res = sim.ppe_solve(1e-6, 5000)
        its.append(int(it[0]))
        sim.close()
    assert its[1] < its[0]
