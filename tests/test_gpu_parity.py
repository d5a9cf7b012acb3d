"""CUDA path (through the C-ABI) against the FP64 CPU oracle.

* neighbour sets: bit-exact, in both precisions (the predicate is FP64);
* FP64 form: 1e-10 relative on every field, with the number of PPE sweeps
  forced equal on both sides (tol = 0, max_iter = N), because a residual that
  lands within rounding of the tolerance could otherwise stop one side a
  sweep earlier;
* MIXED form: relative L2 error of the pressure <= 1e-4 after both sides
  converge to the same tolerance (the stated FP32 bound);
* a batch member is bit-identical to its solo run, graph replay is
  bit-identical to direct launches, and a checkpoint resumes bit-identically.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


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


def with_params(case, **over):
    c = dict(case)
    c["params"] = dict(case["params"], **over)
    return c


def small_cases():
    return {
        "tgv_lattice": workloads.taylor_green(50),
        "tgv_perturbed": workloads.taylor_green(40, perturb=0.05, seed=1908),
        "ldc": workloads.lid_driven_cavity(30),
        "tank": workloads.still_tank_2d(16, 16),
        "db2d": workloads.dam_break_2d(dx=0.04),
        "db3d": workloads.dam_break_3d(dx=0.05),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_neighbor_sets_bit_exact(sisph, name, prec):
    case = CASES[name]
    sim = sisph.Simulation(case, precision=prec)
    cg, ig = sim.neighbors()
    co, io = oracle.neighbors(case)
    assert np.array_equal(cg, co)
    assert np.array_equal(ig, io)
    sim.close()


def test_neighbors_ragged_tiles_and_tiny_case(sisph):
    # a case smaller than one tile and one with a ragged last tile
    for case in (workloads.still_tank_2d(3, 3), workloads.taylor_green(27)):
        sim = sisph.Simulation(case, block=64)
        cg, ig = sim.neighbors()
        co, io = oracle.neighbors(case)
        assert np.array_equal(cg, co) and np.array_equal(ig, io)
        sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_neighbors_of_particles_outside_the_box(sisph, dim):
    # fluid that left a non-periodic box is clamped into the edge cells; its
    # neighbours must still match the definition exactly
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
    sim = sisph.Simulation(case, precision=sisph.MIXED)
    cg, ig = sim.neighbors()
    co, io = oracle.neighbors(case)
    assert np.array_equal(cg, co) and np.array_equal(ig, io)
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_density_with_particles_outside_the_box(sisph, dim):
    """Particles clamped out of a closed box are outside the near range, which
    the FP32 mirror carries in the sign of the mass: the MIXED density (the
    separate pass, and the one the step's first refresh sums in its filter)
    still uses |m| and the exact pair set, and matches the oracle within the
    MIXED bound (the far cluster's pair vectors are FP32 differences of
    coordinates some 10 cells from their cell's origin)."""
    case = workloads.dam_break_2d(dx=0.05) if dim == 2 else workloads.dam_break_3d(dx=0.06)
    case = dict(case)
    rng = np.random.Generator(np.random.PCG64(5))
    fl = np.nonzero(case["kind"] == 0)[0]
    pick = rng.choice(fl, 12, replace=False)
    for key, k in (("x", 0), ("y", 1), ("z", 2))[:dim]:
        a = case[key].copy()
        a[pick[:6]] = case["hi"][k] + 0.05 * rng.uniform(0, 1, 6)   # outside, near the wall
        a[pick[6:]] = case["hi"][k] + 3.0 + 0.02 * rng.uniform(0, 1, 6)   # over 8 cells out, together
        case[key] = a
    ref = oracle.Sim(case)
    ref.density()
    want = ref.get("rho")
    fluid = case["kind"] == 0
    a = sisph.Simulation(case, precision=sisph.MIXED)
    a.density()
    b = sisph.Simulation(case, precision=sisph.MIXED)
    b.step(1)                       # the density of the step's first refresh
    for got in (a.get("rho"), b.get("rho")):
        assert np.max(np.abs(got[fluid] - want[fluid]) / want[fluid]) < 1e-4
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["tgv_perturbed", "ldc", "db2d", "db3d"])
def test_density_and_normals_fp64(sisph, name):
    case = CASES[name]
    sim = sisph.Simulation(case)
    sim.density()
    ref = oracle.Sim(case)
    ref.density()
    assert relerr(sim.get("rho"), ref.get("rho")) < FP64_TOL
    for f in ("nx", "ny", "nz") if case["dim"] == 3 else ("nx", "ny"):
        assert np.max(np.abs(sim.get(f) - ref.get(f))) < 1e-10
    sim.close()


@pytest.mark.parametrize("name,sweeps", [("tank", 40), ("ldc", 25), ("tgv_perturbed", 30),
                                         ("db3d", 12)])
def test_ppe_solve_fp64(sisph, name, sweeps):
    case = CASES[name]
    rng = np.random.Generator(np.random.PCG64(5))
    fl = case["kind"] == 0
    c = dict(case)
    c["u"] = case["u"] + np.where(fl, rng.normal(0, 0.1, case["n"]), 0)
    c["v"] = case["v"] + np.where(fl, rng.normal(0, 0.1, case["n"]), 0)
    sim = sisph.Simulation(c)
    sim.density()
    rc, it, res = sim.ppe_solve(0.0, sweeps)
    ref = oracle.Sim(c)
    ref.density()
    rco, d = ref.ppe_solve(0.0, sweeps)
    assert it[0] == d.iters == sweeps
    assert abs(res[0] - d.residual) <= 1e-8 * abs(d.residual)
    for f in ("rhs", "diag"):
        g, o = sim.get(f), ref.get(f)
        assert relerr(g[fl], o[fl]) < FP64_TOL
    assert relerr(sim.get("p"), ref.get("p")) < FP64_TOL
    sim.close()


def _resync(ref, sim, case):
    """Copy the GPU state into the oracle (walls keep the oracle's own velocity)."""
    fl = case["kind"] == 0
    names = ["x", "y", "ut", "vt", "p", "rho"] + (["z", "wt"] if case["dim"] == 3 else [])
    for f in names:
        ref.set(f, sim.get(f))
    for f in ["u", "v"] + (["w"] if case["dim"] == 3 else []):
        ref.set(f, np.where(fl, sim.get(f), ref.get(f)))


def test_tgv_lattice_steps_fp64_resynced(sisph):
    # On the unperturbed 50 x 50 lattice the sweeps at tol = 0 leave the
    # periodic PPE's mean pressure drifting, and every step starts from the
    # oracle's state again so that a rounding difference in one step is not
    # carried into the next: each step is checked from a common state.
    case = with_params(workloads.taylor_green(50), tol=0.0, max_iter=20)
    sim = sisph.Simulation(case)
    ref = oracle.Sim(case)
    for st in range(10):
        sim.step(1)
        ref.step(1)
        for f in ("x", "y", "u", "v", "ut", "vt", "p", "rho"):
            assert relerr(sim.get(f), ref.get(f)) < FP64_TOL, (st, f)
        _resync(ref, sim, case)
    sim.close()


STEP_CASES = [
    ("tgv_pert", lambda: workloads.taylor_green(40, perturb=0.05), 5, 15),
    ("ldc", lambda: workloads.lid_driven_cavity(30), 5, 15),
    ("db2d", lambda: workloads.dam_break_2d(dx=0.04), 4, 10),
    ("db3d", lambda: workloads.dam_break_3d(dx=0.05), 3, 8),
    ("tgv_symm_K3", lambda: with_params(workloads.taylor_green(30, perturb=0.05),
                                        pgrad_symm=1, gtvf_K=3), 4, 10),
    ("ldc_noslip", lambda: with_params(workloads.lid_driven_cavity(24), ustar_slip=0), 4, 10),
]


@pytest.mark.parametrize("name,make,nsteps,sweeps", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_time_steps_fp64(sisph, name, make, nsteps, sweeps):
    case = with_params(make(), tol=0.0, max_iter=sweeps)
    sim = sisph.Simulation(case)
    ref = oracle.Sim(case)
    sim.step(nsteps)
    ref.step(nsteps)
    fl = case["kind"] == 0
    fields = ["x", "y", "u", "v", "ut", "vt", "p", "rho"]
    if case["dim"] == 3:
        fields += ["z", "w", "wt"]
    for f in fields:
        g, o = sim.get(f), ref.get(f)
        if f in ("u", "v", "w"):
            g, o = g[fl], o[fl]
        assert relerr(g, o) < FP64_TOL, f
    st = sim.stats()[0]
    assert st.iters == sweeps and st.solves == nsteps
    if case["params"]["pref_mode"] == 1:
        assert abs(st.p_ref - ref.p_ref) <= 1e-10 * abs(ref.p_ref)
    sim.close()


def test_natural_convergence_matches(sisph):
    # the paper's dam-break tolerance converges in a couple of sweeps with a
    # wide margin; both sides must take the same number of sweeps
    case = workloads.dam_break_2d(dx=0.02)
    sim = sisph.Simulation(case)
    ref = oracle.Sim(case)
    for _ in range(5):
        sim.step(1)
        rc, ds = ref.step(1)
        assert sim.stats()[0].iters == ds[0].iters
    assert relerr(sim.get("p"), ref.get("p")) < FP64_TOL
    sim.close()


@pytest.mark.parametrize("name", ["tgv_perturbed", "ldc", "tank", "db3d"])
def test_mixed_precision_pressure_bound(sisph, name):
    case = with_params(CASES[name], tol=1e-6, max_iter=20000)
    rng = np.random.Generator(np.random.PCG64(9))
    flm = case["kind"] == 0
    case["u"] = case["u"] + np.where(flm, rng.normal(0, 0.1, case["n"]), 0)
    case["v"] = case["v"] + np.where(flm, rng.normal(0, 0.1, case["n"]), 0)
    g = sisph.Simulation(case, precision=sisph.MIXED)
    g.density()
    rc, it, res = g.ppe_solve(1e-6, 20000)
    ref = oracle.Sim(case)
    ref.density()
    ref.ppe_solve(1e-6, 20000)
    pg, po = g.get("p"), ref.get("p")
    fl = case["kind"] == 0
    if name == "tgv_perturbed":      # singular periodic system: compare mean-free
        pg = pg - pg[fl].mean()
        po = po - po[fl].mean()
    l2 = np.linalg.norm(pg[fl] - po[fl]) / np.linalg.norm(po[fl])
    assert l2 <= 1e-4, l2
    g.close()


@pytest.mark.parametrize("name", ["ldc", "db2d"])
def test_mixed_steps_stay_close(sisph, name):
    # FP32 sums and sweeps against the FP64 oracle over 10 steps, same sweeps
    make = {"ldc": lambda: workloads.lid_driven_cavity(30),
            "db2d": lambda: workloads.dam_break_2d(dx=0.04)}[name]
    case = with_params(make(), tol=0.0, max_iter=10)
    g = sisph.Simulation(case, precision=sisph.MIXED)
    ref = oracle.Sim(case)
    g.step(10)
    ref.step(10)
    fl = case["kind"] == 0
    for f in ("u", "v"):
        a, b = g.get(f)[fl], ref.get(f)[fl]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4, f
    p, po = g.get("p")[fl], ref.get("p")[fl]
    assert np.linalg.norm(p - po) / np.linalg.norm(po) < 1e-4
    h = case["params"]["h"]
    assert np.max(np.abs(g.get("x") - ref.get("x"))) < 1e-5 * h
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_member_equals_solo(sisph, prec):
    cases = [workloads.taylor_green(24, re=300.0, tol=1e-3),
             workloads.lid_driven_cavity(20, re=400.0),
             workloads.taylor_green(33, perturb=0.05, re=80.0, tol=1e-3)]
    batch = sisph.Simulation(cases, precision=prec)
    batch.step(4)
    offs = np.cumsum([0] + [c["n"] for c in cases])
    bst = batch.stats()
    for k, c in enumerate(cases):
        solo = sisph.Simulation(c, precision=prec)
        solo.step(4)
        for f in ("x", "y", "u", "v", "p", "ut"):
            assert np.array_equal(batch.get(f)[offs[k]:offs[k + 1]], solo.get(f)), (k, f)
        assert bst[k].total_iters == solo.stats()[0].total_iters
        solo.close()
    batch.close()


def test_batch_beyond_the_balanced_case_count(sisph):
    """More than 1024 cases: the grid-barrier sweeps then hand out every tile
    of the batch and skip the finished cases' instead of spreading only the
    unfinished ones; members still equal their solo runs bit for bit."""
    rng = np.random.Generator(np.random.PCG64(77))
    cases = []
    for q in range(1100):
        if q % 2:
            cases.append(workloads.lid_driven_cavity(int(rng.integers(11, 15)),
                                                     re=float(rng.uniform(100, 400))))
        else:
            cases.append(workloads.taylor_green(int(rng.integers(11, 15)),
                                                re=float(rng.uniform(50, 300)), tol=1e-3))
    batch = sisph.Simulation(cases, precision=sisph.MIXED)
    batch.step(2)
    offs = np.cumsum([0] + [c["n"] for c in cases])
    bst = batch.stats()
    assert len(set(s.total_iters for s in bst)) > 1          # cases stop at different sweeps
    for k in (0, 1, 1099):
        solo = sisph.Simulation(cases[k], precision=sisph.MIXED)
        solo.step(2)
        for f in ("x", "y", "u", "v", "p"):
            assert np.array_equal(batch.get(f)[offs[k]:offs[k + 1]], solo.get(f)), (k, f)
        assert bst[k].total_iters == solo.stats()[0].total_iters
        solo.close()
    batch.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["db2d", "ldc", "tgv_perturbed", "db3d"])
def test_sweep_sync_forms_agree(sisph, prec, name):
    """Point-to-point sweeps (per-tile flags, decisions one sweep behind) and
    the grid-barrier form give the same pressures and sweep counts."""
    case = CASES[name]
    out = []
    for sync in (2, 1):
        sim = sisph.Simulation(case, precision=prec, ppe_sync=sync)
        sim.step(4)
        out.append(({f: sim.get(f) for f in ("x", "y", "u", "v", "p")}, sim.stats()[0].total_iters))
        sim.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    for f in a:
        assert np.array_equal(a[f], b[f]), f


def test_sweep_sync_forms_agree_with_an_empty_case(sisph):
    tank = workloads.still_tank_2d(6, 6, dx=0.1)
    walls = {k: (v[tank["kind"] == 1] if isinstance(v, np.ndarray) and v.shape == (tank["n"],) else v)
             for k, v in tank.items()}
    walls["n"] = int(np.sum(tank["kind"] == 1))
    cases = [workloads.taylor_green(20, tol=1e-2), walls, workloads.dam_break_2d(dx=0.05)]
    res = []
    for sync in (2, 1):
        sim = sisph.Simulation(cases, ppe_sync=sync)
        sim.step(3)
        res.append((sim.get("p"), [(s.iters, s.solves) for s in sim.stats()]))
        sim.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_sync_forms_agree_on_a_3d_batch(sisph, prec):
    """Two 3D dam breaks in one handle, the second at a tight tolerance: once
    the first stops, the barrier form finishes the second in its per-case
    tail (the 3D batch kernel); both sync forms give the same bits and the
    same sweep counts."""
    def cases():
        a = workloads.dam_break_3d(dx=0.07)
        b = workloads.dam_break_3d(dx=0.06)
        b["params"]["tol"] = 1e-5
        return [a, b]
    out = []
    for sync in (2, 1):
        sim = sisph.Simulation(cases(), precision=prec, ppe_sync=sync)
        sim.step(2)
        out.append(({f: sim.get(f) for f in ("x", "y", "z", "u", "v", "w", "p")},
                    [(s.iters, s.total_iters) for s in sim.stats()]))
        sim.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    assert ib[1][0] > ib[0][0]          # the tight case swept on alone
    for f in a:
        assert np.array_equal(a[f], b[f]), f


def test_sweep_sync_forms_agree_when_a_case_stops_at_max_iter(sisph):
    """A batch whose cavity cannot reach its tolerance: the vortex stops
    after its 2 sweeps, so the barrier form finishes the cavity in its
    per-case tail, where it stops at max_iter (SISPH_ENOTCONVERGED, which a
    step reports and carries on from); both sync forms give the same bits
    and the same sweep counts."""
    def cases():
        cav = workloads.lid_driven_cavity(30)
        cav["params"]["tol"] = 1e-14
        cav["params"]["max_iter"] = 7
        return [workloads.taylor_green(24, tol=1e-2), cav, workloads.dam_break_2d(dx=0.05)]
    res = []
    for sync in (2, 1):
        sim = sisph.Simulation(cases(), ppe_sync=sync)
        sim.step(2)
        st = sim.stats()
        res.append((sim.get("p"), sim.get("u"), [(s.iters, s.total_iters, s.status) for s in st]))
        sim.close()
    assert res[0][2] == res[1][2]
    assert res[1][2][1][0] == 7 and res[1][2][1][2] == sisph.ENOTCONVERGED
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_direct(sisph, prec):
    case = workloads.lid_driven_cavity(24)
    a = sisph.Simulation(case, precision=prec, use_graph=1)
    b = sisph.Simulation(case, precision=prec, use_graph=0)
    a.step(3)
    b.step(3)
    a.step(2)
    b.step(2)
    for f in ("x", "y", "u", "v", "p"):
        assert np.array_equal(a.get(f), b.get(f)), f
    a.close()
    b.close()


def test_checkpoint_resumes_bit_identically(sisph, tmp_path):
    case = workloads.lid_driven_cavity(20)
    a = sisph.Simulation(case, precision=sisph.MIXED)
    a.step(3)
    path = tmp_path / "ck.bin"
    sisph.sisph_save(a.h, path)
    a.step(3)
    b = sisph.Simulation(case, precision=sisph.MIXED)
    sisph.sisph_load(b.h, path)
    b.step(3)
    for f in ("x", "y", "u", "v", "p", "ut", "vt"):
        assert np.array_equal(a.get(f), b.get(f)), f
    a.close()
    b.close()


def test_eisph_single_sweep_matches_oracle(sisph):
    # EISPH (Sec. 4.2): the same PPE with a single Jacobi iteration per step
    case = with_params(workloads.taylor_green(40, perturb=0.05), max_iter=1)
    sim = sisph.Simulation(case, min_iter=1)
    ref = oracle.Sim(case, min_iter=1)
    for _ in range(3):
        rc = sim.step(1)
        ref.step(1)
        st = sim.stats()[0]
        assert st.iters == 1
    for f in ("x", "y", "u", "v", "p"):
        assert relerr(sim.get(f), ref.get(f)) < FP64_TOL, f
    sim.close()
