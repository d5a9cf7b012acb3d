"""Physics pins of the oracle's whole time step (Algorithm 1).

* hydrostatics: a still tank keeps p = rho0 g (H - y) (Sec. 3.4, Eq.
  p-shepard builds the wall pressure to reproduce it);
* Taylor-Green vortex: max|u| and the kinetic energy decay as exp(b t),
  exp(2 b t), b = -8 pi^2 / Re (Eq. tgv), over 40 steps of the 50 x 50 lattice;
* pairwise antisymmetry: the "symm" pressure gradient and the viscous force
  conserve momentum in a periodic box (Eqs. mom:sph:press:symm, mom:sph:visc);
* GTVF sub-steps: with K = 1 the displacement is dt^2/2 f(r*) exactly, and
  K sub-steps agree with K = 1 to higher order (Eqs. int:gtvf:pos, :vel:tmp);
* wall normals of a flat wall point out of the solid (Sec. 3.4.1).
Planted mistakes in the oracle show that each pin bites.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

RHO0, G = 1000.0, 9.81


def _hydro_error(s, c):
    p = s.get("p"); y = s.get("y"); x = s.get("x")
    h = c["params"]["h"]
    H = 20 * 0.05
    fl = c["kind"] == 0
    sel = fl & (y > 3 * h) & (y < H - 3 * h) & (x > 3 * h) & (x < 1 - 3 * h)
    ex = RHO0 * G * (H - y[sel])
    return np.abs(p[sel] - ex).sum() / np.abs(ex).sum()


def test_hydrostatic_tank(oracle_lib):
    c = workloads.still_tank_2d(20, 20)
    s = oracle.Sim(c)
    s.step(1)
    assert _hydro_error(s, c) < 0.05
    s.step(49)
    assert _hydro_error(s, c) < 0.05
    fl = c["kind"] == 0
    assert np.abs(s.get("v")[fl]).max() < 0.1 * math.sqrt(2 * G * 1.0)


def test_planted_wall_sign_breaks_hydrostatics(oracle_lib):
    c = workloads.still_tank_2d(20, 20)
    oracle.plant_mistake(3)
    try:
        s = oracle.Sim(c)
        s.step(1)
        err = _hydro_error(s, c)
    finally:
        oracle.plant_mistake(0)
    assert err > 0.05


def _tgv_run(plant=0, nsteps=40):
    c = workloads.taylor_green(50)
    oracle.plant_mistake(plant)
    umax = []
    l1_10 = None
    try:
        s = oracle.Sim(c)
        for k in range(nsteps):
            rc, ds = s.step(1)
            umax.append(ds[0].umax)
            if k == 9:
                tt = 10 * c["params"]["dt"]
                ue, ve, _ = workloads.tgv_exact(s.get("x"), s.get("y"), tt)
                l1_10 = np.sum(np.abs(np.hypot(s.get("u"), s.get("v")) - np.hypot(ue, ve))) / \
                    np.sum(np.hypot(ue, ve))
            if not np.isfinite(ds[0].umax) or ds[0].umax > 10:
                break
    finally:
        oracle.plant_mistake(0)
    t = len(umax) * c["params"]["dt"]
    e0 = np.sum(c["m"] * (c["u"] ** 2 + c["v"] ** 2))
    e1 = np.sum(c["m"] * (s.get("u") ** 2 + s.get("v") ** 2))
    # kinetic energy of the exact field decays as exp(2 b t)
    s.l1_10 = l1_10
    return c, s, t, math.log(e1 / e0) / (2 * t), np.array(umax)


def test_tgv_decay_rate(oracle_lib):
    b = -8 * math.pi ** 2 / 100.0
    c, s, t, rate, umax = _tgv_run()
    dt = c["params"]["dt"]
    assert umax.size == 40
    # energy decay rate over 40 steps (t = 0.2)
    assert abs(rate - b) < 0.05 * abs(b)
    # max|u| follows U exp(b t) (U = the lattice maximum at t = 0) within 3 %
    u0 = np.hypot(c["u"], c["v"]).max()
    tk = dt * np.arange(1, 41)
    assert np.max(np.abs(umax / (u0 * np.exp(b * tk)) - 1)) < 0.03
    # L1 error of |u| against the exact field at the particle positions, t = 0.05
    assert s.l1_10 < 0.02
    # background pressure: twice the maximum pressure after the first solve
    assert 0.5 < s.p_ref < 2.0


@pytest.mark.parametrize("plant", [4, 6])
def test_planted_tgv_mistakes_are_caught(oracle_lib, plant):
    b = -8 * math.pi ** 2 / 100.0
    c, s, t, rate, umax = _tgv_run(plant)
    assert not (abs(rate - b) < 0.05 * abs(b) and umax.size == 40)


def _random_periodic(seed):
    c = workloads.taylor_green(24, perturb=0.25, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    c["rho"] = rng.uniform(0.9, 1.1, c["n"])
    c["p"] = rng.normal(0, 1, c["n"])
    c["u"] = rng.normal(0, 1, c["n"])
    c["v"] = rng.normal(0, 1, c["n"])
    return c


def test_symm_pressure_gradient_conserves_momentum(oracle_lib):
    c = _random_periodic(21)
    s = oracle.Sim(c, pgrad_symm=1)
    s.pressure_gradient()
    m = c["m"]
    fx, fy = s.get("fx"), s.get("fy")
    assert abs(np.sum(m * fx)) < 1e-12 * np.sum(m * np.abs(fx))
    assert abs(np.sum(m * fy)) < 1e-12 * np.sum(m * np.abs(fy))
    # the "asymm" form does not conserve momentum for a random field
    s2 = oracle.Sim(c, pgrad_symm=0)
    s2.pressure_gradient()
    assert abs(np.sum(m * s2.get("fx"))) > 1e-6 * np.sum(m * np.abs(s2.get("fx")))


def test_viscous_force_conserves_momentum(oracle_lib):
    c = _random_periodic(22)
    s = oracle.Sim(c, p_ref=0.0)
    # transport velocity equal to u switches the artificial stress off
    s.set("ut", s.get("u")); s.set("vt", s.get("v"))
    s.stage1()
    m = c["m"]
    fx, fy = s.get("fx"), s.get("fy")
    assert abs(np.sum(m * fx)) < 1e-12 * np.sum(m * np.abs(fx))
    assert abs(np.sum(m * fy)) < 1e-12 * np.sum(m * np.abs(fy))


def test_gtvf_single_substep_closed_form(oracle_lib):
    c = _random_periodic(23)
    c["p"] = np.abs(c["p"])
    s = oracle.Sim(c, gtvf_K=1, pref_mode=2, p_ref=50.0)
    s.gtvf()
    dt = c["params"]["dt"]
    for a, f in (("dx", "fx"), ("dy", "fy")):
        d, force = s.get(a), s.get(f)
        assert np.array_equal(d, 0.5 * dt * dt * force)
    assert np.abs(s.get("fx")).max() > 0


def test_gtvf_substeps_agree_to_higher_order(oracle_lib):
    # With a constant force the K sub-steps give dt^2/2 f for every K; the
    # force here changes only through the sub-step motion, so the relative
    # K=4 vs K=1 difference shrinks in proportion to the displacement.
    c = _random_periodic(24)
    rel = []
    for pref in (1.0, 0.1):
        s1 = oracle.Sim(c, gtvf_K=1, p_ref=pref)
        s1.gtvf()
        s4 = oracle.Sim(c, gtvf_K=4, p_ref=pref)
        s4.gtvf()
        d1 = np.stack([s1.get("dx"), s1.get("dy")])
        d4 = np.stack([s4.get("dx"), s4.get("dy")])
        assert np.abs(d1).max() > 0
        rel.append(np.abs(d4 - d1).max() / np.abs(d1).max())
    assert rel[0] < 1e-2
    assert 0.05 < rel[1] / rel[0] < 0.2


def test_flat_wall_normals(oracle_lib):
    c = workloads.still_tank_2d(12, 12, dx=0.1)
    s = oracle.Sim(c)
    nx, ny = s.get("nx"), s.get("ny")
    x, y = c["x"], c["y"]
    wall = c["kind"] == 1
    # first bottom layer away from the corners: normal +y, out of the solid
    bottom = wall & np.isclose(y, -0.05) & (x > 0.4) & (x < 0.8)
    assert bottom.sum() > 0
    assert np.allclose(ny[bottom], 1.0) and np.allclose(nx[bottom], 0.0, atol=1e-12)
    left = wall & np.isclose(x, -0.05) & (y > 0.4) & (y < 0.8)
    assert np.allclose(nx[left], 1.0) and np.allclose(ny[left], 0.0, atol=1e-12)
    assert np.all(nx[~wall] == 0) and np.all(ny[~wall] == 0)
    mag = np.hypot(nx, ny)
    assert np.all((np.abs(mag - 1) < 1e-12) | (mag == 0))


def _layer_normals():
    # resting tank with three wall layers (dx = 0.1): the bottom layers sit at
    # y = -0.05, -0.15, -0.25 and the left ones at x = -0.05, -0.15, -0.25
    c = workloads.still_tank_2d(12, 12, dx=0.1)
    s = oracle.Sim(c)
    x, y, wall = c["x"], c["y"], c["kind"] == 1
    mid = (x > 0.4) & (x < 0.8)
    layer = {k: wall & np.isclose(y, yy) & mid for k, yy in (("inner", -0.05), ("middle", -0.15), ("outer", -0.25))}
    corner = wall & np.isclose(x, -0.05) & np.isclose(y, -0.05)
    return s.get("nx"), s.get("ny"), layer, corner


def _check_layer_normals(nx, ny, layer, corner):
    # the middle layer sees one layer on either side at the same distance: its
    # raw gradient sum cancels (below the zero threshold) and so does the
    # smoothed sum of the inner (+y) and outer (-y) normals, so it has none
    assert np.all(nx[layer["middle"]] == 0.0) and np.all(ny[layer["middle"]] == 0.0)
    # the inner layer points into the tank, the outer layer away from the solid
    assert np.allclose(ny[layer["inner"]], 1.0, rtol=0, atol=1e-12)
    assert np.allclose(ny[layer["outer"]], -1.0, rtol=0, atol=1e-12)
    # the inner corner particle is symmetric about the diagonal: the bisector
    assert corner.sum() == 1
    assert np.allclose(nx[corner], math.sqrt(0.5), rtol=0, atol=1e-12)
    assert np.allclose(ny[corner], math.sqrt(0.5), rtol=0, atol=1e-12)


def test_wall_normals_of_symmetric_layers(oracle_lib):
    """Eqs. normal-approx, normal: geometry fixes the normals of a three-layer
    wall -- none on the middle layer, whose neighbourhood is symmetric, +-y on
    the inner and outer layers, the diagonal at the inner corner."""
    _check_layer_normals(*_layer_normals())


@pytest.mark.parametrize("plant", [9, 10])
def test_planted_normal_thresholds_are_caught(oracle_lib, plant):
    # 9: the smoothed normal normalised however small; 10: the raw one
    oracle.plant_mistake(plant)
    with pytest.raises(AssertionError):
        _check_layer_normals(*_layer_normals())


def test_adaptive_time_step_in_free_fall(oracle_lib):
    """Adaptive dt (Sec. 3.2) against the closed form of a free fall: the only
    force is g, so max|f| = g and max|u^n| = g t_n.  The step after one
    starting at rest is force-limited, 0.25 sqrt(h/g); once g t_n exceeds
    sqrt(g h) the CFL limit 0.25 h/(g t_n) takes over.  The position update
    r^{n+1} = r^n + dt (u~^{n+1} + u~^n)/2 is exact for constant acceleration
    with any sequence of steps: y = y0 - g t^2 / 2."""
    import math
    case = workloads.free_fall_blob()
    h, g = case["params"]["h"], 9.81
    sim = oracle.Sim(case)
    dts, starts, t = [], [], 0.0
    for _ in range(12):
        starts.append(t)
        rc, d = sim.step(1)
        dts.append(d[0].dt)
        t += d[0].dt
    assert np.all(sim.get("p") == 0.0)
    dt_f = 0.25 * math.sqrt(h / g)
    assert dts[0] == case["params"]["dt"]
    kinds = []
    for k in range(1, len(dts)):
        t_prev = starts[k - 1]                      # u at the start of step k-1 is g t_prev
        cfl = 0.25 * h / (g * t_prev) if t_prev > 0 else math.inf
        expect = min(dt_f, cfl)
        kinds.append("cfl" if cfl < dt_f else "force")
        assert abs(dts[k] - expect) <= 1e-12 * expect, (k, dts[k], expect)
    assert "cfl" in kinds and "force" in kinds      # both limits were exercised
    assert np.allclose(sim.get("v"), -g * t, rtol=1e-12, atol=0)
    assert np.allclose(sim.get("y"), case["y"] - 0.5 * g * t * t, rtol=0, atol=1e-12)
    assert np.allclose(sim.get("x"), case["x"], rtol=0, atol=1e-15)


def test_adaptive_time_step_tgv_first_step_is_cfl(oracle_lib):
    """TGV: the step after step 0 follows the CFL limit of the initial speed
    field, 0.25 h / max|u^0| (max over the lattice from the initial
    condition), which is below the force and viscous limits here."""
    case = workloads.taylor_green(50)
    case["params"] = dict(case["params"], adaptive_dt=1)
    sim = oracle.Sim(case)
    rc, d = sim.step(2)
    umax0 = float(np.max(np.hypot(case["u"], case["v"])))
    h = case["params"]["h"]
    assert d[0].dt == case["params"]["dt"]
    assert abs(d[1].dt - 0.25 * h / umax0) <= 1e-13 * d[1].dt
    assert d[1].dt < 0.25 * h * h / case["params"]["nu"]


def _moving_block(a, seed):
    """A 12 x 12 block of fluid at lattice spacing (slightly perturbed) in an
    open box, no walls, velocity u = a (r - r_c): dilating for a > 0."""
    c = workloads.free_fall_blob(n_side=12, dx=0.05, spacing=1.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    c["x"] = c["x"] + rng.uniform(-0.005, 0.005, c["n"])
    c["y"] = c["y"] + rng.uniform(-0.005, 0.005, c["n"])
    xc, yc = c["x"].mean(), c["y"].mean()
    c["u"] = a * (c["x"] - xc)
    c["v"] = a * (c["y"] - yc)
    return c, xc, yc


def _avisc_only(c, **over):
    # no viscosity, no gravity, transport velocity = u (no artificial stress):
    # stage 1's force is the artificial viscosity alone
    s = oracle.Sim(c, nu=0.0, g=(0.0, 0.0, 0.0), alpha=1.0, c0=10.0, adaptive_dt=0, **over)
    s.set("ut", s.get("u"))
    s.set("vt", s.get("v"))
    s.stage1()
    return s.get("fx"), s.get("fy")


def test_artificial_viscosity_conserves_momentum(oracle_lib):
    c = _random_periodic(24)
    c["params"] = dict(c["params"], adaptive_dt=0)
    fx, fy = _avisc_only(c)
    m = c["m"]
    assert np.abs(fx).max() > 0
    assert abs(np.sum(m * fx)) < 1e-12 * np.sum(m * np.abs(fx))
    assert abs(np.sum(m * fy)) < 1e-12 * np.sum(m * np.abs(fy))


@pytest.mark.parametrize("plant", [0, 7, 8])
def test_artificial_viscosity_acts_only_against_compression(oracle_lib, plant):
    oracle.plant_mistake(plant)
    try:
        # dilation: every pair recedes (u_ij . r_ij > 0), no force at all
        c, xc, yc = _moving_block(0.5, 31)
        fx, fy = _avisc_only(c)
        dilation_free = np.abs(fx).max() == 0.0 and np.abs(fy).max() == 0.0
        # compression: the force pushes the particles apart (outward)
        c, xc, yc = _moving_block(-0.5, 32)
        fx, fy = _avisc_only(c)
        outward = np.sum(fx * (c["x"] - xc) + fy * (c["y"] - yc))
    finally:
        oracle.plant_mistake(0)
    if plant == 0:
        assert dilation_free and outward > 0
    else:
        # 7 lets receding pairs feel it, 8 turns its sign
        assert not (dilation_free and outward > 0)


def _tank_density():
    # resting tank: fluid lattice continued by three wall layers on the same
    # lattice (m_w = rho0 dx^2); every fluid particle whose support stays
    # below the free surface sees a complete lattice, walls included
    c = workloads.still_tank_2d(16, 16)
    s = oracle.Sim(c)
    s.density()
    rho = s.get("rho") / c["params"]["rho0"]
    fl = c["kind"] == 0
    h = c["params"]["h"]
    deep = fl & (c["y"] < c["y"][fl].max() - 3 * h)
    near_wall = deep & ((c["y"] < 3 * h) | (c["x"] < 3 * h))
    return rho, deep, near_wall


@pytest.mark.parametrize("plant", [0, 13])
def test_summation_density_of_a_lattice_with_walls(oracle_lib, plant):
    """Eq. summation_density over fluid and wall neighbours (reading 9): on a
    lattice the sum is rho0 times the lattice partition of unity, 1.00006322
    for the 2D quintic at h = dx, also next to the walls."""
    oracle.plant_mistake(plant)
    try:
        rho, deep, near_wall = _tank_density()
    finally:
        oracle.plant_mistake(0)
    assert near_wall.sum() > 20
    ok = np.allclose(rho[deep], 1.00006322, rtol=0, atol=1e-8)
    # 13 leaves the walls out of the fluid's sums
    assert ok == (plant == 0)


@pytest.mark.parametrize("plant", [0, 14])
def test_free_surface_particles_keep_zero_pressure(oracle_lib, plant):
    """Sec. 3: fluid below 0.8 rho0 (the top rows of a resting tank, whose
    support reaches above the surface) is a Dirichlet row p = 0 -- the
    surface value of the hydrostatic p = rho0 g (H - y) -- while the deep
    fluid carries the hydrostatic pressure."""
    c = workloads.still_tank_2d(16, 16)
    oracle.plant_mistake(plant)
    try:
        s = oracle.Sim(c)
        s.density()
        s.ppe_solve(1e-6, 5000)
        p, rho = s.get("p"), s.get("rho") / c["params"]["rho0"]
    finally:
        oracle.plant_mistake(0)
    fl = c["kind"] == 0
    top = fl & (rho < 0.8)
    h = c["params"]["h"]
    deep = fl & (c["y"] < c["y"][fl].max() - 3 * h)
    assert 16 <= top.sum() <= 48 and deep.sum() > 150
    ok = np.all(p[top] == 0.0) and np.all(p[deep] > 0.0)
    # 14 solves the surface rows like interior ones
    assert ok == (plant == 0)


@pytest.mark.parametrize("plant", [0, 15])
def test_reference_pressure_of_the_taylor_green_vortex(oracle_lib, plant):
    """Internal flows take p_ref = 2 max_i p_i from the first solve and keep
    it (reading 16).  The vortex's pressure -rho U^2/4 (cos 4 pi x + cos 4 pi y)
    e^{2bt} peaks at rho U^2 / 2, so p_ref is rho U^2 = 1 to the method's
    accuracy after one step."""
    c = workloads.taylor_green(50)
    oracle.plant_mistake(plant)
    try:
        s = oracle.Sim(c)
        s.step(1)
        p1 = s.p_ref
        s.step(1)
        p2 = s.p_ref
    finally:
        oracle.plant_mistake(0)
    assert abs(p1 - 1.0) < 0.01
    # 15 takes p_ref again after every solve
    assert (p2 == p1) == (plant == 0)


def _astress_only(c, ut, vt):
    # no viscosity, no artificial viscosity, no gravity: stage 1's force is the
    # artificial stress alone (Eq. mom:sph:gtvf:stress)
    s = oracle.Sim(c, nu=0.0, g=(0.0, 0.0, 0.0), alpha=0.0, adaptive_dt=0)
    s.set("ut", ut)
    s.set("vt", vt)
    s.stage1()
    return s.get("fx"), s.get("fy")


def _stress_of_a_linear_field():
    """A 24 x 24 lattice block (h = dx, uniform rho), u = (U, 0) and
    u~ - u = (0, beta y): A = rho u (x) (u~ - u) has the one entry
    A_xy = rho U beta y, so (1/rho) div A = (U beta, 0).  The symmetric SPH
    form is that divergence for particles whose support lies inside the
    block."""
    U, beta = 0.7, 3.0
    c = workloads.free_fall_blob(n_side=24, dx=0.05, spacing=1.0, adaptive=False)
    c["u"] = np.full(c["n"], U)
    c["v"] = np.zeros(c["n"])
    yc = c["y"].mean()
    fx, fy = _astress_only(c, c["u"], beta * (c["y"] - yc))
    h = c["params"]["h"]
    x, y = c["x"], c["y"]
    inner = ((x - x.min() > 6 * h) & (x.max() - x > 6 * h) & (y - y.min() > 6 * h)
             & (y.max() - y > 6 * h))
    assert inner.sum() >= 100
    return fx[inner], fy[inner], U * beta


@pytest.mark.parametrize("plant", [0, 11, 12])
def test_artificial_stress_of_a_linear_field(oracle_lib, plant):
    oracle.plant_mistake(plant)
    try:
        fx, fy, expect = _stress_of_a_linear_field()
    finally:
        oracle.plant_mistake(0)
    ok = np.allclose(fx, expect, rtol=2e-3, atol=0) and np.all(fy == 0.0)
    # 11 transposes the tensor (u~ - u) (x) u, 12 drops the neighbour's A_j
    assert ok == (plant == 0)


def test_artificial_stress_conserves_momentum(oracle_lib):
    c = _random_periodic(25)
    c["params"] = dict(c["params"], adaptive_dt=0)
    rng = np.random.Generator(np.random.PCG64(26))
    fx, fy = _astress_only(c, c["u"] + rng.normal(0, 0.3, c["n"]), c["v"] + rng.normal(0, 0.3, c["n"]))
    m = c["m"]
    assert np.abs(fx).max() > 0
    assert abs(np.sum(m * fx)) < 1e-12 * np.sum(m * np.abs(fx))
    assert abs(np.sum(m * fy)) < 1e-12 * np.sum(m * np.abs(fy))


@pytest.mark.parametrize("slip", [0, 1])
def test_ghost_velocity_of_a_uniform_flow(oracle_lib, slip):
    # fluid moving uniformly along the bottom wall of the still tank, U =
    # (0.3, 0).  Slip form: the fluid's own velocity extended into the wall,
    # so every wall that sees fluid carries U exactly (a Shepard mean of a
    # constant).  No-slip form on the bottom wall away from the corners
    # (normal +y, U tangential): 2 u_wall - U = -U, nothing into the solid.
    # A wall with no fluid within the kernel's reach keeps u_wall = 0.
    c = workloads.still_tank_2d(20, 20)
    fl = c["kind"] == 0
    c["u"] = np.where(fl, 0.3, 0.0)
    c["v"] = np.zeros(c["n"])
    s = oracle.Sim(c)
    s.build_neighbors()
    s.wall_normals()
    s.ghost_velocity(slip)
    ug, vg = s.get("ugx"), s.get("ugy")
    h = c["params"]["h"]
    reach = 3.0 * (h if slip else 0.5 * h)      # support of the Shepard kernel
    pos = np.stack([c["x"], c["y"]], 1)
    fpos = pos[fl]
    dmin = np.array([np.sqrt(np.min(np.sum((fpos - p) ** 2, axis=1))) for p in pos])
    walls = ~fl
    sees = walls & (dmin < 0.99 * reach)
    none = walls & (dmin >= reach)
    assert np.count_nonzero(sees) > 20 and np.count_nonzero(none) > 5
    if slip:
        pick = sees
        expect = 0.3
    else:
        pick = sees & (c["y"] < 0) & (c["x"] > 0.3) & (c["x"] < 0.7)
        expect = -0.3
        assert np.count_nonzero(pick) > 5
    assert np.allclose(ug[pick], expect, rtol=0, atol=1e-12)
    assert np.allclose(vg[pick], 0.0, rtol=0, atol=1e-12)
    assert np.all(ug[none] == 0.0) and np.all(vg[none] == 0.0)
