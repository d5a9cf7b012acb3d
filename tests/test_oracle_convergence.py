"""Pins of the oracle's convergence test (Sec. 3, Eq. convergence) and of the
external-flow background pressure (Sec. 2.2, the text after Eq. mom:sph:gtvf).

Eq. convergence, as read here:
    res = sum_i |p_i^{k+1} - p_i^k| / max(Lambda, sum_i |p_i^{k+1}|),
    Lambda = max_i |RHS_i / D_ii|,
with both sums over the fluid rows and Lambda over the active fluid rows
(not on the free surface, D_ii != 0); the sweeps go on while k < min_iter or
res >= eps, and stop at max_iter.

* One sweep from p = 0 without gravity moves nothing but the source:
  p^1 = omega RHS / D exactly, so the residual has a closed form in the
  exported RHS and D: omega sum|RHS/D| / Lambda when Lambda is the larger
  term, exactly 1 when sum|p^1| is.  The input makes every plausible slip
  change that number: the largest |RHS/D| of the active rows is negative
  (Lambda without the absolute value differs), a free-surface row carries a
  larger |RHS/D| than any active row (counting it in Lambda differs), and
  Lambda < 1 (the algorithm listing's max(1, .) differs).
* With gravity and a hydrostatic start the walls carry pressure, and the
  residual of every sweep is recomputed from the fluid pressures of two
  successive sweeps (counting the walls in the sums differs).
* The solve stops at the first k >= 2 whose residual is below eps.
* The external background pressure p0_i = min(10 |p_i|, p_ref) makes the
  GTVF force on particle i proportional to min(|s|, 1) when p_i = s p_ref/10,
  and the internal-flow p_ref makes it independent of p_i.
"""
import numpy as np
import pytest

import oracle
import workloads


def _tank(g=True, seed=4):
    """A 12 x 12 still tank (3 wall layers), rho = rho0 everywhere, so every
    fluid row is active unless its density is lowered below 0.8 rho0."""
    c = workloads.still_tank_2d(12, 12, dx=0.1)
    if not g:
        c["params"] = dict(c["params"], g=(0.0, 0.0, 0.0))
        c["p"][:] = 0.0
    c["rho"][:] = c["params"]["rho0"]
    return c


def _source_case():
    """No gravity, p = 0; the fluid particles within 1.5 h of one particle q
    move away from it (u* = U e_jq), and q sits on the free surface
    (rho_q = 0.79 rho0)."""
    c = _tank(g=False)
    fl = np.nonzero(c["kind"] == 0)[0]
    h = c["params"]["h"]
    cx, cy = 0.55, 0.65
    q = fl[np.argmin((c["x"][fl] - cx) ** 2 + (c["y"][fl] - cy) ** 2)]
    dx, dy = c["x"] - c["x"][q], c["y"] - c["y"][q]
    r = np.hypot(dx, dy)
    near = (c["kind"] == 0) & (r < 1.5 * h) & (r > 0)
    U = 1e-5
    c["u"] = np.where(near, U * dx / np.where(r > 0, r, 1), 0.0)
    c["v"] = np.where(near, U * dy / np.where(r > 0, r, 1), 0.0)
    c["rho"][q] = 0.79 * c["params"]["rho0"]
    return c, q


def _one_sweep(c, **over):
    s = oracle.Sim(c, **over)
    rc, d = s.ppe_solve(0.0, 1)
    assert d.iters == 1
    return s, d


@pytest.mark.parametrize("residual_form", [0, 1])
@pytest.mark.parametrize("omega", [0.02, 0.5])
def test_first_sweep_residual_closed_form(oracle_lib, omega, residual_form):
    c, q = _source_case()
    s, d = _one_sweep(c, omega=omega, residual_form=residual_form)
    ex = s.ppe_export()
    fl = c["kind"] == 0
    act = fl & (ex["active"] == 1)
    assert not ex["active"][q] and act.sum() == fl.sum() - 1
    ratio = np.zeros(c["n"])
    ratio[act] = ex["rhs"][act] / ex["diag"][act]
    p1 = s.get("p")
    # no pressure anywhere before the sweep and no gravity: p^1 = omega RHS/D
    assert np.array_equal(p1[act], omega * ex["rhs"][act] / ex["diag"][act])
    assert p1[q] == 0.0
    lam = np.max(np.abs(ratio[act]))
    assert d.lambda_ == lam
    # the input is built so that each misreading would change the result
    assert abs(ex["rhs"][q] / ex["diag"][q]) > 1.2 * lam          # free-surface row dominates
    assert np.max(ratio[act]) < 0.9 * lam                         # the largest |RHS/D| is negative
    assert lam < 0.5                                              # below the listing's max(1, .)
    tot = np.sum(np.abs(p1[fl]))
    lam_d = fl.sum() * lam if residual_form == 1 else lam
    if lam_d > tot:
        expect = omega * np.sum(np.abs(ratio[act])) / lam_d
        assert expect < 0.9
    else:
        expect = 1.0
        assert tot < 0.5
    assert d.residual == pytest.approx(expect, rel=1e-13)


def test_first_sweep_takes_both_branches(oracle_lib):
    """The two omega values of the closed-form test put Lambda and sum|p^1|
    on either side of each other, so both branches of the max are pinned."""
    c, q = _source_case()
    branch = []
    for omega in (0.02, 0.5):
        s, d = _one_sweep(c, omega=omega)
        fl = c["kind"] == 0
        branch.append(d.lambda_ > np.sum(np.abs(s.get("p")[fl])))
    assert branch == [True, False]


def _sweeps(c, k, **over):
    s = oracle.Sim(c, **over)
    rc, d = s.ppe_solve(0.0, k)
    assert d.iters == k
    return s, d


def _hydro_case():
    c = _tank(g=True)
    rng = np.random.Generator(np.random.PCG64(31))
    fl = c["kind"] == 0
    c["u"] = np.where(fl, rng.normal(0, 0.05, c["n"]), 0.0)
    c["v"] = np.where(fl, rng.normal(0, 0.05, c["n"]), 0.0)
    return c


def test_residual_of_later_sweeps_from_two_pressures(oracle_lib):
    c = _hydro_case()
    fl = c["kind"] == 0
    walls = c["kind"] == 1
    prev = c["p"].copy()
    for k in range(1, 5):
        s, d = _sweeps(c, k)
        ex = s.ppe_export()
        act = fl & (ex["active"] == 1)
        lam = np.max(np.abs(ex["rhs"][act] / ex["diag"][act]))
        p = s.get("p")
        num = np.sum(np.abs(p[fl] - prev[fl]))
        den = np.sum(np.abs(p[fl]))
        assert den > lam                     # the sum|p| branch
        assert np.sum(np.abs(p[walls])) > 0.05 * den      # walls carry pressure
        assert d.residual == pytest.approx(num / max(lam, den), rel=1e-12)
        prev = p


def test_stop_at_first_sweep_below_tolerance(oracle_lib):
    c = _hydro_case()
    res = [None] + [_sweeps(c, k)[1].residual for k in range(1, 13)]
    # eps above the first residual: min_iter = 2 still takes two sweeps
    tols = [1.5 * res[1] + 1.0]
    for k in range(2, 12):
        if res[k + 1] < res[k]:
            tols.append(0.5 * (res[k] + res[k + 1]))
    assert len(tols) >= 4
    for eps in tols:
        want = next(k for k in range(2, 13) if res[k] < eps)
        s = oracle.Sim(c)
        rc, d = s.ppe_solve(eps, 1000)
        assert d.converged == 1
        assert d.iters == want
        assert d.residual == res[want]


@pytest.mark.parametrize("mistake", [16, 17, 18, 19, 20])
def test_planted_convergence_mistakes_are_caught(oracle_lib, mistake):
    """Each of these misreadings of Eq. convergence or of the loop test fails
    at least one of the pins above."""
    tests = [lambda: test_first_sweep_residual_closed_form(oracle_lib, 0.02, 0),
             lambda: test_first_sweep_residual_closed_form(oracle_lib, 0.5, 0),
             lambda: test_residual_of_later_sweeps_from_two_pressures(oracle_lib),
             lambda: test_stop_at_first_sweep_below_tolerance(oracle_lib)]
    oracle.plant_mistake(mistake)
    failed = 0
    try:
        for t in tests:
            try:
                t()
            except AssertionError:
                failed += 1
    finally:
        oracle.plant_mistake(0)
    assert failed > 0


# ---- external-flow background pressure (Sec. 2.2) --------------------------

def _gtvf_force(pref_mode, s_val, which):
    """GTVF force on particle `which` of a free 10 x 10 block (no walls) with
    p_which = s_val p_ref / 10 and p = 0 elsewhere."""
    c = workloads.taylor_green(10)
    c["periodic"] = (0, 0, 0)
    c["lo"] = (-1.0, -1.0, 0.0)
    c["hi"] = (2.0, 2.0, 1.0)
    c["rho"][:] = 1.0
    p_ref = 50.0
    c["p"][:] = 0.0
    c["p"][which] = s_val * p_ref / 10.0
    c["params"] = dict(c["params"], pref_mode=pref_mode, p_ref=p_ref, gtvf_hfac=0.5)
    s = oracle.Sim(c)
    s.build_neighbors()
    s.gtvf()
    return np.array([s.get("fx")[which], s.get("fy")[which]])


def test_external_background_pressure_rule(oracle_lib):
    corner = 0                     # (0.05, 0.05): its neighbourhood is one-sided
    ref = _gtvf_force(workloads.PREF_EXTERNAL, 5.0, corner)
    assert np.linalg.norm(ref) > 0
    for s_val, scale in [(0.1, 0.1), (0.5, 0.5), (-0.5, 0.5), (1.0, 1.0), (2.0, 1.0), (-7.0, 1.0)]:
        f = _gtvf_force(workloads.PREF_EXTERNAL, s_val, corner)
        assert np.allclose(f, scale * ref, rtol=1e-13, atol=0), (s_val, f, ref)
    # internal flows: p0 = p_ref whatever p_i is
    a = _gtvf_force(workloads.PREF_FIXED, 0.1, corner)
    b = _gtvf_force(workloads.PREF_FIXED, -3.0, corner)
    assert np.array_equal(a, b) and np.allclose(a, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("mistake", [21, 22])
def test_planted_background_pressure_mistakes_are_caught(oracle_lib, mistake):
    oracle.plant_mistake(mistake)
    try:
        with pytest.raises(AssertionError):
            test_external_background_pressure_rule(oracle_lib)
    finally:
        oracle.plant_mistake(0)
