"""Seeded synthetic particle sets shaped like the SISPH paper's test problems.

This module only *generates inputs*: lattice positions, initial fields, masses,
particle kinds, domain bounds and the per-case physical parameters that the
paper states for each problem.  It contains none of the scheme's arithmetic (no
kernel, no neighbour sums, no pressure solve) and imports nothing from either
the CUDA package or the CPU oracle, so both sides can be fed the same arrays.

Problems (paper section in brackets):
  * Taylor-Green vortex, periodic unit square            [Sec. 4.1, Eq. tgv]
  * lid-driven cavity, unit square with 3 wall layers     [Sec. 4.2]
  * 2D dam break, 1 x 2 m column in a 4 x 4 m tank        [Sec. 4.4]
  * 3D dam break, 0.55 x 1.0 x 0.55 m column in a tank    [Sec. 4.5]
  * a seeded batch of uneven TGV / cavity cases

Every case is a plain dict of numpy arrays plus scalars; `dim`, `lo`, `hi`,
`periodic` describe the box.  Walls are `kind == 1`, fluid `kind == 0`.
Time steps follow the paper's fixed-step rule (Sec. 3.2: the minimum of the
CFL, viscous and body-force limits) or the problem-specific rule it states.
"""
from __future__ import annotations

import math

import numpy as np

FLUID = 0
WALL = 1

# p_ref / background-pressure modes (Sec. 2.1, Eq. mom:sph:gtvf and the text
# after it): a fixed value, "twice the maximum pressure after the first
# iteration" (internal flows), or p0_i = min(10|p_i|, p_ref) (external flows).
PREF_FIXED = 0
PREF_TWICE_MAX_FIRST = 1
PREF_EXTERNAL = 2


def _params(**kw):
    """Per-case physical and solver parameters with the paper's defaults."""
    base = dict(
        h=0.0, dt=0.0, rho0=1.0, nu=0.0, g=(0.0, 0.0, 0.0),
        alpha=0.0, c0=0.0,              # artificial viscosity (alpha = 0: off)
        tol=1e-2, max_iter=1000,        # PPE tolerance and cap (Listing 1)
        pgrad_symm=0,                   # 0: "asymm", 1: "symm" pressure gradient
        free_surface=0,                 # rho/rho0 < 0.8 -> p = 0 and wall clamp
        pref_mode=PREF_FIXED, p_ref=0.0,
        gtvf_hfac=1.0, gtvf_K=1,        # h~ = hfac * h, K GTVF sub-steps
        ustar_slip=1,                   # slip ghost velocity for u* in the PPE
        adaptive_dt=0,                  # 1: next dt from max|u|, max|f| (Sec. 3.2)
    )
    base.update(kw)
    base["g"] = tuple(float(v) for v in base["g"])
    return base


def fixed_dt(h, umax, nu, gmag):
    """Fixed time step of Sec. 3.2: min of the CFL, viscous and force limits."""
    cands = []
    if umax > 0:
        cands.append(0.25 * h / umax)
    if nu > 0:
        cands.append(0.25 * h * h / nu)
    if gmag > 0:
        cands.append(0.25 * math.sqrt(h / gmag))
    return min(cands)


def _lattice2(nx, ny, dx, x0=0.0, y0=0.0):
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    x = x0 + (i.ravel() + 0.5) * dx
    y = y0 + (j.ravel() + 0.5) * dx
    return x.astype(np.float64), y.astype(np.float64)


def _lattice3(nx, ny, nz, dx, x0=0.0, y0=0.0, z0=0.0):
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = x0 + (i.ravel() + 0.5) * dx
    y = y0 + (j.ravel() + 0.5) * dx
    z = z0 + (k.ravel() + 0.5) * dx
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def _case(dim, x, y, z, u, v, w, m, rho, p, kind, wall_u, lo, hi, periodic, params, name):
    n = x.size
    z = np.zeros(n) if z is None else z
    w = np.zeros(n) if w is None else w
    wall_u = np.zeros((3, n)) if wall_u is None else wall_u
    return dict(
        name=name, dim=dim, n=n,
        x=np.ascontiguousarray(x, np.float64), y=np.ascontiguousarray(y, np.float64),
        z=np.ascontiguousarray(z, np.float64),
        u=np.ascontiguousarray(u, np.float64), v=np.ascontiguousarray(v, np.float64),
        w=np.ascontiguousarray(w, np.float64),
        m=np.ascontiguousarray(m, np.float64), rho=np.ascontiguousarray(rho, np.float64),
        p=np.ascontiguousarray(p, np.float64),
        kind=np.ascontiguousarray(kind, np.int32),
        wall_u=np.ascontiguousarray(wall_u[0], np.float64),
        wall_v=np.ascontiguousarray(wall_u[1], np.float64),
        wall_w=np.ascontiguousarray(wall_u[2], np.float64),
        lo=tuple(float(t) for t in lo), hi=tuple(float(t) for t in hi),
        periodic=tuple(int(t) for t in periodic),
        params=params,
    )


def taylor_green(nside=50, re=100.0, U=1.0, perturb=0.0, seed=1908, hdx=1.0,
                 tol=1e-4, rho0=1.0, pgrad_symm=0, p_ref=0.0):
    """Periodic TGV on the unit square (Sec. 4.1, Eq. tgv at t = 0).

    Lattice ((i+1/2)dx, (j+1/2)dx); optional seeded uniform perturbation of
    +-perturb*dx per coordinate; m = rho0 dx^2, rho = rho0; u, v, p from the
    exact solution at t = 0.  Background pressure by the text's rule for
    internal flows: p_ref = 2 max_i p_i after the first PPE solve, then
    constant, with h~ = h.  (Listing 1 passes p_ref = 100; a background
    pressure of that size, constant or capped at min(10|p|, 100), makes the
    GTVF update unstable at the TGV time step, so the text's rule is used.)
    """
    dx = 1.0 / nside
    x, y = _lattice2(nside, nside, dx)
    if perturb > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = x + rng.uniform(-perturb * dx, perturb * dx, x.size)
        y = y + rng.uniform(-perturb * dx, perturb * dx, y.size)
    n = x.size
    u = -U * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = U * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    p = -U * U * (np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) / 4.0
    h = hdx * dx
    nu = U * 1.0 / re
    prm = _params(h=h, dt=fixed_dt(h, U, nu, 0.0), rho0=rho0, nu=nu, tol=tol,
                  pgrad_symm=pgrad_symm, pref_mode=PREF_TWICE_MAX_FIRST, p_ref=p_ref,
                  gtvf_hfac=1.0)
    return _case(2, x, y, None, u, v, None, np.full(n, rho0 * dx * dx), np.full(n, rho0),
                 p * rho0, np.zeros(n, np.int32), None, (0, 0, 0), (1, 1, 1), (1, 1, 0),
                 prm, f"tgv{nside}_re{re:g}")


def _wall_box2(nx, ny, dx, layers, x0, y0, top=True):
    """Dummy wall particles around [x0, x0+nx dx] x [y0, y0+ny dx], `layers` deep."""
    pts = []
    for k in range(layers):
        off = (k + 0.5) * dx
        # bottom (spans the corners)
        xs = x0 + (np.arange(-layers, nx + layers) + 0.5) * dx
        pts.append(np.stack([xs, np.full(xs.size, y0 - off)], 1))
        if top:
            pts.append(np.stack([xs, np.full(xs.size, y0 + ny * dx + off)], 1))
        ys = y0 + (np.arange(ny) + 0.5) * dx
        pts.append(np.stack([np.full(ys.size, x0 - off), ys], 1))
        pts.append(np.stack([np.full(ys.size, x0 + nx * dx + off), ys], 1))
    w = np.concatenate(pts, 0)
    return w[:, 0].copy(), w[:, 1].copy()


def lid_driven_cavity(nside=50, re=100.0, U=1.0, layers=3, tol=1e-2, rho0=1.0):
    """Lid-driven cavity on the unit square (Sec. 4.2), lid velocity U along x.

    3 layers of dummy wall particles on every side; the top layers (y > 1)
    move with the lid.  "symm" pressure gradient, p_ref = 2 max(p) after the
    first PPE solve, h~ = h (internal flow).
    """
    dx = 1.0 / nside
    xf, yf = _lattice2(nside, nside, dx)
    xw, yw = _wall_box2(nside, nside, dx, layers, 0.0, 0.0, top=True)
    x = np.concatenate([xf, xw]); y = np.concatenate([yf, yw])
    nf, nw = xf.size, xw.size
    kind = np.concatenate([np.zeros(nf, np.int32), np.ones(nw, np.int32)])
    wall_u = np.zeros((3, x.size))
    lid = (kind == WALL) & (y > 1.0)
    wall_u[0, lid] = U
    h = dx
    nu = U * 1.0 / re
    prm = _params(h=h, dt=fixed_dt(h, U, nu, 0.0), rho0=rho0, nu=nu, tol=tol, pgrad_symm=1,
                  pref_mode=PREF_TWICE_MAX_FIRST, p_ref=0.0, gtvf_hfac=1.0)
    n = x.size
    pad = layers * dx
    return _case(2, x, y, None, np.zeros(n), np.zeros(n), None, np.full(n, rho0 * dx * dx),
                 np.full(n, rho0), np.zeros(n), kind, wall_u, (-pad, -pad, 0),
                 (1 + pad, 1 + pad, 1), (0, 0, 0), prm, f"ldc{nside}_re{re:g}")


def dam_break_2d(dx=0.004, layers=3, rho0=1000.0, g=9.81, alpha=0.05, tol=1e-2,
                 tank=(4.0, 4.0), column=(1.0, 2.0)):
    """2D dam break (Sec. 4.4): 1 x 2 m column at the left of a 4 x 4 m tank.

    h = dx (3 wall layers then cover the 3h support), dt = 0.125 h / sqrt(2 g h_w),
    initial hydrostatic pressure rho0 g (h_w - y), free surface on, "symm"
    gradient, artificial viscosity alpha with c = 10 sqrt(2 g h_w), and the
    external-flow background pressure min(10|p|, rho0 c^2) with h~ = h/2.
    """
    nfx = int(round(column[0] / dx)); nfy = int(round(column[1] / dx))
    ntx = int(round(tank[0] / dx)); nty = int(round(tank[1] / dx))
    xf, yf = _lattice2(nfx, nfy, dx)
    xw, yw = _wall_box2(ntx, nty, dx, layers, 0.0, 0.0, top=False)
    x = np.concatenate([xf, xw]); y = np.concatenate([yf, yw])
    nf, nw = xf.size, xw.size
    kind = np.concatenate([np.zeros(nf, np.int32), np.ones(nw, np.int32)])
    hw = column[1]
    vref = math.sqrt(2 * g * hw)
    c0 = 10 * vref
    h = dx
    p = np.zeros(x.size)
    p[:nf] = rho0 * g * (hw - yf)
    prm = _params(h=h, dt=0.125 * h / vref, rho0=rho0, nu=0.0, g=(0.0, -g, 0.0),
                  alpha=alpha, c0=c0, tol=tol, pgrad_symm=1, free_surface=1,
                  pref_mode=PREF_EXTERNAL, p_ref=rho0 * c0 * c0, gtvf_hfac=0.5)
    n = x.size
    pad = layers * dx
    return _case(2, x, y, None, np.zeros(n), np.zeros(n), None, np.full(n, rho0 * dx * dx),
                 np.full(n, rho0), p, kind, None, (-pad, -pad, 0),
                 (tank[0] + pad, tank[1] * 1.5, 1), (0, 0, 0), prm, f"db2d_dx{dx:g}")


def _wall_box3(nx, ny, nz, dx, layers):
    """Open-top box of wall particles around [0,nx dx] x [0,ny dx] x [0,nz dx]."""
    pts = []
    X = (np.arange(-layers, nx + layers) + 0.5) * dx
    Y = (np.arange(-layers, ny + layers) + 0.5) * dx
    Z = (np.arange(nz) + 0.5) * dx
    for k in range(layers):
        off = (k + 0.5) * dx
        a, b = np.meshgrid(X, Y, indexing="ij")
        pts.append(np.stack([a.ravel(), b.ravel(), np.full(a.size, -off)], 1))
        yy = (np.arange(ny) + 0.5) * dx
        a, b = np.meshgrid(yy, Z, indexing="ij")
        pts.append(np.stack([np.full(a.size, -off), a.ravel(), b.ravel()], 1))
        pts.append(np.stack([np.full(a.size, nx * dx + off), a.ravel(), b.ravel()], 1))
        a, b = np.meshgrid(X, Z, indexing="ij")
        pts.append(np.stack([a.ravel(), np.full(a.size, -off), b.ravel()], 1))
        pts.append(np.stack([a.ravel(), np.full(a.size, ny * dx + off), b.ravel()], 1))
    w = np.concatenate(pts, 0)
    return w[:, 0].copy(), w[:, 1].copy(), w[:, 2].copy()


def dam_break_3d(dx=0.008, layers=3, rho0=1000.0, g=9.81, alpha=0.25, tol=1e-2,
                 tank=(1.6, 1.0, 0.6), column=(0.55, 1.0, 0.55)):
    """3D dam break (Sec. 4.5): x = length, y = width, z = up, gravity along -z.

    h = dx, dt = h / (8 v_ref), v_ref = sqrt(2 g h_w), alpha = 0.25, free
    surface on, external-flow background pressure with h~ = h/2.
    """
    nfx = int(round(column[0] / dx)); nfy = int(round(column[1] / dx)); nfz = int(round(column[2] / dx))
    ntx = int(round(tank[0] / dx)); nty = int(round(tank[1] / dx)); ntz = int(round(tank[2] / dx))
    xf, yf, zf = _lattice3(nfx, nfy, nfz, dx)
    xw, yw, zw = _wall_box3(ntx, nty, ntz, dx, layers)
    x = np.concatenate([xf, xw]); y = np.concatenate([yf, yw]); z = np.concatenate([zf, zw])
    nf, nw = xf.size, xw.size
    kind = np.concatenate([np.zeros(nf, np.int32), np.ones(nw, np.int32)])
    hw = column[2]
    vref = math.sqrt(2 * g * hw)
    c0 = 10 * vref
    h = dx
    p = np.zeros(x.size)
    p[:nf] = rho0 * g * (hw - zf)
    prm = _params(h=h, dt=h / (8 * vref), rho0=rho0, nu=0.0, g=(0.0, 0.0, -g),
                  alpha=alpha, c0=c0, tol=tol, pgrad_symm=1, free_surface=1,
                  pref_mode=PREF_EXTERNAL, p_ref=rho0 * c0 * c0, gtvf_hfac=0.5)
    n = x.size
    pad = layers * dx
    return _case(3, x, y, z, np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, rho0 * dx ** 3),
                 np.full(n, rho0), p, kind, None, (-pad, -pad, -pad),
                 (tank[0] + pad, tank[1] + pad, tank[2] * 1.5), (0, 0, 0), prm,
                 f"db3d_dx{dx:g}")


def still_tank_2d(nx=20, ny=20, dx=0.05, layers=3, rho0=1000.0, g=9.81, tol=1e-3,
                  alpha=0.05):
    """A tank of fluid at rest under gravity with hydrostatic initial pressure.

    Used to check the wall-pressure extrapolation (Eq. p-shepard) against
    p = rho0 g (H - y).  Free surface on, artificial viscosity alpha = 0.05
    as in the paper's 2D dam break (without any dissipation the inviscid
    tank does not settle).
    """
    xf, yf = _lattice2(nx, ny, dx)
    xw, yw = _wall_box2(nx, ny, dx, layers, 0.0, 0.0, top=False)
    x = np.concatenate([xf, xw]); y = np.concatenate([yf, yw])
    nf, nw = xf.size, xw.size
    kind = np.concatenate([np.zeros(nf, np.int32), np.ones(nw, np.int32)])
    H = ny * dx
    h = dx
    p = np.zeros(x.size)
    p[:nf] = rho0 * g * (H - yf)
    c0 = 10 * math.sqrt(2 * g * H)
    prm = _params(h=h, dt=fixed_dt(h, math.sqrt(2 * g * H), 0.0, g), rho0=rho0, nu=0.0,
                  g=(0.0, -g, 0.0), alpha=alpha, c0=c0, tol=tol, pgrad_symm=1,
                  free_surface=1, pref_mode=PREF_EXTERNAL, p_ref=rho0 * c0 * c0,
                  gtvf_hfac=0.5)
    n = x.size
    pad = layers * dx
    return _case(2, x, y, None, np.zeros(n), np.zeros(n), None, np.full(n, rho0 * dx * dx),
                 np.full(n, rho0), p, kind, None, (-pad, -pad, 0),
                 (nx * dx + pad, H * 2, 1), (0, 0, 0), prm, f"tank{nx}x{ny}")


def free_fall_blob(n_side=4, dx=0.05, spacing=2.2, g=9.81, rho0=1000.0, adaptive=True):
    """A sparse square of fluid particles (spacing * dx apart, so every
    particle is below the free-surface density and keeps p = 0) falling
    freely in a large closed box without walls: no viscosity, no artificial
    viscosity, zero background pressure.  The only force is gravity, so the
    motion and the adaptive time steps (Sec. 3.2) have closed forms."""
    x, y = _lattice2(n_side, n_side, spacing * dx, x0=4.0, y0=4.0)
    n = x.size
    h = dx
    prm = _params(h=h, dt=0.25 * math.sqrt(h / g), rho0=rho0, nu=0.0, g=(0.0, -g, 0.0),
                  alpha=0.0, tol=1e-3, free_surface=1, pref_mode=PREF_FIXED, p_ref=0.0,
                  adaptive_dt=1 if adaptive else 0)
    return _case(2, x, y, None, np.zeros(n), np.zeros(n), None, np.full(n, rho0 * dx * dx),
                 np.full(n, rho0), np.zeros(n), np.zeros(n, np.int32), None, (0, 0, 0),
                 (10, 10, 1), (0, 0, 0), prm, f"free_fall{n_side}")


def batch_ensemble(ncases=64, seed=1762, nmin=50, nmax=300, total=(2.3e6, 2.7e6),
                   tol=1e-2, scale=1.0):
    """A seeded batch: half TGV (Re log-uniform in [50, 1000]) and half cavity
    (Re log-uniform in [100, 1000]) with uneven n_side ~ U{nmin..nmax}.

    The side lengths are redrawn until the total particle count lies in
    `total` (scaled by `scale`, so tests can draw a small batch of the same
    shape).  Returns a list of cases.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    half = ncases // 2
    lo_t, hi_t = total[0] * scale, total[1] * scale
    for _ in range(10000):
        sides = rng.integers(nmin, nmax + 1, ncases)
        re_t = np.exp(rng.uniform(np.log(50), np.log(1000), half))
        re_l = np.exp(rng.uniform(np.log(100), np.log(1000), ncases - half))
        ntot = int(np.sum(sides[:half] ** 2) + np.sum(sides[half:] ** 2 + 12 * sides[half:] + 36))
        if lo_t <= ntot <= hi_t:
            break
    else:
        raise RuntimeError("could not draw a batch in the requested size window")
    cases = []
    for c in range(half):
        cases.append(taylor_green(int(sides[c]), re=float(re_t[c]), tol=tol))
    for c in range(ncases - half):
        cases.append(lid_driven_cavity(int(sides[half + c]), re=float(re_l[c]), tol=tol))
    return cases


def tgv_exact(x, y, t, re=100.0, U=1.0):
    """Exact TGV velocity and pressure (Eq. tgv)."""
    b = -8 * np.pi ** 2 / re
    e = np.exp(b * t)
    u = -U * e * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = U * e * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    p = -U * U * e * e * (np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) / 4
    return u, v, p
