"""Pins of the oracle's smoothing kernel (quintic spline, support 3h).

The paper only names "the quintic spline" (Sec. 2.1, Sec. 4.1).  These tests
fix it by properties that any correct normalised quintic must have:
unit integral in 1, 2 and 3 D (quadrature), dW/dr equal to the derivative of
W (central differences), lattice partition-of-unity sums, and the vanishing
lattice sum of gradients.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("h", [1.0, 0.02, 0.0035])
def test_unit_integral(oracle_lib, dim, h):
    # integral of W over its support (radial measure 2, 2 pi r, 4 pi r^2)
    meas = {1: lambda r: 2.0, 2: lambda r: 2 * math.pi * r, 3: lambda r: 4 * math.pi * r * r}[dim]
    tot = 0.0
    for a, b in ((0, h), (h, 2 * h), (2 * h, 3 * h)):   # integrate piecewise: kinks at h, 2h
        val, _ = integrate.quad(lambda r: meas(r) * oracle.kernel_w(r, h, dim), a, b,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        tot += val
    assert abs(tot - 1.0) < 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_support_and_continuity(oracle_lib, dim):
    h = 0.5
    assert oracle.kernel_w(3 * h, h, dim) == 0.0
    assert oracle.kernel_w(3.5 * h, h, dim) == 0.0
    assert oracle.kernel_dwdr(3 * h, h, dim) == 0.0
    for q in (1.0, 2.0):   # value and slope continuous at the knots
        a = oracle.kernel_w(q * h * (1 - 1e-12), h, dim)
        b = oracle.kernel_w(q * h * (1 + 1e-12), h, dim)
        assert abs(a - b) < 1e-9 * abs(a)
    assert oracle.kernel_dwdr(0.0, h, dim) == 0.0
    assert oracle.kernel_w(0.0, h, dim) > oracle.kernel_w(0.5 * h, h, dim) > 0


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_derivative_is_central_difference(oracle_lib, dim):
    h = 0.013
    for q in np.linspace(0.05, 2.95, 59):
        if abs(q - 1) < 0.02 or abs(q - 2) < 0.02:
            continue
        r = q * h
        e = 1e-6 * h
        fd = (oracle.kernel_w(r + e, h, dim) - oracle.kernel_w(r - e, h, dim)) / (2 * e)
        an = oracle.kernel_dwdr(r, h, dim)
        scale = abs(oracle.kernel_dwdr(0.7 * h, h, dim))
        assert abs(fd - an) < 1e-8 * scale


def _lattice_sum(dim, hdx):
    dx = 1.0
    h = hdx * dx
    rng = range(-4, 5)
    acc = 0.0
    for off in itertools.product(rng, repeat=dim):
        r = math.sqrt(sum((o * dx) ** 2 for o in off))
        acc += dx ** dim * oracle.kernel_w(r, h, dim)
    return acc


@pytest.mark.parametrize("dim,hdx,expect", [(2, 1.0, 1.00006322), (2, 1.3, 0.99995482),
                                            (3, 1.0, 0.99997996)])
def test_lattice_partition_of_unity(oracle_lib, dim, hdx, expect):
    # sum_j (m_j / rho0) W_ij on an infinite square / cubic lattice of the
    # unit-integral quintic (close to, but not exactly, 1).  In 3D the value
    # belongs to sigma = 1/(120 pi h^3); the often-quoted 3/(359 pi h^3)
    # would give 1.0027654 and fails the unit-integral test above.
    s = _lattice_sum(dim, hdx)
    assert abs(s - expect) < 1e-8
    assert abs(s - 1.0) < 3e-3


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_gradient_sum_vanishes(oracle_lib, dim):
    h = 1.0
    acc = np.zeros(dim)
    for off in itertools.product(range(-4, 5), repeat=dim):
        v = np.array(off, float)
        r = np.linalg.norm(v)
        if r == 0:
            continue
        acc += oracle.kernel_dwdr(r, h, dim) * (-v) / r
    assert np.all(np.abs(acc) < 1e-14)


def test_planted_kernel_mistake_is_caught(oracle_lib):
    """Dropping the 15 (1-q)^5 term breaks the unit integral."""
    oracle.plant_mistake(1)
    try:
        val = sum(integrate.quad(lambda r: 2 * math.pi * r * oracle.kernel_w(r, 1.0, 2), a, b)[0]
                  for a, b in ((0, 1), (1, 2), (2, 3)))
    finally:
        oracle.plant_mistake(0)
    assert abs(val - 1.0) > 1e-3
