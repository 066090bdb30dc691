"""Pins of the oracle's moving-least-squares transfer (Sec. 2.2 cites Vanella
and Balaras 2009 for it) against facts other than its own code: the cubic
spline's closed-form values and smoothness, the weighted least-squares fit
solved by numpy's lstsq (wall nodes holding the wall's zero velocity, the
reading the Peskin stencil follows), exact reproduction of linear fields away
from walls, exact constant density at walls (renormalised over the fluid),
second-order interior error, conservation of spread force away from walls
and the adjoint identity between spreading and interpolation."""
import math

import numpy as np
import pytest

import oracle

MLS = oracle.TRANSFER_MLS


def test_weight_closed_forms():
    w = oracle.mls_weight
    assert w(0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert w(1.0) == pytest.approx(1.0 / 6.0, abs=1e-16) and w(-1.0) == w(1.0)
    assert w(2.0) == 0.0 and w(2.5) == 0.0 and w(-3.0) == 0.0
    rs = np.arange(-1250, 1251) / 500.0  # exactly symmetric sample points
    v = np.array([w(r) for r in rs])
    assert (v >= 0).all() and np.array_equal(v, v[::-1])
    # C2 at |r| = 1 (q = 1/2) and at |r| = 2: one-sided value, slope and curvature agree
    h = 1e-4
    for r0 in (1.0, 2.0):
        d1l = (w(r0) - w(r0 - h)) / h
        d1r = (w(r0 + h) - w(r0)) / h
        assert abs(d1l - d1r) < 1e-3
        d2l = (w(r0) - 2 * w(r0 - h) + w(r0 - 2 * h)) / h**2
        d2r = (w(r0 + 2 * h) - 2 * w(r0 + h) + w(r0)) / h**2
        assert abs(d2l - d2r) < 1e-2
    # the cubic B-spline of unit knot spacing integrates to 1; stretched by 2
    # and scaled by 1/2 (its peak 2/3 at q = 0): integral over r of w = 1
    xs = np.linspace(-2, 2, 40001)
    assert np.trapezoid([w(x) for x in xs], xs) == pytest.approx(1.0, rel=1e-7)


def _stencil(nx, ny, X, Y):
    i0, j0 = math.floor(X) - 1, math.floor(Y - 0.5) - 1
    return [(i, j) for j in range(j0, j0 + 4) for i in range(i0, i0 + 4) if 0 <= i < nx and 0 <= j < ny]


POINTS = [(5.3, 4.1), (7.0, 5.5), (0.2, 0.1), (11.0, 9.9), (3.7, 0.0), (0.0, 10.0), (6.49, 0.51), (10.8, 2.2)]


def test_fit_equals_weighted_least_squares():
    """The velocity-type reconstruction and its gradient are the weighted
    least-squares fit of a + b (x - X) + c (y - Y) over the whole 4 x 4
    stencil, nodes beyond a wall or a lattice end holding zero (solved here by
    numpy's lstsq on the sqrt(W)-scaled system)."""
    rng = np.random.default_rng(0)
    nx, ny = 12, 10
    f = rng.normal(0, 1, (ny, nx))
    for X, Y in POINTS:
        i0, j0 = math.floor(X) - 1, math.floor(Y - 0.5) - 1
        nodes = [(i, j) for j in range(j0, j0 + 4) for i in range(i0, i0 + 4)]
        vals = np.array([f[j, i] if 0 <= i < nx and 0 <= j < ny else 0.0 for i, j in nodes])
        P = np.array([[1.0, i - X, j + 0.5 - Y] for i, j in nodes])
        W = np.array([oracle.mls_weight(i - X) * oracle.mls_weight(j + 0.5 - Y) for i, j in nodes])
        keep = W > 0
        sw = np.sqrt(W[keep])
        coef, *_ = np.linalg.lstsq(P[keep] * sw[:, None], vals[keep] * sw, rcond=None)
        S, v, gx, gy = oracle.interp(f, X, Y, kind=MLS)
        inside = all(0 <= i < nx and 0 <= j < ny for i, j in nodes)
        if inside:
            assert S == pytest.approx(1.0, abs=1e-13)
        assert v == pytest.approx(coef[0], abs=1e-12)
        assert gx == pytest.approx(coef[1], abs=1e-12)
        assert gy == pytest.approx(coef[2], abs=1e-12)


def test_linear_fields_and_wall_density():
    nx, ny = 12, 10
    jj, ii = np.mgrid[0:ny, 0:nx]
    interior = [(5.3, 4.1), (7.0, 5.5), (2.6, 1.6), (8.99, 8.4)]
    for a, b, c in ((0.3, 0.7, -1.1), (2.0, 0.0, 0.0), (-1.0, 0.25, 3.0)):
        f = a + b * ii + c * (jj + 0.5)
        for X, Y in interior:
            S, v, gx, gy = oracle.interp(f, X, Y, kind=MLS)
            assert S == pytest.approx(1.0, abs=1e-13)
            assert v == pytest.approx(a + b * X + c * Y, abs=1e-12)
            assert gx == pytest.approx(b, abs=1e-12) and gy == pytest.approx(c, abs=1e-12)
    # a uniform density is reproduced exactly everywhere, walls included
    rho = np.full((ny, nx), 1.0137)
    for X, Y in POINTS:
        S, v, gx, gy = oracle.interp(rho, X, Y, renorm=True, kind=MLS)
        assert S > 0 and v == pytest.approx(1.0137, abs=1e-13)
        assert abs(gx) < 1e-12 and abs(gy) < 1e-12
    # at a wall the velocity-type fit sees the wall nodes' zero: a uniform
    # field is reconstructed as the fluid share of the shape functions
    S, v, _, _ = oracle.interp(np.ones((ny, nx)), 5.0, 0.2, kind=MLS)
    assert 0.3 < S < 0.9 and v == pytest.approx(S, abs=1e-14)


def test_interior_error_is_second_order():
    """Away from walls a linear-basis fit of a smooth field errs by O(h^2):
    at the same phase of the field and the same position in the cell, halving
    the field's curvature scale (L -> 2 L) quarters the error."""
    nx, ny = 80, 40
    jj, ii = np.mgrid[0:ny, 0:nx]
    errs = []
    for L in (8.0, 16.0):
        f = np.sin(ii / L + 0.3) + 0.0 * jj
        X, Y = 3.0 * L, 20.2  # X / L fixed and X on a node column
        _, v, _, _ = oracle.interp(f, X, Y, kind=MLS)
        errs.append(abs(v - math.sin(X / L + 0.3)))
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def test_spreading_conserves_force_and_is_the_adjoint():
    rng = np.random.default_rng(1)
    nx, ny = 14, 9
    n = 12
    X = rng.uniform(2, nx - 3, n)
    Y = rng.uniform(2, ny - 2, n)
    Fx, Fy, ds = rng.normal(0, 1, n), rng.normal(0, 1, n), rng.uniform(0.5, 1.5, n)
    ox, oy = oracle.spread(nx, ny, X, Y, Fx, Fy, ds, kind=MLS)
    # away from walls every shape function lands in the fluid
    assert ox.sum() == pytest.approx((Fx * ds).sum(), abs=1e-12)
    assert oy.sum() == pytest.approx((Fy * ds).sum(), abs=1e-12)
    # markers at the walls and lattice ends: the wall takes the share that
    # falls on wall nodes; spreading stays the adjoint of the interpolation
    X[:3] = (0.0, 13.0, 6.5)
    Y[:3] = (0.1, 8.95, 0.0)
    ox, oy = oracle.spread(nx, ny, X, Y, Fx, Fy, ds, kind=MLS)
    u = rng.normal(0, 1, (ny, nx))
    lhs = (u * ox).sum()
    rhs = sum(Fx[m] * ds[m] * oracle.interp(u, X[m], Y[m], kind=MLS)[1] for m in range(n))
    assert lhs == pytest.approx(rhs, abs=1e-12)
    assert abs(ox.sum() - (Fx * ds).sum()) > 1e-3
