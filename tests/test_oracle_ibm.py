"""Pins of the oracle's immersed-boundary pieces: Peskin's discrete delta,
interpolation and spreading (Sec. 2.2, Sec. 2.8) and the element tractions of
Eqs. 14-15 with the 1.2 dx probe of Sec. 2.6.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _probe_length():
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.startswith("probe_length"):
                return float(line.split()[1])
    raise KeyError("probe_length")


@pytest.mark.parametrize("r", np.linspace(0.0, 0.999, 23))
def test_peskin_kernel_identities(r):
    """Peskin (2002): unit mass, zero first moment, even/odd split 1/2 and
    sum of squares 3/8 at every offset."""
    js = np.arange(-3, 4)
    ph = np.array([oracle.phi(r - j) for j in js])
    assert ph.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.sum((r - js) * ph) == pytest.approx(0.0, abs=1e-15)
    assert ph[js % 2 == 0].sum() == pytest.approx(0.5, abs=1e-15)
    assert np.sum(ph**2) == pytest.approx(3.0 / 8.0, abs=1e-15)
    assert oracle.phi(2.0) == 0.0 and oracle.phi(2.5) == 0.0


@pytest.mark.parametrize("r", [-1.7, -1.2, -0.6, -0.1, 0.2, 0.7, 1.3, 1.8])
def test_peskin_derivative_matches_finite_difference(r):
    h = 1e-6
    fd = (oracle.phi(r + h) - oracle.phi(r - h)) / (2 * h)
    assert oracle.dphi(r) == pytest.approx(fd, abs=1e-8)


def test_interpolation_of_linear_field_is_exact_with_exact_gradient():
    nx, ny = 20, 16
    a, b, c = 0.3, -0.02, 0.045
    xs = np.arange(nx)[None, :]
    ys = np.arange(ny)[:, None] + 0.5  # nodes sit half a spacing off the wall
    fld = a + b * xs + c * ys
    rng = np.random.default_rng(6)
    for X, Y in rng.uniform([3, 3], [nx - 4, ny - 3], size=(30, 2)):
        W, v, gx, gy = oracle.interp(fld, X, Y)
        assert W == pytest.approx(1.0, abs=1e-14)
        assert v == pytest.approx(a + b * X + c * Y, abs=1e-14)
        assert gx == pytest.approx(b, abs=1e-13) and gy == pytest.approx(c, abs=1e-13)


def test_wall_truncation_velocity_type_and_density_type():
    """Stencil nodes beyond a wall are wall nodes: a velocity-type interpolant
    is the plainly truncated sum (the wall's velocity is zero), so a constant
    field reads W c; a density-type interpolant renormalises and reads c."""
    fld = np.full((8, 12), 1.7)
    for Y in (0.0, 0.1, 0.4, 1.1, 7.6, 8.0):
        W, v, _, _ = oracle.interp(fld, 5.3, Y)
        assert 0.0 < W < 1.0
        assert v == pytest.approx(1.7 * W, abs=1e-14)
        W2, v2, gx, gy = oracle.interp(fld, 5.3, Y, renorm=True)
        assert W2 == W
        assert v2 == pytest.approx(1.7, abs=1e-14) and abs(gx) < 1e-13 and abs(gy) < 1e-13
    W, v, _, _ = oracle.interp(fld, 5.3, 3.7)
    assert W == pytest.approx(1.0, abs=1e-15) and v == pytest.approx(1.7, abs=1e-14)


def test_spreading_is_the_adjoint_of_interpolation_and_conserves_force():
    """<spread(F ds), u> = <F ds, interp(u)> everywhere; the total spread force
    is sum F ds W, i.e. exactly sum F ds away from the walls."""
    nx, ny = 24, 12
    rng = np.random.default_rng(7)
    n = 40
    X = rng.uniform(2.5, nx - 3.5, n)
    Y = rng.uniform(0.0, ny, n)  # includes points next to the walls
    Fx = rng.normal(size=n)
    Fy = rng.normal(size=n)
    ds = rng.uniform(0.5, 1.5, n)
    ox, oy = oracle.spread(nx, ny, X, Y, Fx, Fy, ds)
    one = np.ones((ny, nx))
    W = np.array([oracle.interp(one, X[m], Y[m])[0] for m in range(n)])
    assert ox.sum() == pytest.approx(np.sum(Fx * ds * W), rel=1e-13)
    assert oy.sum() == pytest.approx(np.sum(Fy * ds * W), rel=1e-13)
    inner = (Y > 2.5) & (Y < ny - 2.5)
    assert np.allclose(W[inner], 1.0, atol=1e-15)
    u = rng.normal(size=(ny, nx))
    v = rng.normal(size=(ny, nx))
    iu = np.array([oracle.interp(u, X[m], Y[m])[1] for m in range(n)])
    iv = np.array([oracle.interp(v, X[m], Y[m])[1] for m in range(n)])
    lhs = np.sum(ox * u) + np.sum(oy * v)
    rhs = np.sum(Fx * ds * iu) + np.sum(Fy * ds * iv)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _body_on_fields(rho, ux, uy, xy):
    ny, nx = rho.shape
    s = oracle.OracleSim(nx, ny, tau=1.0, re=0.0, bc=oracle.BC_PERIODIC_FORCE)
    s.add_body(oracle.CELL, oracle.FIXED, xy, ca=0.0)
    s.set_macro(rho, ux, uy)
    return s


def _normals(xy):
    d = np.roll(xy, -1, axis=0) - xy
    L = np.hypot(d[:, 0], d[:, 1])
    n = np.stack([d[:, 1], -d[:, 0]], 1) / L[:, None]
    c = 0.5 * (xy + np.roll(xy, -1, axis=0))
    return c, n, L


def test_pressure_traction_of_a_linear_pressure_field():
    """Eq. 14 on p = cs^2 (rho - 1), rho = 1 + G x: the probe moves each
    evaluation point 1.2 dx outward, so the total is Archimedes' -G A / 3
    plus the closed-form probe term -(G/3) 1.2 sum(n_x n l)."""
    nx, ny, G, x0 = 40, 40, 1e-3, 13.0
    xy = wl.circle(48, 20.2, 19.7, 7.0)
    X = np.arange(nx)[None, :] * np.ones((ny, 1))
    rho = 1.0 + G * (X - x0)
    zero = np.zeros((ny, nx))
    s = _body_on_fields(rho, zero, zero, xy)
    fx, fy = s.traction(0)
    c, n, L = _normals(xy)
    A = oracle.polygon(xy)["A"]
    pl = _probe_length()
    assert fx.sum() == pytest.approx(-(G / 3) * (A + pl * np.sum(n[:, 0] ** 2 * L)), rel=1e-10)
    assert fy.sum() == pytest.approx(-(G / 3) * pl * np.sum(n[:, 0] * n[:, 1] * L), abs=1e-13)
    p = (G / 3) * (c[:, 0] + pl * n[:, 0] - x0)
    assert np.allclose(fx, -p * n[:, 0] * L, atol=1e-14)


def test_viscous_traction_rotation_strain_and_shear():
    """Eq. 15 with tau = rho nu (grad u + grad u^T): zero for rigid rotation,
    2 nu eps (n_x, -n_y) l for pure strain, and rho nu g (n_y, n_x) l plus the
    uniform-pressure term for simple shear."""
    nx, ny = 40, 40
    nu = 1.0 / 6.0
    xy = wl.ellipse(40, 20.3, 20.1, 8.0, 5.0)
    c, n, L = _normals(xy)
    X = np.arange(nx)[None, :] * np.ones((ny, 1))
    Y = (np.arange(ny)[:, None] + 0.5) * np.ones((1, nx))
    one = np.ones((ny, nx))
    x0, y0 = 19.0, 21.0
    Om = 1e-3
    s = _body_on_fields(one, -Om * (Y - y0), Om * (X - x0), xy)
    fx, fy = s.traction(0)
    assert np.abs(fx).max() < 1e-15 and np.abs(fy).max() < 1e-15
    eps = 2e-4
    s = _body_on_fields(one, eps * (X - x0), -eps * (Y - y0), xy)
    fx, fy = s.traction(0)
    assert np.allclose(fx, 2 * nu * eps * n[:, 0] * L, atol=1e-16)
    assert np.allclose(fy, -2 * nu * eps * n[:, 1] * L, atol=1e-16)
    gam, r = 3e-4, 1.01
    s = _body_on_fields(r * one, gam * (Y - y0), 0 * one, xy)
    fx, fy = s.traction(0)
    p = (r - 1.0) / 3.0
    assert np.allclose(fx, (-p * n[:, 0] + r * nu * gam * n[:, 1]) * L, atol=1e-15)
    assert np.allclose(fy, (-p * n[:, 1] + r * nu * gam * n[:, 0]) * L, atol=1e-15)


def test_probes_that_cross_a_wall_stop_at_it():
    """A probe pushed through a wall (the particle's base next to the lower
    wall) is evaluated on the wall: under a uniform pressure every element,
    clamped or not, carries -p n l and the closed body feels no net force."""
    nx, ny = 40, 20
    xy = wl.ellipse(32, 20.0, 2.1, 8.0, 2.0)
    one = np.ones((ny, nx))
    s = _body_on_fields(1.003 * one, 0 * one, 0 * one, xy)
    fx, fy = s.traction(0)
    c, n, L = _normals(xy)
    probe_y = c[:, 1] + _probe_length() * n[:, 1]
    assert (probe_y < 0.0).any()
    assert np.allclose(fx, -(0.003 / 3) * n[:, 0] * L, atol=1e-15)
    assert np.allclose(fy, -(0.003 / 3) * n[:, 1] * L, atol=1e-15)
    assert abs(fx.sum()) < 1e-15 and abs(fy.sum()) < 1e-15
