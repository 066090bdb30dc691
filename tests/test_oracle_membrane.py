"""Pins of the oracle's structure mechanics: Eqs. 7-8 (stretching), Eq. 10
(bending), Eq. 11 (area penalty), Eq. 12 (repulsion), Eq. 19 (rigid BDF2)
and the polygon measures behind delta_p and r.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _const(name):
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.split()[:1] == [name]:
                return float(line.split()[1])
    raise KeyError(name)


def _lengths(xy):
    d = np.roll(xy, -1, axis=0) - xy
    return np.hypot(d[:, 0], d[:, 1])


def _turning(xy):
    a = xy - np.roll(xy, 1, axis=0)
    b = np.roll(xy, -1, axis=0) - xy
    return np.arctan2(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0], np.sum(a * b, 1))


def test_regular_polygon_measures():
    N, R = 37, 4.3
    xy = wl.circle(N, 1.5, -2.0, R)
    p = oracle.polygon(xy)
    assert p["A"] == pytest.approx(0.5 * N * R * R * np.sin(2 * np.pi / N), rel=1e-14)
    assert p["P"] == pytest.approx(2 * N * R * np.sin(np.pi / N), rel=1e-14)
    assert p["cx"] == pytest.approx(1.5, abs=1e-13) and p["cy"] == pytest.approx(-2.0, abs=1e-13)
    tri = np.array([[0.0, 0.0], [3.0, 0.2], [0.7, 2.5]])
    pt = oracle.polygon(tri)
    assert pt["cx"] == pytest.approx(tri[:, 0].mean(), rel=1e-14)
    assert pt["cy"] == pytest.approx(tri[:, 1].mean(), rel=1e-14)
    rect = np.array([[0.0, 0.0], [6.0, 0.0], [6.0, 2.0], [0.0, 2.0]]) + 5.0
    assert oracle.polygon(rect)["Jc"] == pytest.approx(12.0 * (36 + 4) / 12.0, rel=1e-13)


def test_stretching_force_is_minus_gradient_of_energy():
    """Eq. 8 is the derivative of Eq. 7: brute-force central differences."""
    rng = np.random.default_rng(8)
    xy0 = wl.circle(7, 0.0, 0.0, 3.0)
    l0 = _lengths(xy0) * rng.uniform(0.8, 1.2, 7)
    xy = xy0 + rng.normal(scale=0.3, size=xy0.shape)
    ks = 0.37
    fs, _, _ = oracle.membrane_forces(xy, l0, np.zeros(7), 1.0, ks, 0.0, 0.0)
    h = 1e-6
    for v in range(7):
        for k in range(2):
            p = xy.copy(); p[v, k] += h
            m = xy.copy(); m[v, k] -= h
            g = (oracle.stretch_energy(p, l0, ks) - oracle.stretch_energy(m, l0, ks)) / (2 * h)
            assert fs[v, k] == pytest.approx(-g, abs=1e-8)


def test_internal_forces_vanish_on_the_stress_free_shape():
    xy = wl.biconcave(64, 10.0, 20.0, 12.0)
    l0, th0 = _lengths(xy), _turning(xy)
    A0 = oracle.polygon(xy)["A"]
    fs, fb, fa = oracle.membrane_forces(xy, l0, th0, A0, 0.1, 0.01, 1.0)
    assert np.abs(fs).max() < 1e-15 and np.abs(fb).max() < 1e-15 and np.abs(fa).max() < 1e-15


def test_internal_forces_are_self_equilibrated():
    """Stretching is central (no net force or torque); bending (Eq. 10) and
    the area penalty (Eq. 11) sum to zero on a closed chain."""
    rng = np.random.default_rng(9)
    xy0 = wl.circle(24, 3.0, 4.0, 6.0)
    l0, th0 = _lengths(xy0), _turning(xy0)
    A0 = oracle.polygon(xy0)["A"]
    xy = xy0 + rng.normal(scale=0.4, size=xy0.shape)
    fs, fb, fa = oracle.membrane_forces(xy, l0, th0, A0, 0.2, 0.05, 1.0)
    for f in (fs, fb, fa):
        assert np.abs(f.sum(0)).max() < 1e-14
    torque = np.sum(xy[:, 0] * fs[:, 1] - xy[:, 1] * fs[:, 0])
    assert abs(torque) < 1e-13


def test_bending_uses_the_turning_angle_and_restores_a_bump():
    """A regular N-gon turns by 2 pi / N at every vertex, so with theta_0 =
    2 pi / N no bending force acts on it at any scale; pushing one vertex
    outward makes the force on it point inward and on its neighbours outward."""
    N = 20
    xy = wl.circle(N, 0.0, 0.0, 5.0)
    th0 = np.full(N, 2 * np.pi / N)
    l0 = _lengths(xy)
    for scale in (1.0, 0.7, 1.9):
        _, fb, _ = oracle.membrane_forces(scale * xy, l0, th0, 1.0, 0.0, 0.3, 0.0)
        assert np.abs(fb).max() < 1e-14
    bump = xy.copy()
    bump[0] *= 1.1
    _, fb, _ = oracle.membrane_forces(bump, l0, th0, 1.0, 0.0, 0.3, 0.0)
    out = bump[0] / np.hypot(*bump[0])
    assert fb[0] @ out < 0
    assert fb[1] @ (bump[1] / np.hypot(*bump[1])) > 0 and fb[-1] @ (bump[-1] / np.hypot(*bump[-1])) > 0
    _, fb2, _ = oracle.membrane_forces(bump, l0, th0, 1.0, 0.0, 0.6, 0.0)
    assert np.allclose(fb2, 2 * fb, atol=1e-15)


@pytest.mark.parametrize("s", [0.9, 1.0, 1.05])
def test_area_penalty_on_a_scaled_regular_polygon(s):
    """Eq. 11 with half of each element's force on each vertex: on a regular
    N-gon scaled by s the force on a vertex is k_a (1 - s^2) p_ref l cos(pi/N)
    along the outward radius (outward when compressed)."""
    N, R, ka, pref = 30, 8.0, 1.0, 1.0 / 3.0
    xy0 = wl.circle(N, 0.0, 0.0, R)
    A0 = oracle.polygon(xy0)["A"]
    xy = s * xy0
    _, _, fa = oracle.membrane_forces(xy, _lengths(xy0), np.zeros(N), A0, 0.0, 0.0, ka, pref)
    l = 2 * s * R * np.sin(np.pi / N)
    mag = ka * (1 - s * s) * pref * l * np.cos(np.pi / N)
    radial = xy / np.hypot(xy[:, 0], xy[:, 1])[:, None]
    assert np.allclose(fa, mag * radial, atol=1e-15)


def test_repulsion_coefficient_and_exponent():
    """Eq. 12: 10^-4 / (8 sqrt 2) at d = dx and the d^(-5/2) law."""
    assert oracle.repulsion_magnitude(1.0) == pytest.approx(_const("repulsion_coefficient"), rel=1e-15)
    for d in (0.3, 0.8, 1.7):
        assert oracle.repulsion_magnitude(d) / oracle.repulsion_magnitude(2 * d) == pytest.approx(
            2**2.5, rel=1e-13)


def test_rigid_bdf2_constant_acceleration_closed_form():
    """Eq. 19 from rest under a constant acceleration a: u_n = a (n + 1/2) +
    (a / 6) 3^-n (roots 1 and 1/3 of the BDF2 recurrence)."""
    a = 2.5e-6
    u1 = u2 = 0.0
    for n in range(40):
        u = oracle.rigid_bdf2(u1, u2, a)
        assert u == pytest.approx(a * (n + 0.5) + a / 6 * 3.0**-n, rel=1e-13)
        u2, u1 = u1, u
