"""Pins of three oracle pieces that the GPU comparison alone cannot vouch for:
the deformable vertex update (Eqs. 17-18, Sec. 2.8), explicit direct forcing
(Sec. 2.2, the reading: F_L = rho (U_struct - U*) / dt at the element
centroids, spread with weight ds = element length) and the distribution of
the bending force over a hinge (Eq. 10, Sec. 2.3).  Every expected value is
worked out in the test from geometry, closed forms or textbook properties
(constant-acceleration kinematics, the BDF2 = derivative-of-the-interpolating-
quadratic identity, torque balance), never from the oracle's own arithmetic.
CPU only."""
import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

CS2 = 1.0 / 3.0


def _nu(tau):
    return CS2 * (tau - 0.5)  # Sec. 2.1


def _polygon_area(xy):
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


# ------------------------------------------------------- Eqs. 17-18 (Sec. 2.8)

def _displaced_cell(nx=64, ny=64, nv=32, R=10.0, delta=0.05, tau=1.0, re=0.5, ca=1e-3, rho_b=1.0):
    """A stress-free regular polygon in fluid at rest with vertex 0 pushed out
    radially by delta; k_b = k_a = 0, so only the two springs (Eq. 8) of
    vertex 0 act, on vertices nv-1, 0 and 1."""
    ref = wl.circle(nv, nx / 2, ny / 2, R)
    xy = ref.copy()
    rad = (ref[0] - (nx / 2, ny / 2)) / R
    xy[0] = ref[0] + delta * rad
    s = oracle.OracleSim(nx, ny, tau=tau, re=re, bc=oracle.BC_PERIODIC_FORCE)
    s.add_body(oracle.CELL, oracle.DEFORMABLE, xy, xy_ref=ref, ca=ca, beta=0.0, ka=0.0, density_ratio=rho_b)
    # hand-computed constants: u_max = Re nu / H (Sec. 3.1), k_s = rho nu u_max / Ca
    # (Sec. 3.1), m_v = rho_body A_0 / nv (Sec. 2.8) with A_0 the regular polygon's area
    nu = _nu(tau)
    umax = re * nu / ny
    ks = nu * umax / ca
    A0 = 0.5 * nv * R * R * np.sin(2 * np.pi / nv)
    mv = rho_b * A0 / nv
    l0 = 2 * R * np.sin(np.pi / nv)
    F = np.zeros_like(xy)
    for a, b in ((0, 1), (0, nv - 1)):
        r = xy[a] - xy[b]
        L = np.hypot(*r)
        F[a] += -ks * (L - l0) * r / L
        F[b] += ks * (L - l0) * r / L
    return s, xy, F, mv


@pytest.mark.parametrize("rho_b", [1.0, 1.1])
def test_first_verlet_step_from_rest_is_half_a_dt_squared(rho_b):
    """Fluid at rest interpolates to zero velocity at every vertex, so the
    tentative velocity of Eq. 17 is zero and the first step is the motion of a
    point released at rest under a constant force: x^1 - x^0 = (1/2) (F/m_v)
    dt^2 (dt = 1), exactly.  The body is released at rest (x^{-1} = x^0), so
    Eq. 18 gives u^1 = (3/2)(x^1 - x^0) = (3/4) F/m_v; both halves of the
    force's distribution (the spring pulls vertex 0 in and its neighbours
    out) and the vertex mass are computed here independently."""
    s, xy0, F, mv = _displaced_cell(rho_b=rho_b)
    s.step(1)
    x1 = s.body_xy(0)
    assert np.abs(s.body(0, "uvx")).max() == 0.0 and np.abs(s.body(0, "uvy")).max() == 0.0
    d = x1 - xy0
    scale = np.abs(F).max() / mv
    assert scale > 1e-6
    # positions near 40 dx round at ~7e-15: the bound is a few of their ulps
    eps = 8 * np.spacing(np.abs(xy0).max())
    assert np.abs(d - 0.5 * F / mv).max() < eps
    v1 = np.stack([s.body(0, "vx"), s.body(0, "vy")], 1)
    assert np.abs(v1 - 0.75 * F / mv).max() < 2 * eps
    # the spring pulls the pushed-out vertex back towards the centre
    assert F[0] @ (xy0[0] - (32.0, 32.0)) < 0 and d[0] @ (xy0[0] - (32.0, 32.0)) < 0


def test_verlet_and_bdf2_over_five_coupled_steps():
    """Five coupled steps (the fluid moves once the first direct force is
    spread): each step's displacement is the constant-acceleration solution
    from the step's own tentative velocity and total force (Eq. 17, dt = 1),
    and each structure velocity is the derivative, at the new time level, of
    the quadratic through the last three positions (BDF2, Eq. 18; the
    position before the release is the release position)."""
    s, _, _, mv = _displaced_cell(re=2.0)
    hist = [s.body_xy(0)]
    for k in range(1, 6):
        s.step(1)
        xk = s.body_xy(0)
        uv = np.stack([s.body(0, "uvx"), s.body(0, "uvy")], 1)
        ft = np.stack([s.body(0, "ftx"), s.body(0, "fty")], 1)
        xp = np.stack([s.body(0, "xp"), s.body(0, "yp")], 1)
        assert np.array_equal(xp, hist[-1])
        if k > 1:
            assert np.abs(uv).max() > 0  # the coupling is live
        step = xk - hist[-1]
        assert np.abs(step - (uv + 0.5 * ft / mv)).max() < 8 * np.spacing(np.abs(xk).max())
        hist.append(xk)
        prev = hist[-3] if k >= 2 else hist[0]
        t = np.array([k - 2.0, k - 1.0, float(k)])
        v = np.stack([s.body(0, "vx"), s.body(0, "vy")], 1)
        for i in (0, 1, 5):
            for c in range(2):
                pts = np.array([prev[i, c], hist[-2][i, c], xk[i, c]])
                coef = np.polyfit(t - k, pts - pts[2], 2)
                expect = np.polyval(np.polyder(coef), 0.0)
                assert v[i, c] == pytest.approx(expect, abs=16 * np.spacing(np.abs(xk).max()))


# ------------------------------------------------- direct forcing (Sec. 2.2)

def _uniform_flow_around_fixed_circle(nx, ny, rho0, u0, R=6.0, nv=40):
    s = oracle.OracleSim(nx, ny, tau=1.0, re=1e-2, bc=oracle.BC_PERIODIC_FORCE)
    feq = oracle.equilibrium(rho0, u0, 0.0)
    s.set_fpost(np.broadcast_to(feq[:, None, None], (9, ny, nx)).copy())
    xy = wl.circle(nv, nx / 2, ny / 2, R, phase=0.1)
    s.add_body(oracle.PARTICLE, oracle.FIXED, xy, ca=0.0)
    return s, xy


def test_direct_force_of_a_fixed_body_in_uniform_flow():
    """A fixed body (U_struct = 0) in a uniform flow u_0 at density rho_0: on
    the first step every element centroid sees u* = u_0 and rho = rho_0, so
    its direct force is F_L = rho_0 (0 - u_0) / dt per unit length (a density
    other than one and a length other than one catch a missing rho or ds
    applied twice); the spread field carries the whole force, -rho_0 u_0
    times the perimeter of the polygon."""
    nx, ny, R, nv = 64, 48, 6.0, 40
    rho0, u0 = 1.02, 0.01
    s, xy = _uniform_flow_around_fixed_circle(nx, ny, rho0, u0, R, nv)
    s.step(1)
    ds = 2 * R * np.sin(np.pi / nv)
    assert abs(ds - 1) > 0.05
    assert np.allclose(s.body(0, "mds"), ds, rtol=1e-13)
    assert np.allclose(s.body(0, "mfx"), -rho0 * u0, rtol=1e-12)
    assert np.abs(s.body(0, "mfy")).max() < 1e-14 * u0
    fx, fy = s.force_field()
    perim = nv * ds
    assert fx.sum() == pytest.approx(-rho0 * u0 * perim, rel=1e-12)
    assert abs(fy.sum()) < 1e-13 * u0 * perim
    # markers at the element centroids of the fixed chain
    c = 0.5 * (xy + np.roll(xy, -1, axis=0))
    assert np.allclose(s.body(0, "mx"), c[:, 0], atol=1e-13)
    assert np.allclose(s.body(0, "my"), c[:, 1], atol=1e-13)


def test_direct_forcing_brings_the_fluid_at_the_markers_to_rest():
    """The explicit forcing drives the fluid velocity at a fixed body towards
    the body's zero velocity: after 100 steps the velocity interpolated at any
    vertex is below 16% of the undisturbed stream half a channel length away
    (about 12% with the one-pass forcing; the stream itself still carries
    99% of u_0).  Half the direct force leaves about 22%, a flipped sign
    diverges."""
    nx, ny = 160, 48
    s, _ = _uniform_flow_around_fixed_circle(nx, ny, 1.0, 0.01)
    s.step(100)
    assert not s.diverged
    s.step(1)
    uv = np.hypot(s.body(0, "uvx"), s.body(0, "uvy"))
    _, ux, _ = s.macro()
    far = ux[ny // 2, 0]
    assert 0.99 * 0.01 < far < 0.01
    assert uv.max() < 0.16 * far


# -------------------------------------------------------- Eq. 10 (Sec. 2.3)

def test_bending_force_on_an_irregular_hinge_by_hand():
    """Triangle A(0,0) -> B(4,0) -> C(4,3), counter-clockwise, bent at B only
    (theta_0 = theta at A and C, theta_0 = theta - d at B).  At B the edge on
    the left (A-B) is 4 long and the edge on the right (B-C) 3 long; in Sec.
    2.3's definitions l_right is the left edge's length and l_left the right
    edge's, so F_A = k_b d (3/7) n_B, F_B = -k_b d n_B, F_C = k_b d (4/7) n_B,
    with n_B the normalised mean of the outward normals (0,-1) of A-B and
    (1,0) of B-C.  The other assignment would put 4/7 on A and 3/7 on C."""
    xy = np.array([[0.0, 0.0], [4.0, 0.0], [4.0, 3.0]])
    a = xy - np.roll(xy, 1, axis=0)
    b = np.roll(xy, -1, axis=0) - xy
    th = np.arctan2(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0], np.sum(a * b, 1))
    assert th[1] == pytest.approx(np.pi / 2, rel=1e-15)  # left turn of 90 degrees at B
    d, kb = 0.2, 0.7
    th0 = th.copy()
    th0[1] -= d
    l0 = np.hypot(*(np.roll(xy, -1, axis=0) - xy).T)
    _, fb, _ = oracle.membrane_forces(xy, l0, th0, _polygon_area(xy), 0.0, kb, 0.0)
    n = np.array([1.0, -1.0]) / np.sqrt(2.0)
    expect = np.array([kb * d * 3 / 7 * n, -kb * d * n, kb * d * 4 / 7 * n])
    assert np.allclose(fb, expect, atol=1e-15)


def _torque(xy, f):
    return float(np.sum(xy[:, 0] * f[:, 1] - xy[:, 1] * f[:, 0]))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_internal_forces_exert_no_net_torque(seed):
    """Internal forces of a membrane change neither its momentum nor its
    angular momentum: on an irregular chain with random stress-free angles the
    bending (Eq. 10), stretching (Eq. 8) and area (Eq. 11) forces sum to zero
    force and zero torque about the origin and about a far point."""
    rng = np.random.default_rng(seed)
    nv = 11
    t = np.sort(rng.uniform(0, 2 * np.pi, nv))
    r = rng.uniform(3.0, 6.0, nv)
    xy = np.stack([r * np.cos(t) + 2.0, r * np.sin(t) - 1.0], 1)
    l0 = np.hypot(*(np.roll(xy, -1, axis=0) - xy).T) * rng.uniform(0.9, 1.1, nv)
    th0 = rng.normal(0.5, 0.3, nv)
    fs, fb, fa = oracle.membrane_forces(xy, l0, th0, 1.3 * _polygon_area(xy), 0.3, 0.2, 1.0)
    for f in (fs, fb, fa):
        mag = np.abs(f).max()
        assert mag > 1e-3
        assert np.abs(f.sum(0)).max() < 1e-13 * mag * nv
        assert abs(_torque(xy, f)) < 1e-12 * mag * nv
        assert abs(_torque(xy - (100.0, -40.0), f)) < 1e-10 * mag * nv
