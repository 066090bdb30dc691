"""Pins of the oracle's fluid solver (Eqs. 1-6, Sec. 2.2 and Sec. 3.1
boundary conditions) against closed forms and lattice identities.  CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def test_lattice_matches_printed_weights_and_isotropy():
    """Eq. 3 velocities with the printed weights satisfy the D2Q9 isotropy
    identities up to fourth order (a wrong direction or weight breaks one)."""
    c = _constants()
    ex, ey, w, opp = oracle.lattice()
    assert w[0] == pytest.approx(c["w0"], abs=1e-16)
    assert np.allclose(w[1:5], c["w1"], atol=1e-16) and np.allclose(w[5:], c["w5"], atol=1e-16)
    e = np.stack([ex, ey], 1).astype(float)
    cs2 = c["cs2"]
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(w @ e, 0.0, atol=1e-16)
    d = np.eye(2)
    for a, b in itertools.product(range(2), repeat=2):
        assert np.sum(w * e[:, a] * e[:, b]) == pytest.approx(cs2 * d[a, b], abs=1e-15)
    for a, b, g in itertools.product(range(2), repeat=3):
        assert abs(np.sum(w * e[:, a] * e[:, b] * e[:, g])) < 1e-16
    for a, b, g, h in itertools.product(range(2), repeat=4):
        lhs = np.sum(w * e[:, a] * e[:, b] * e[:, g] * e[:, h])
        rhs = cs2 * cs2 * (d[a, b] * d[g, h] + d[a, g] * d[b, h] + d[a, h] * d[b, g])
        assert lhs == pytest.approx(rhs, abs=1e-15)
    # first axis speed along +x, first diagonal along (+1, +1), as Eq. 3 orders them
    assert (ex[1], ey[1]) == (1, 0) and (ex[5], ey[5]) == (1, 1)
    assert all(ex[opp[i]] == -ex[i] and ey[opp[i]] == -ey[i] for i in range(9))


def test_equilibrium_moments():
    """Eq. 2 reproduces rho, rho u and rho cs^2 I + rho u u exactly."""
    ex, ey, _, _ = oracle.lattice()
    e = np.stack([ex, ey], 1).astype(float)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.1, 0.1, 2)
        feq = oracle.equilibrium(rho, u[0], u[1])
        assert feq.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(feq @ e, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", feq, e, e)
        assert np.allclose(P, rho / 3.0 * np.eye(2) + rho * np.outer(u, u), atol=1e-14)


def test_guo_forcing_moments():
    """Eq. 4's moments: zero mass, (1 - 1/2tau) F momentum and the symmetric
    (1 - 1/2tau)(uF + Fu) second moment (Guo et al. 2002)."""
    ex, ey, _, _ = oracle.lattice()
    e = np.stack([ex, ey], 1).astype(float)
    rng = np.random.default_rng(2)
    for _ in range(20):
        tau = rng.uniform(0.55, 2.0)
        u = rng.uniform(-0.1, 0.1, 2)
        F = rng.uniform(-1e-3, 1e-3, 2)
        g = oracle.guo_term(u[0], u[1], F[0], F[1], tau)
        k = 1.0 - 0.5 / tau
        assert abs(g.sum()) < 1e-18
        assert np.allclose(g @ e, k * F, atol=1e-18)
        S = np.einsum("i,ia,ib->ab", g, e, e)
        assert np.allclose(S, k * (np.outer(u, F) + np.outer(F, u)), atol=1e-18)


def test_streaming_moves_each_population_along_its_speed():
    """Eq. 1 left-hand side: a lone value in direction q at an interior node
    arrives at x + e_q; on a wall row it is bounced back into opp(q) at the
    same node (halfway bounce-back)."""
    ex, ey, _, opp = oracle.lattice()
    nx, ny = 7, 6
    for q in range(9):
        f = np.zeros((9, ny, nx))
        f[q, 3, 3] = 1.0
        g = oracle.stream_bc(f, bc=oracle.BC_PERIODIC_FORCE)
        assert g[q, 3 + ey[q], 3 + ex[q]] == 1.0 and g.sum() == 1.0
    for q in range(9):
        if ey[q] >= 0:
            continue
        f = np.zeros((9, ny, nx))
        f[q, 0, 3] = 1.0
        g = oracle.stream_bc(f, bc=oracle.BC_PERIODIC_FORCE)
        assert g[opp[q], 0, 3] == 1.0 and g.sum() == 1.0
        f = np.zeros((9, ny, nx))
        f[opp[q], ny - 1, 3] = 1.0
        g = oracle.stream_bc(f, bc=oracle.BC_PERIODIC_FORCE)
        assert g[q, ny - 1, 3] == 1.0 and g.sum() == 1.0


def test_periodic_streaming_conserves_mass():
    f = wl.random_populations(17, 9, seed=3)
    g = oracle.stream_bc(f, bc=oracle.BC_PERIODIC_FORCE)
    assert g.sum() == pytest.approx(f.sum(), rel=1e-14)


def test_zou_he_inlet_outlet_constraints():
    """After streaming, the inlet column carries exactly the prescribed
    parabolic velocity (Sec. 3.1) with zero transverse velocity, the outlet
    column exactly rho_out, and both obey non-equilibrium bounce-back along x
    (Zou & He 1997), corners included."""
    ex, ey, _, _ = oracle.lattice()
    nx, ny, umax, rho_out = 12, 10, 0.03, 1.002
    f = wl.random_populations(nx, ny, seed=4, eps=1e-2)
    g = oracle.stream_bc(f, bc=oracle.BC_INLET_OUTLET, umax=umax, rho_out=rho_out)
    assert np.all(np.isfinite(g))
    y = np.arange(ny) + 0.5
    uin = 4 * umax * y * (ny - y) / ny**2
    for x, kind in ((0, "in"), (nx - 1, "out")):
        col = g[:, :, x]
        rho = col.sum(0)
        jx = np.einsum("q,qy->y", ex.astype(float), col)
        jy = np.einsum("q,qy->y", ey.astype(float), col)
        assert np.allclose(jy, 0.0, atol=1e-15)
        if kind == "in":
            assert np.allclose(jx, rho * uin, atol=1e-15)
        else:
            assert np.allclose(rho, rho_out, atol=1e-15)
        for j in range(ny):
            feq = oracle.equilibrium(rho[j], jx[j] / rho[j], 0.0)
            assert (col[1, j] - feq[1]) == pytest.approx(col[3, j] - feq[3], abs=1e-15)


def test_rest_state_is_stationary():
    s = oracle.OracleSim(8, 6, tau=0.8, re=0.0, bc=oracle.BC_PERIODIC_FORCE)
    f0 = s.fpost()
    s.step(10)
    assert np.abs(s.fpost() - f0).max() < 1e-15


def test_first_step_velocity_is_half_force():
    """Eq. 6 read with the body force: from rest, u = F / (2 rho)."""
    gx, gy = 3e-5, -1e-5
    s = oracle.OracleSim(5, 4, tau=1.0, re=0.0, bc=oracle.BC_PERIODIC_FORCE, g=(gx, gy))
    s.step(1)
    rho, ux, uy = s.macro()
    assert np.allclose(rho, 1.0, atol=1e-15)
    assert np.allclose(ux, gx / 2, rtol=1e-12) and np.allclose(uy, gy / 2, rtol=1e-12)


@pytest.mark.parametrize("tau", [0.7, 0.5 + np.sqrt(3) / 4, 1.0, 1.6])
def test_forced_poiseuille_closed_form(tau):
    """Steady BGK + Guo forcing + halfway bounce-back in a periodic channel is
    the parabola g y (H - y) / (2 nu) plus the uniform wall slip
    g (16 L - 3) / (24 nu), L = (tau - 1/2)^2 (analytic BGK bounce-back result,
    He, Zou, Luo & Dembo 1997; Ginzburg & d'Humieres 2003); the slip vanishes
    at L = 3/16."""
    ny = 12
    nu = (tau - 0.5) / 3
    g = 8 * nu * 0.02 / ny**2
    s = oracle.OracleSim(3, ny, tau=tau, re=0.0, bc=oracle.BC_PERIODIC_FORCE, g=(g, 0.0))
    s.step(int(6 * ny * ny / nu) + 2000)
    _, ux, uy = s.macro()
    y = np.arange(ny) + 0.5
    lam = (tau - 0.5) ** 2
    exact = g / (2 * nu) * y * (ny - y) + g * (16 * lam - 3) / (24 * nu)
    assert np.abs(ux[:, 1] - exact).max() < 1e-11 * exact.max()
    assert np.abs(uy).max() < 1e-14


def test_inlet_outlet_channel_develops_the_inlet_parabola():
    """Sec. 3.1: a parabolic inlet and a constant-pressure outlet give plane
    Poiseuille flow along the channel.  At steady state the mass flux is the
    same through every column and every column's profile has the inlet's
    parabolic shape (tau where bounce-back puts the wall exactly halfway;
    residual compressibility at u_max = 0.005 is below 1e-3)."""
    tau = 0.5 + np.sqrt(3) / 4
    nx, ny = 40, 12
    nu = (tau - 0.5) / 3
    re = 0.005 * ny / nu
    s = oracle.OracleSim(nx, ny, tau=tau, re=re, bc=oracle.BC_INLET_OUTLET)
    s.step(16000)
    rho, ux, uy = s.macro()
    y = np.arange(ny) + 0.5
    prof = 4 * s.umax * y * (ny - y) / ny**2
    flux = (rho * ux).sum(0)
    assert np.abs(flux - flux[0]).max() < 1e-9 * flux[0]
    assert flux[0] == pytest.approx((rho[:, 0] * prof).sum(), rel=1e-12)
    for x in (1, nx // 2, nx - 2):
        shape = ux[:, x] / ux[:, x].sum()
        assert np.abs(shape - prof / prof.sum()).max() < 1e-3 * (prof / prof.sum()).max()
    assert np.abs(uy[:, 2:-2]).max() < 1e-3 * prof.max()


def test_mirror_symmetry_in_y():
    """Reflecting the channel about its centre line commutes with a full step
    (exchanges 2<->4, 5<->8, 6<->7): catches index slips in streaming,
    bounce-back, Zou-He and forcing."""
    nx, ny = 14, 9
    mirror = [0, 1, 4, 3, 2, 8, 7, 6, 5]
    f = wl.random_populations(nx, ny, seed=5, eps=1e-2)
    fm = f[mirror][:, ::-1, :]
    a = oracle.OracleSim(nx, ny, tau=0.9, re=0.3, bc=oracle.BC_INLET_OUTLET)
    b = oracle.OracleSim(nx, ny, tau=0.9, re=0.3, bc=oracle.BC_INLET_OUTLET)
    a.set_fpost(f)
    b.set_fpost(fm)
    a.step(3)
    b.step(3)
    assert np.abs(a.fpost()[mirror][:, ::-1, :] - b.fpost()).max() < 1e-15
