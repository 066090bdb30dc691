"""Pins of the oracle's ligand-receptor model (Sec. 2.5, Eq. 13) and of the
counter-based random stream it draws from.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert oracle.philox4x32_10(ctr, key).tolist() == out


def test_bond_uniform_draw_layout_and_distribution():
    """u = (word0 >> 8) 2^-24 with counter (step_lo, step_hi, site, 0) and
    key (seed_lo, seed_hi); the draws are uniform on [0, 1)."""
    seed, step, site = 0x0123456789ABCDEF, (5 << 32) + 7, 11
    w = oracle.philox4x32_10([7, 5, 11, 0], [0x89ABCDEF, 0x01234567])
    assert oracle.bond_uniform(seed, step, site) == (int(w[0]) >> 8) / 2**24
    u = np.array([oracle.bond_uniform(3, s, k) for s in range(200) for k in range(100)])
    assert 0.0 <= u.min() and u.max() < 1.0
    assert u.mean() == pytest.approx(0.5, abs=0.01) and u.var() == pytest.approx(1 / 12, abs=0.003)


def _flat_particle_sim(gap, y_cr, y_eq, kf_dt, kr0_dt, xi, sigma=0.0, n_lig=480, seed=0):
    """A heavy rigid 20 x 4 rectangle, base `gap` above the lower wall, in a
    periodic channel at rest.  Vertices one lattice unit apart (corners are
    vertices); ligand sites one per element, at mid-element."""
    nx, ny = 48, 24
    h = 4.0
    xy = wl.rectangle(48, 24.0, gap + h / 2, 20.0, h)
    s = oracle.OracleSim(nx, ny, tau=1.0, re=1.0, bc=oracle.BC_PERIODIC_FORCE, seed=seed)
    b = s.add_body(oracle.PARTICLE, oracle.RIGID, xy, ca=0.0, density_ratio=1e12)
    s.set_adhesion(b, n_lig, sigma, y_cr, y_eq, kf_dt, kr0_dt, xi)
    return s, b


@pytest.mark.parametrize("xi_scale", [0.0, 1.0])
def test_bond_survival_follows_the_reverse_probability(xi_scale):
    """With no rebinding a bound site survives n steps with probability
    (1 - P_r)^n, P_r = 1 - exp(-k_r0 dt exp(xi (y - y_eq)^2)) at the bond
    length y (binomial 4-sigma bands)."""
    y_cr, y_eq, gap, kr0 = 0.2, 0.1, 0.18, 0.01
    xi = xi_scale * np.log(3.0) / (gap - y_eq) ** 2
    s, b = _flat_particle_sim(gap, y_cr, y_eq, 0.0, kr0, xi, n_lig=480)
    n0 = int(s.body_scalars(b)["nl0"])
    assert n0 >= 150
    q = np.exp(-kr0 * np.exp(xi * (gap - y_eq) ** 2))
    done = 0
    for n in (10, 20, 40):
        s.step(n - done)
        done = n
        k = s.obs()["n_bound"]
        p = q**n
        assert abs(k - n0 * p) < 4 * np.sqrt(n0 * p * (1 - p)) + 1


def test_bound_fraction_relaxes_to_the_two_state_equilibrium():
    """Formation with P_f and rupture with P_r, one draw per site and step,
    give the stationary bound fraction P_f / (P_f + P_r) of N_L (normalised by
    the bonds engaged at t = 0, Sec. 3.3)."""
    pf, pr = 0.1, 0.05
    s, b = _flat_particle_sim(0.1, 0.2, 0.1, -np.log(1 - pf), -np.log(1 - pr), 0.0, n_lig=480)
    s.step(100)
    acc = []
    for _ in range(500):
        s.step(1)
        acc.append(s.obs()["n_l"])
    assert np.mean(acc) == pytest.approx(pf / (pf + pr), abs=0.03)


def test_bond_force_is_a_linear_spring_normal_to_the_wall_at_formation():
    """Eq. 13 with sigma in units rho nu^2 / H (Sec. 2.5): every base bond,
    perpendicular to the wall when it forms, pulls along the base's outward
    normal (towards the wall) with sigma (y - y_eq); only the twenty base sites
    are within y_cr."""
    gap, y_cr, y_eq, sigma = 0.3, 0.35, 0.1, 2.0
    s, b = _flat_particle_sim(gap, y_cr, y_eq, 0.0, 0.0, 0.0, sigma=sigma, n_lig=48)
    assert s.body_scalars(b)["nl0"] == 20
    s.step(1)
    fwx, fwy = s.body(b, "fwx"), s.body(b, "fwy")
    nu, ny = 1.0 / 6.0, 24
    assert fwy.sum() == pytest.approx(-20 * sigma * nu * nu / ny * (gap - y_eq), rel=1e-6)
    assert abs(fwx.sum()) < 1e-12 * abs(fwy.sum())


def test_bond_force_resists_the_drift_of_its_site():
    """A linear spring pulls a site back towards its receptor: a rigid particle
    dragged downstream by a forced channel flow stretches its bonds along x,
    and their total force then opposes the drift (x component of opposite sign
    to the sites' mean displacement from their anchors) while still pulling
    towards the wall."""
    nx, ny = 48, 24
    s = oracle.OracleSim(nx, ny, tau=1.0, re=0.0, bc=oracle.BC_PERIODIC_FORCE, g=(2e-6, 0.0), seed=0)
    xy = np.stack([np.linspace(14, 30, 40, endpoint=False), np.full(40, 0.2)], 1)
    top = np.stack([np.linspace(30, 14, 40, endpoint=False), np.full(40, 2.2)], 1)
    rect = np.concatenate([xy, [[30, 0.2], [30, 1.2]], top, [[14, 2.2], [14, 1.2]]])
    b = s.add_body(oracle.PARTICLE, oracle.RIGID, rect, None, 0.0, 0.0, 1.0, 1.1)
    s.set_adhesion(b, 60, 1.0, 0.35, 0.1, 0.0, 0.0, 0.0)  # bonds neither form nor break
    nl0 = s.body_scalars(b)["nl0"]
    assert nl0 > 10
    s.step(400)
    bound, ax, ay, _ = s.bonds(b, 60)
    xp = s.body_xy(b)[:, 0].mean()
    drift = xp - 22.0
    assert drift > 1e-4  # dragged downstream
    fwx, fwy = s.body(b, "fwx"), s.body(b, "fwy")
    assert fwx.sum() < 0 and fwy.sum() < 0
    assert abs(fwx.sum()) > 1e-3 * abs(fwy.sum())


def test_fixed_particle_keeps_its_bonds():
    """sigma = inf is a particle fixed to the wall: N_L stays 1."""
    s, b = _flat_particle_sim(0.1, 0.2, 0.1, 0.5, 0.5, 0.0, sigma=np.inf)
    nx, ny = 48, 24
    s2 = oracle.OracleSim(nx, ny, tau=1.0, re=1.0, bc=oracle.BC_PERIODIC_FORCE)
    xy = wl.rectangle(48, 24.0, 2.1, 20.0, 4.0)
    b2 = s2.add_body(oracle.PARTICLE, oracle.FIXED, xy, ca=0.0)
    s2.set_adhesion(b2, 480, np.inf, 0.2, 0.1, 0.5, 0.5, 0.0)
    s2.step(20)
    assert s2.obs()["n_l"] == 1.0
