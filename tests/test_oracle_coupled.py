"""Checks of the oracle's full coupled step: observables (Sec. 3.1) against
closed forms, the quiescent-relaxation and area-conservation behaviour the
paper reports for k_a = 1 (Sec. 2.3), and stability of the small capillary.
CPU only."""
import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl


def build(cap):
    s = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, bc=cap.bc, g=cap.g, seed=cap.seed)
    for b in cap.bodies:
        i = s.add_body(b.kind, b.motion, b.xy, b.xy_ref, b.ca, b.beta, b.ka, b.density_ratio)
        if b.adhesion is not None:
            a = b.adhesion
            s.set_adhesion(i, a.n_lig, a.sigma, a.y_cr, a.y_eq, a.kf_dt, a.kr0_dt, a.xi)
    return s


def test_observables_of_fixed_bodies():
    """delta_p = (p - p0) / p0 of a cell held at s times its stress-free
    circle is s - 1; r is the distance between the two area centroids; N_L of a
    particle fixed to the wall stays 1."""
    s = oracle.OracleSim(80, 40, tau=1.0, re=1e-2, bc=oracle.BC_INLET_OUTLET)
    ref = wl.circle(48, 25.0, 20.0, 8.0)
    scale = 1.07
    cell = 25.0 + scale * (ref[:, 0] - 25.0), 20.0 + scale * (ref[:, 1] - 20.0)
    s.add_body(oracle.CELL, oracle.FIXED, np.stack(cell, 1), xy_ref=ref, ca=0.0)
    part = wl.rectangle(40, 55.0, 2.1, 10.0, 4.0)
    p = s.add_body(oracle.PARTICLE, oracle.FIXED, part, ca=0.0)
    s.set_adhesion(p, 40, np.inf, 0.2, 0.1, 0.1, 0.1, 0.0)
    s.step(3)
    o = s.obs()
    assert o["delta_p"] == pytest.approx(scale - 1.0, abs=1e-13)
    assert o["r"] == pytest.approx(np.hypot(55.0 - 25.0, 2.1 - 20.0), abs=1e-12)
    assert o["n_l"] == 1.0 and o["step"] == 3
    assert o["t_star"] == pytest.approx(3 * s.umax / 40, rel=1e-14)


def test_quiescent_relaxation_towards_the_stress_free_shape():
    """Sec. 2.3 (Supp. Fig. 3 claim): in fluid at rest a deformed cell keeps
    evolving under its internal stresses only and returns towards its
    stress-free circle, its stretching ratio decaying while k_a = 1 holds the
    area within 1% of A_0."""
    R, nv = 10.0, 64
    ref = wl.circle(nv, 30.0, 20.0, R)
    t = 2 * np.pi * np.arange(nv) / nv
    xy = np.stack([30.0 + 11.5 * np.cos(t), 20.0 + 8.5 * np.sin(t)], 1)
    s = oracle.OracleSim(60, 40, tau=1.0, re=1.0, bc=oracle.BC_PERIODIC_FORCE)
    s.add_body(oracle.CELL, oracle.DEFORMABLE, xy, xy_ref=ref, ca=3e-4, beta=0.0)

    def roundness():
        p = s.body_xy(0)
        r = np.hypot(*(p - p.mean(0)).T)
        return (r.max() - r.min()) / R

    dps, shapes = [], []
    for _ in range(6):
        s.step(500)
        sc = s.body_scalars(0)
        assert abs(sc["area"] / sc["A0"] - 1) < 1e-2
        dps.append(s.obs()["delta_p"])
        shapes.append(roundness())
    assert not s.diverged
    assert all(a > b for a, b in zip(dps, dps[1:]))
    assert all(a > b for a, b in zip(shapes, shapes[1:]))
    assert dps[-1] < 0.4 * dps[0] and shapes[-1] < 0.7 * shapes[0]


def test_small_capillary_is_stable_and_conserves_cell_area():
    """The 240 x 60 capillary (biconcave cell, rigid adhering ellipse) over its
    2000 steps: finite state, cell area within 1e-3 of A_0, bonds between 0
    and all sites."""
    cap = wl.small_capillary()
    s = build(cap)
    s.step(cap.steps)
    assert not s.diverged
    sc = s.body_scalars(0)
    assert abs(sc["area"] / sc["A0"] - 1) < 1e-3
    o = s.obs()
    assert 0 <= o["n_bound"] <= cap.bodies[1].adhesion.n_lig
    rho, ux, uy = s.macro()
    assert np.all(np.isfinite(ux)) and np.abs(rho - 1).max() < 1e-2


def test_sweep_workload_covers_the_parameter_matrix():
    """64 capillaries: each (AR, Ca, cell, seed) combination of Sec. 3.1's
    sweep once, lengths within [600, 1600], H = 150; rigid exactly when Ca = 0;
    particle thickness = AR x length."""
    caps = wl.sweep_capillaries()
    assert len(caps) == 64
    seen = set()
    for c in caps:
        assert 600 <= c.nx <= 1600 and c.ny == 150 and c.storage == "fp32"
        cell, part = c.bodies
        ext = part.xy.max(0) - part.xy.min(0)
        ar = round(float(ext[1] / ext[0]), 2)
        shape = "globular" if np.ptp(np.hypot(*(cell.xy - cell.xy.mean(0)).T)) < 1e-6 else "biconcave"
        seen.add((ar, part.ca, shape, c.seed))
        assert (part.motion == wl.RIGID) == (part.ca == 0.0)
        assert part.adhesion.n_lig == 200
    assert seen == {(ar, ca, cell, s) for ar in wl.SWEEP_AR for ca in wl.SWEEP_CA for cell in wl.SWEEP_CELLS
                    for s in wl.SWEEP_SEEDS}
    assert wl.sweep_capillaries()[5].nx == caps[5].nx  # seeded


def test_threaded_node_loops_give_the_same_bits():
    """The oracle's streaming and collision loops may run on several host
    threads; every node's arithmetic and every sum keep one order, so the
    small capillary after 40 steps is the same bits on 1 and 4 threads."""
    cap = wl.small_capillary()
    n0 = oracle.set_threads(0)
    out = []
    try:
        for n in (1, 4):
            assert oracle.set_threads(n) == n
            s = build(cap)
            s.step(40)
            out.append((s.fpost(), s.body_xy(0), s.body_xy(1), s.macro()[1], s.obs()))
    finally:
        oracle.set_threads(n0)
    (f1, a1, b1, u1, o1), (f4, a4, b4, u4, o4) = out
    assert np.array_equal(f1, f4) and np.array_equal(a1, a4) and np.array_equal(b1, b4)
    assert np.array_equal(u1, u4) and o1 == o4
