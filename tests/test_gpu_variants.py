"""Paper variants of Sec. 3.1 on the GPU: bullet- and parachute-shaped cells
generated by the solver (the circular and biconcave cells' steady shapes in
the capillary flow, transported with the undeformed shape as stress-free
configuration), a deformed cell with a separate stress-free shape against the
oracle, and circular particles (compared in the paper with square ones of the
same thickness) against the oracle.

Parity bars as test_gpu_coupled.py (FP64: positions 1e-9 dx, velocity 1e-9
relative L2; bond decisions identical up to logged ties).  The generated
shapes are checked for what the paper says of them, not against numbers: the
run converged, area is held (k_a = 1 keeps the membrane incompressible,
Sec. 2.3), the shape is symmetric about the channel's centre line, and the
bullet leads with its nose while the parachute's rims trail."""
import dataclasses
import math

import numpy as np
import pytest

from helpers import oracle_from, rel_l2
from paper_2210_06043_gb300 import cell_shapes as cs
from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NY, NV = 30, 64


def _area(xy):
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _check_shape(r, ref):
    R = math.sqrt(_area(ref) / math.pi)
    assert r.converged, (r.steps, r.change)
    assert abs(_area(r.xy) / _area(ref) - 1.0) < 1e-2
    assert abs(r.xy[:, 1].max() + r.xy[:, 1].min()) < 1e-3 * R  # centre-line symmetry
    front, rear = r.xy[:, 0].max(), -r.xy[:, 0].min()
    return R, front, rear


def test_bullet_cell_from_the_circular_cell():
    dx = wl.H_UM / NY
    ref = wl.circle(NV, 0.0, 0.0, wl.CELL_RADIUS_UM / dx)
    r = cs.bullet_cell(NV, NY)
    R, front, rear = _check_shape(r, ref)
    assert front - rear > 0.1 * R  # rounded nose ahead, flattened back
    assert wl.reduced_area(r.xy) < 0.95  # no longer a circle
    # transported with the circle as stress-free shape, the bullet stays a bullet
    start = np.array([1.5 * NY, 0.5 * NY])
    cap = wl.Capillary("bullet", 8 * NY, NY, 1.0, 0.2, 0, "fp32", 0,
                       [wl.Body(wl.CELL, wl.DEFORMABLE, r.xy + start, ca=1e-3, beta=0.0, xy_ref=ref + start)])
    s = lbib.from_capillary(cap)
    s.advance(int(0.2 * NY * NY * 6.0 / 0.2))
    m = s.markers(0)
    c, _ = cs._centroid(m)
    assert (m[:, 0] - c[0]).max() + (m[:, 0] - c[0]).min() > 0.1 * R
    s.close()


def test_parachute_cell_from_the_biconcave_cell():
    dx = wl.H_UM / NY
    ref = wl.biconcave(NV, 0.0, 0.0, wl.CELL_RADIUS_UM / dx)
    r = cs.parachute_cell(NV, NY)
    R, front, rear = _check_shape(r, ref)
    assert rear > front  # rims trail the centre
    assert r.xy[:, 1].max() < 0.9 * ref[:, 1].max()  # rims folded back from the across-channel disc


def test_deformed_cell_with_its_own_stress_free_shape_fp64():
    """A cell starting from an ellipse of the circle's area with the circle as
    stress-free shape (how bullet and parachute cells are transported)."""
    nx, ny = 120, 30
    dx = wl.H_UM / ny
    r0 = 0.8 * wl.CELL_RADIUS_UM / dx
    ref = wl.circle(NV, 30.0, 15.0, r0)
    xy = wl.ellipse(NV, 30.0, 15.0, 1.15 * r0, r0 / 1.15)
    cap = wl.Capillary("deformed", nx, ny, 1.0, 0.5, 300, "fp64", 0,
                       [wl.Body(wl.CELL, wl.DEFORMABLE, xy, ca=1e-2, beta=1e-2, xy_ref=ref)])
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    o.step(1)
    s.advance(1)
    for f in ("fsx", "fbx", "fax", "ftx"):
        a, b = o.body(0, f), s.body_field(0, f)
        assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max() + 1e-13, f
    assert np.abs(o.body(0, "fsx")).max() > 1e-6  # the springs are loaded
    o.step(299)
    s.advance(299)
    assert np.abs(o.body_xy(0) - s.markers(0)).max() < 1e-9
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-9
    s.close()


@pytest.mark.parametrize("shape", ["circle", "square"])
def test_circular_and_square_particles_fp64(shape):
    """A rigid adhering particle of thickness 1 um, circular or square, under
    the cell in the 240 x 60 capillary."""
    cap = wl.particle_comparison_capillary(shape, 1.0, nx=240, ny=60, storage="fp64")
    dx = wl.H_UM / 60
    cell = wl.biconcave(128, wl.CELL_X_UM / dx, wl.CELL_Y_UM / dx, wl.CELL_RADIUS_UM / dx)
    cap = dataclasses.replace(cap, bodies=[wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-3, beta=1e-2),
                                           cap.bodies[1]])
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    n_lig = cap.bodies[1].adhesion.n_lig
    for chunk in (1, 499):
        o.step(chunk)
        s.advance(chunk)
        for bi in range(2):
            assert np.abs(o.body_xy(bi) - s.markers(bi)).max() < 1e-9
        ob, _, _, om = o.bonds(1, n_lig)
        gb, _, _, _ = s.bonds(1)
        diff = np.nonzero(ob != gb)[0]
        assert all(om[k] < 1e-9 for k in diff)
    assert s.observables()[-1]["n_bound"] > 0
    s.close()
