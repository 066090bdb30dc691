"""GPU parity of the full coupled step (lattice + Lagrangian kernels) against
the oracle, called through the C ABI.

Tolerances.  FP64 storage: both sides compute the same sequence in double;
differences come from summation order and FMA contraction only, so positions
agree to 1e-9 dx and the velocity field to 1e-9 relative L2 after the 2000
steps of the small capillary.  FP32 storage: the stated bar is 1e-5 relative
L2 on velocity; positions (kept in FP64, displacements computed in FP32) to
1e-6 dx.  Bond events are integer decisions: identical unless the oracle's
logged margin |u - P| of a flipped event is below 1e-5 (a tie, reported)."""
import dataclasses

import numpy as np
import pytest

from helpers import oracle_from, rel_l2
from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS_1STEP = ("uvx", "uvy", "fsx", "fsy", "fbx", "fby", "fax", "fay", "fpx", "fpy", "fwx", "fwy", "fhx", "fhy",
                "ftx", "fty", "vx", "vy", "mx", "my", "mfx", "mfy", "mds")


def _bonds_match(o, s, cap, tie=1e-5):
    for bi, b in enumerate(cap.bodies):
        if b.adhesion is None:
            continue
        ob, _, _, om = o.bonds(bi, b.adhesion.n_lig)
        gb, _, _, _ = s.bonds(bi)
        diff = np.nonzero(ob != gb)[0]
        assert all(om[k] < tie for k in diff), (diff, om[diff])
        if len(diff):
            print(f"bond ties on body {bi}: sites {diff.tolist()} margins {om[diff].tolist()}")


def test_small_capillary_first_step_every_force_fp64():
    cap = wl.small_capillary()
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    o.step(1)
    s.advance(1)
    for bi in range(len(cap.bodies)):
        # x/y components are compared against their joint magnitude: a
        # component that is zero in exact arithmetic carries rounding noise
        for fx in FIELDS_1STEP:
            if not fx.endswith("x"):
                continue
            fy = fx[:-1] + "y"
            ax, ay = o.body(bi, fx), o.body(bi, fy)
            bx, by = s.body_field(bi, fx), s.body_field(bi, fy)
            scale = np.hypot(ax, ay).max()
            err = max(np.abs(ax - bx).max(), np.abs(ay - by).max())
            # floor 1e-13: rounding noise of components that vanish exactly at
            # t = 0 (the area force is k_a p_ref l ~ 0.3 times A/A0 - 1 ~ 1e-16)
            # and of BDF2 velocities formed from positions ~1e2 (ulp 1.4e-14)
            assert err <= 1e-10 * scale + 1e-13, (bi, fx, err, scale)
        a, b = o.body(bi, "mds"), s.body_field(bi, "mds")
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
        assert np.abs(o.body_xy(bi) - s.markers(bi)).max() < 1e-12
    fo = o.fpost()
    assert np.abs(s.populations() - fo).max() < 1e-14
    s.close()


def test_small_capillary_full_run_fp64():
    """240 x 60, biconcave cell + rigid adhering ellipse, 2000 steps."""
    cap = wl.small_capillary()
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    for chunk in (1, 99, 400, 1500):
        o.step(chunk)
        s.advance(chunk)
        for bi in range(len(cap.bodies)):
            assert np.abs(o.body_xy(bi) - s.markers(bi)).max() < 1e-9
        _bonds_match(o, s, cap, tie=1e-9)
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-9
    obs = s.observables()
    assert len(obs) == cap.steps and obs[-1]["step"] == cap.steps
    oo = o.obs()
    assert obs[-1]["delta_p"] == pytest.approx(oo["delta_p"], abs=1e-10)
    assert obs[-1]["r"] == pytest.approx(oo["r"], abs=1e-9)
    assert obs[-1]["n_bound"] == oo["n_bound"]
    assert obs[-1]["t_star"] == pytest.approx(oo["t_star"], rel=1e-12)
    s.close()


def test_production_capillary_full_lattice_fp32():
    """1200 x 150 with the globular cell and the soft AR 0.5 particle, FP32
    populations, 300 steps on the full-size lattice in the launch
    configuration the benchmark times (graph-captured steps)."""
    cap = wl.production_capillary()
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    n = 300
    o.step(n)
    s.advance(n)
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-5
    for bi in range(len(cap.bodies)):
        assert np.abs(o.body_xy(bi) - s.markers(bi)).max() < 1e-6
    _bonds_match(o, s, cap)
    oo, go = o.obs(), s.observables()[-1]
    assert go["step"] == n
    assert go["delta_p"] == pytest.approx(oo["delta_p"], abs=1e-6)
    assert go["r"] == pytest.approx(oo["r"], abs=1e-5)
    s.close()


def test_bodies_near_inlet_walls_and_each_other_fp64():
    """Ragged 70 x 20 lattice; a deformable cell 1.5 dx above a rigid adhering
    rectangle (repulsion active), both within a few nodes of the inlet column
    and of the lower wall."""
    nx, ny = 70, 20
    part = wl.rectangle(24, 9.0, 0.1 + 1.5, 8.0, 3.0)
    cell = wl.circle(40, 9.0, 3.1 + 1.5 + 5.0, 5.0)
    cap = wl.Capillary("edge", nx, ny, 0.9, 2.0, 300, "fp64", 3, [
        wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-2, beta=5e-2),
        wl.Body(wl.PARTICLE, wl.RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1,
                adhesion=wl.Adhesion(30, 1.0, 0.2, 0.1, 0.2, 0.05, 25.0)),
    ])
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    o.step(1)
    s.advance(1)
    fp = o.body(0, "fpy")
    assert np.abs(fp).max() > 0, "repulsion should be active in this set-up"
    assert np.abs(s.body_field(0, "fpy") - fp).max() < 1e-12 * np.abs(fp).max()
    o.step(299)
    s.advance(299)
    for bi in range(2):
        assert np.abs(o.body_xy(bi) - s.markers(bi)).max() < 1e-9
    _bonds_match(o, s, cap, tie=1e-9)
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-9
    s.close()


def test_fixed_particle_and_deformable_particle_fp32():
    """sigma = inf (fixed to the wall) next to a soft particle in FP32."""
    base = wl.production_capillary()
    nx, ny = 400, 150
    fixed = dataclasses.replace(base.bodies[1], motion=wl.FIXED,
                                adhesion=dataclasses.replace(base.bodies[1].adhesion, sigma=np.inf),
                                xy=base.bodies[1].xy + np.array([-150.0, 0.0]))
    cap = dataclasses.replace(base, nx=nx, ny=ny, bodies=[base.bodies[0], fixed])
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    o.step(200)
    s.advance(200)
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-5
    assert s.observables()[-1]["n_l"] == 1.0
    s.close()


def test_checkpoint_restart_is_bit_identical():
    cap = wl.small_capillary()
    a = lbib.from_capillary(cap)
    a.advance(150)
    blob = a.save_state()
    a.advance(150)
    xa, ua = a.markers(0), a.velocity()[0]
    ba = a.bonds(1)[0]
    b = lbib.from_capillary(cap)
    b.load_state(blob)
    assert b.step_count() == 150
    b.advance(150)
    assert np.array_equal(b.markers(0), xa)
    assert np.array_equal(b.velocity()[0], ua)
    assert np.array_equal(b.bonds(1)[0], ba)
    a.close()
    b.close()


def test_profiling_and_pipeline_bookkeeping():
    cap = wl.small_capillary()
    s = lbib.from_capillary(cap)
    s.set_profiling(True)
    s.advance(3)
    s.advance(1)
    bulk, lag, near = s.kernel_times()
    assert bulk > 0 and lag > 0 and near > 0
    d = s.describe()
    assert d["kernels_per_step"] == 6 and 0 < d["near_tiles"] < d["tiles"]
    assert s.step_count() == 4
    obs = s.observables()
    assert [o["step"] for o in obs] == [1, 2, 3, 4]
    assert s.observables() == []
    s.close()


def test_stream_from_torch_and_device_readback():
    torch = pytest.importorskip("torch")
    cap = wl.small_capillary()
    st = torch.cuda.Stream()
    s = lbib.from_capillary(cap, stream=st.cuda_stream)
    s.advance(20)
    ux = torch.empty(cap.ny * cap.nx, dtype=torch.float64, device="cuda")
    uy = torch.empty_like(ux)
    s.velocity_device(ux.data_ptr(), uy.data_ptr(), ux.numel(), 1)
    st.synchronize()
    hx, hy = s.velocity()
    assert np.array_equal(ux.cpu().numpy().reshape(cap.ny, cap.nx), hx)
    s.close()


def test_invalid_arguments_are_rejected():
    s = lbib.Solver(40, 20)
    with pytest.raises(lbib.LbibError) as e:
        s.add_membrane(wl.CELL, wl.DEFORMABLE, wl.circle(20, 20, 10, 5)[::-1])  # clockwise
    assert e.value.status == lbib.LBIB_ERR_INVALID_ARG
    with pytest.raises(lbib.LbibError):
        s.add_membrane(wl.CELL, wl.DEFORMABLE, wl.circle(20, 20, 10, 5), ca=0.0)
    i = s.add_membrane(wl.PARTICLE, wl.RIGID, wl.circle(20, 20, 10, 5), ca=0.0)
    with pytest.raises(lbib.LbibError):
        s.set_adhesion(i, 10, np.inf, 0.2, 0.1, 0.1, 0.1)  # inf sigma needs FIXED
    s.advance(1)
    with pytest.raises(lbib.LbibError) as e:
        s.add_membrane(wl.CELL, wl.DEFORMABLE, wl.circle(20, 20, 10, 5))
    assert e.value.status == lbib.LBIB_ERR_STATE
    buf = np.zeros(8)
    assert s.lib.lbib_read_markers(s.ctx, 5, buf.ctypes.data, 8) == lbib.LBIB_ERR_INVALID_ARG
    assert s.lib.lbib_read_markers(s.ctx, i, buf.ctypes.data, 2) == lbib.LBIB_ERR_INVALID_ARG
    s.close()


def test_largest_membrane():
    """A cell of 1024 vertices (the largest the ABI accepts) in FP32 against
    the oracle; 1025 vertices are refused; in FP64 a 1024-vertex membrane
    needs more shared memory than a block has and is reported as unsupported."""
    nx, ny = 300, 150
    cell = wl.circle(1024, 90.0, 75.0, 60.0)
    cap = wl.Capillary("1024-vertex cell", nx, ny, 1.0, 1.0, 0, "fp32", 0,
                       [wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-2, beta=1e-2)])
    o = oracle_from(cap)
    s = lbib.from_capillary(cap)
    o.step(60)
    s.advance(60)
    assert np.abs(o.body_xy(0) - s.markers(0)).max() < 1e-6
    _, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert rel_l2(np.stack([gux, guy]), np.stack([ux, uy])) < 1e-5
    s.close()
    t = lbib.Solver(nx, ny, storage=lbib.LBIB_STORE_FP32)
    with pytest.raises(lbib.LbibError) as e:
        t.add_membrane(wl.CELL, wl.DEFORMABLE, wl.circle(1025, 90.0, 75.0, 60.0), ca=1e-2)
    assert e.value.status == lbib.LBIB_ERR_INVALID_ARG
    t.close()
    u = lbib.Solver(nx, ny, storage=lbib.LBIB_STORE_FP64)
    u.add_membrane(wl.CELL, wl.DEFORMABLE, cell, ca=1e-2)
    with pytest.raises(lbib.LbibError) as e:
        u.advance(1)
    assert e.value.status == lbib.LBIB_ERR_UNSUPPORTED
    u.close()


def test_contexts_created_while_others_run_match_lone_runs():
    """Every set-up copy and fill of a context is ordered on its own stream:
    a context created and stepped while another context's steps are still in
    flight computes exactly the lone trajectory.  (With the fills on the
    legacy default stream, which is not ordered with the context's
    non-blocking stream, a busy device let the zero fill of the populations
    land after their initialisation.)"""
    cap = wl.small_capillary()
    lone = lbib.from_capillary(cap)
    lone.advance(15)
    x_lone, u_lone = lone.markers(0), lone.velocity()[0]
    lone.close()
    busy = lbib.from_capillary(cap)
    busy.advance(40)  # in flight while the next context is set up
    s = lbib.from_capillary(cap)
    s.advance(15)
    assert np.array_equal(s.markers(0), x_lone)
    assert np.array_equal(s.velocity()[0], u_lone)
    # a checkpoint written into a context while another one runs
    busy.advance(40)
    blob = s.save_state()
    t = lbib.from_capillary(cap)
    t.load_state(blob)
    t.advance(5)
    s.advance(5)
    assert np.array_equal(t.markers(0), s.markers(0))
    for c in (busy, s, t):
        c.close()
