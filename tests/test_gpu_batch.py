"""GPU parity of batched capillaries: one context stepping several capillaries
of different lengths side by side (a parameter sweep), called through the C ABI.

Each instance of a batch must give bit-for-bit the results of a context that
holds that capillary alone: the lattice update of a node, the Lagrangian
update of a body and the observables of an instance read only that instance's
data, in the same order of operations, with the stencil offsets of the
instance added as exact integers.  So these tests compare with
``np.array_equal``.  The batch is also compared with the FP64 oracle directly
(same tolerances as the single-capillary tests)."""
import dataclasses

import numpy as np
import pytest

from helpers import oracle_from, rel_l2
from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NY = 60


def _mixed_fp64():
    """Four FP64 capillaries sharing ny = 60: the small capillary (seed 0); a
    ragged 77-node channel with a cell 1.5 dx above a rigid adhering rectangle
    near the inlet (seed 3); a 45-node channel without bodies; a 200-node
    channel with the small capillary's bodies and seed 5."""
    a = wl.small_capillary()
    rect = wl.rectangle(24, 14.0, 0.1 + 1.5, 8.0, 3.0)
    cell = wl.circle(48, 14.0, 3.1 + 1.5 + 6.0, 6.0)
    b = wl.Capillary("edge", 77, NY, 1.0, 1e-2, 300, "fp64", 3, [
        wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-2, beta=5e-2),
        wl.Body(wl.PARTICLE, wl.RIGID, rect, ca=0.0, beta=0.0, density_ratio=1.1,
                adhesion=wl.Adhesion(30, 1.0, 0.2, 0.1, 0.2, 0.05, 25.0)),
    ])
    c = wl.Capillary("empty", 45, NY, 1.0, 1e-2, 300, "fp64", 4, [])
    d = dataclasses.replace(wl.small_capillary(seed=5), nx=200)
    return [a, b, c, d]


def _same_state(batch, k, lone, cap, body0, observables=True):
    """Instance k of `batch` (its bodies numbered from body0) equals `lone`
    (observables records too, which moves both cursors)."""
    for bi, b in enumerate(cap.bodies):
        assert np.array_equal(batch.markers(body0 + bi), lone.markers(bi)), (k, bi)
        for f in ("uvx", "uvy", "ftx", "fty", "mfx", "mfy", "vx", "vy"):
            assert np.array_equal(batch.body_field(body0 + bi, f), lone.body_field(bi, f)), (k, bi, f)
        if b.adhesion is not None:
            for x, y in zip(batch.bonds(body0 + bi), lone.bonds(bi)):
                assert np.array_equal(x, y), (k, bi)
    gu, gv = batch.velocity(k)
    lu, lv = lone.velocity()
    assert np.array_equal(gu, lu) and np.array_equal(gv, lv), k
    assert np.array_equal(batch.populations(k), lone.populations()), k
    if not observables:
        return
    ob, ol = batch.observables(instance=k), lone.observables()
    assert len(ob) == len(ol), k
    for x, y in zip(ob, ol):
        for key in ("step", "n_bound"):
            assert x[key] == y[key], (k, key)
        for key in ("t_star", "delta_p", "r", "n_l"):
            assert (x[key] == y[key]) or (np.isnan(x[key]) and np.isnan(y[key])), (k, key, x[key], y[key])


def test_batch_instances_equal_lone_runs_fp64():
    caps = _mixed_fp64()
    batch = lbib.from_capillaries(caps)
    lones = [lbib.from_capillary(c) for c in caps]
    body0 = np.cumsum([0] + [len(c.bodies) for c in caps])
    for chunk in (1, 40, 160):
        batch.advance(chunk)
        for s in lones:
            s.advance(chunk)
        for k, (c, s) in enumerate(zip(caps, lones)):
            _same_state(batch, k, s, c, int(body0[k]))
    assert batch.observables(instance=2) == []  # no bodies, no records
    assert batch.latest_observables()[2]["step"] == -1
    batch.close()
    for s in lones:
        s.close()


def test_batch_against_oracle_fp64():
    caps = _mixed_fp64()
    batch = lbib.from_capillaries(caps)
    n = 300
    batch.advance(n)
    body0 = np.cumsum([0] + [len(c.bodies) for c in caps])
    for k in (1, 2, 3):
        o = oracle_from(caps[k])
        o.step(n)
        _, ux, uy = o.macro()
        gu, gv = batch.velocity(k)
        assert rel_l2(np.stack([gu, gv]), np.stack([ux, uy])) < 1e-9, k
        for bi in range(len(caps[k].bodies)):
            assert np.abs(o.body_xy(bi) - batch.markers(int(body0[k]) + bi)).max() < 1e-9, (k, bi)
        if caps[k].bodies:
            oo, go = o.obs(), batch.observables(instance=k)[-1]
            assert go["step"] == n
            assert go["n_bound"] == oo["n_bound"]
            assert go["delta_p"] == pytest.approx(oo["delta_p"], abs=1e-10)
            assert go["r"] == pytest.approx(oo["r"], abs=1e-9)
    batch.close()


def test_sweep_full_size_fp32_sampled():
    """The 64-capillary sweep (channel lengths 600-1600, H = 150, FP32) in the
    launch configuration the benchmark times; three sampled instances are
    compared bit-for-bit with lone runs and one with the oracle."""
    caps = wl.sweep_capillaries()
    batch = lbib.from_capillaries(caps)
    batch.autotune(steps_per_trial=10)  # as the benchmark does before it times the sweep
    n = 40
    batch.advance(n)
    d = batch.describe()
    assert d["kernels_per_step"] == 6
    latest = batch.latest_observables()
    records = [batch.observables(instance=inst) for inst in range(len(caps))]
    for inst, obs in enumerate(records):
        assert latest[inst] == obs[-1]
        assert len(obs) == n and obs[-1]["step"] == n and obs[-1]["status"] == 0
        assert np.isfinite(obs[-1]["delta_p"]) and np.isfinite(obs[-1]["r"])
    body0 = np.cumsum([0] + [len(c.bodies) for c in caps])
    lengths = [c.nx for c in caps]
    sample = sorted({int(np.argmin(lengths)), int(np.argmax(lengths)), 37})
    for k in sample:
        lone = lbib.from_capillary(caps[k])
        lone.advance(n)
        _same_state(batch, k, lone, caps[k], int(body0[k]), observables=False)
        assert lone.observables() == records[k]
        lone.close()
    k = sample[0]
    o = oracle_from(caps[k])
    o.step(n)
    _, ux, uy = o.macro()
    gu, gv = batch.velocity(k)
    assert rel_l2(np.stack([gu, gv]), np.stack([ux, uy])) < 1e-5
    for bi in range(2):
        assert np.abs(o.body_xy(bi) - batch.markers(int(body0[k]) + bi)).max() < 1e-6
    batch.close()


def test_batch_checkpoint_restart_is_bit_identical():
    caps = _mixed_fp64()
    a = lbib.from_capillaries(caps)
    a.advance(60)
    blob = a.save_state()
    a.advance(60)
    b = lbib.from_capillaries(caps)
    b.load_state(blob)
    c = lbib.from_capillaries(caps)
    c.advance(60)
    for k in range(len(caps)):  # reads right after the restore equal the saved run's
        assert np.array_equal(b.velocity(k)[0], c.velocity(k)[0])
    c.close()
    b.advance(60)
    for k in range(len(caps)):
        assert np.array_equal(a.velocity(k)[0], b.velocity(k)[0])
    for body in range(sum(len(c.bodies) for c in caps)):
        assert np.array_equal(a.markers(body), b.markers(body))
    a.close()
    b.close()


def test_batch_of_one_equals_single_context():
    cap = wl.small_capillary()
    a = lbib.from_capillaries([cap])
    b = lbib.from_capillary(cap)
    a.advance(50)
    b.advance(50)
    _same_state(a, 0, b, cap, 0)
    a.close()
    b.close()


def test_batch_invalid_arguments():
    lib = lbib.load()
    s = lbib.Solver([40, 50], 20)
    desc_xy = np.ascontiguousarray(wl.circle(20, 20, 10, 5).reshape(-1))
    d = lbib.lbib_membrane_desc(kind=wl.CELL, motion=wl.DEFORMABLE, nv=20, xy=lbib._dp(desc_xy), xy_ref=None,
                                ca=1e-3, beta=0.0, ka=1.0, density_ratio=1.0)
    i = lbib.ctypes.c_int32()
    assert lib.lbib_add_membrane_to(s.ctx, 2, lbib.ctypes.byref(d), lbib.ctypes.byref(i)) == lbib.LBIB_ERR_INVALID_ARG
    assert lib.lbib_add_membrane_to(s.ctx, -1, lbib.ctypes.byref(d), lbib.ctypes.byref(i)) == lbib.LBIB_ERR_INVALID_ARG
    for _ in range(16):
        assert lib.lbib_add_membrane_to(s.ctx, 1, lbib.ctypes.byref(d), lbib.ctypes.byref(i)) == lbib.LBIB_OK
    assert lib.lbib_add_membrane_to(s.ctx, 1, lbib.ctypes.byref(d), lbib.ctypes.byref(i)) == lbib.LBIB_ERR_UNSUPPORTED
    buf = np.zeros(2 * 50 * 20)
    assert lib.lbib_read_instance_velocity(s.ctx, 2, lbib._vp(buf), lbib._vp(buf), buf.size) == \
        lbib.LBIB_ERR_INVALID_ARG
    assert lib.lbib_read_instance_velocity(s.ctx, 1, lbib._vp(buf), lbib._vp(buf), 50 * 20 - 1) == \
        lbib.LBIB_ERR_INVALID_ARG
    s.close()
