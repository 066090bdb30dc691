"""Launch configurations and the autotuner, through the C ABI.

No launch configuration may change a result: the lattice kernels update every
node on its own, and the membrane kernel's sums follow one fixed order for
either block size.  So runs under different configurations are compared with
``np.array_equal``, and the autotuner must leave the state (and the
observables cursors) exactly as it found them."""
import dataclasses

import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CONFIGS = [(512, 608, 1, 4, 1, 0, 0, 2432, 0), (256, 300, 2, 1, 2, 1, 1, 1, 1), (256, 1, 4, 2, 1, 0, 1, 608, 0),
           (512, 2000, 4, 1, 2, 1, 0, 7, 1), (512, 9, 1, 2, 2, 0, 1, 5000, 0), (512, 608, 1, 1, 2, 0, 0, 2432, 1),
           (512, 608, 1, 1, 4, 0, 0, 2432, 0), (256, 300, 4, 2, 4, 1, 1, 16, 0), (512, 17, 2, 4, 4, 0, 0, 608, 0)]


def _snapshot(s, caps):
    out = {}
    for k in range(len(caps)):
        out[("u", k)] = s.velocity(k)
        out[("f", k)] = s.populations(k)
    nb = sum(len(c.bodies) for c in caps)
    for b in range(nb):
        out[("x", b)] = s.markers(b)
        out[("ft", b)] = s.body_field(b, "ftx")
    return out


def _equal(a, b):
    assert a.keys() == b.keys()
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, tuple):
            assert all(np.array_equal(p, q) for p, q in zip(x, y)), k
        else:
            assert np.array_equal(x, y), k


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16", "fp16"])
def test_every_launch_configuration_gives_the_same_state(storage):
    caps = [wl.small_capillary(), wl.sweep_capillary(300, 60, 0.75, 5e-4, "biconcave", 1, storage="fp64",
                                                      cell_markers=300, particle_markers=64, n_lig=60)]
    caps = [dataclasses.replace(c, storage=storage) for c in caps]
    ref = None
    for lt, nb, rt, st, npt, ob, pdl, nu, tma in CONFIGS:
        s = lbib.from_capillaries(caps)
        s.set_launch_config(lt, nb, rt, st, npt, ob, pdl, nu, tma)
        assert s.launch_config() == dict(lagrangian_threads=lt, near_blocks=nb, bulk_tiles_y=rt,
                                         activation_stride=st, bulk_nodes_per_thread=npt, observables_branch=ob,
                                         chain_programmatic=pdl, near_update_blocks=nu, bulk_tma=tma)
        s.advance(30)
        snap = _snapshot(s, caps)
        obs = [s.observables(instance=k) for k in range(len(caps))]
        if ref is None:
            ref = (snap, obs)
        else:
            _equal(ref[0], snap)
            assert obs == ref[1]
        s.close()


def test_autotune_leaves_the_state_and_cursors_unchanged():
    caps = [wl.small_capillary(), wl.small_capillary(seed=9)]
    a = lbib.from_capillaries(caps)
    b = lbib.from_capillaries(caps)
    a.advance(25)
    b.advance(25)
    assert len(a.observables(instance=0)) == 25
    before = _snapshot(a, caps)
    chosen = a.autotune(steps_per_trial=5)
    assert chosen == a.launch_config()
    assert chosen["lagrangian_threads"] in (256, 512) and chosen["bulk_tiles_y"] in (1, 2, 4)
    assert chosen["activation_stride"] in (1, 2, 4)
    assert chosen["observables_branch"] in (0, 1) and chosen["chain_programmatic"] in (0, 1)
    assert chosen["near_update_blocks"] >= 1
    assert a.step_count() == 25
    _equal(before, _snapshot(a, caps))
    assert a.observables(instance=0) == []  # cursor kept: nothing new since the last read
    a.advance(15)
    b.advance(15)
    _equal(_snapshot(a, caps), _snapshot(b, caps))
    oa, ob = a.observables(instance=1), b.observables(instance=1)
    assert [o["step"] for o in oa] == list(range(1, 41))
    assert oa == ob
    a.close()
    b.close()


def test_invalid_launch_configurations_are_rejected():
    s = lbib.from_capillary(wl.small_capillary())
    for bad in ((128, 100, 1, 4), (512, 0, 1, 4), (512, 100, 3, 4), (512, 100, 1, 3), (512, 100, 1, 4, 3),
                (512, 100, 1, 4, 8),
                (512, 100, 1, 4, 1, 2), (512, 100, 1, 4, 1, 0, 2), (512, 100, 1, 4, 1, 0, 0, -1), (512, 100, 1, 4, 1, 0, 0, 100, 2)):
        with pytest.raises(lbib.LbibError) as e:
            s.set_launch_config(*bad)
        assert e.value.status == lbib.LBIB_ERR_INVALID_ARG
    with pytest.raises(lbib.LbibError):
        s.autotune(steps_per_trial=0)
    s.close()
