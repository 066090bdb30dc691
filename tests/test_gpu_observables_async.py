"""lbib_read_latest_observables_async: records enqueued every step into
page-locked host memory equal the ring's records of the same steps (read
afterwards with the waiting call), instances without membranes and the
steps before the first membrane update report step = -1, and the loop does not
drain the step pipeline (the state after it equals a plain run's)."""
import dataclasses

import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _caps():
    a = wl.small_capillary()
    b = dataclasses.replace(wl.small_capillary(seed=1), nx=200)
    c = dataclasses.replace(wl.small_capillary(), nx=64, bodies=[])
    return [a, b, c]


def test_async_records_match_the_ring_and_keep_the_pipeline():
    K = 40
    s = lbib.from_capillaries(_caps(), obs_capacity=256)
    buf = torch.zeros((K, 3 * lbib.Solver.OBS_DTYPE.itemsize), dtype=torch.uint8).pin_memory()
    for k in range(K):
        s.advance(1)
        s.latest_observables_async(buf[k].data_ptr())
    s.sync()
    recs = buf.numpy().view(lbib.Solver.OBS_DTYPE).reshape(K, 3)
    assert recs[0]["step"].tolist() == [-1, -1, -1]  # the first membrane update runs with lattice step 2
    assert (recs[:, 2]["step"] == -1).all()
    for i in (0, 1):
        ring = {o["step"]: o for o in s.observables(instance=i)}
        steps = recs[1:, i]["step"]
        assert steps.tolist() == list(range(1, K))  # one step behind the lattice
        for k in range(1, K):
            o = ring[int(recs[k, i]["step"])]
            for f in ("t_star", "delta_p", "r", "n_l"):
                assert recs[k, i][f] == o[f], (i, k, f)
            assert recs[k, i]["n_bound"] == o["n_bound"]
    # the same steps without the reads give the same state
    p = lbib.from_capillaries(_caps(), obs_capacity=256)
    p.advance(K)
    for b in range(4):
        assert np.array_equal(p.markers(b), s.markers(b))
    # pageable memory also works (the call then waits for its copy)
    host = np.zeros(3, lbib.Solver.OBS_DTYPE)
    s.advance(1)
    s.latest_observables_async(host.ctypes.data)
    s.sync()
    assert host["step"][0] == K
    s.close()
    p.close()


def test_async_copies_survive_a_wrapping_ring():
    """With a ring of one record per instance every step overwrites the slot
    the previous read copies from: the step must wait for that copy, so the
    records equal those read through a ring that does not wrap."""
    K = 30
    bufs = []
    for cap in (256, 1):
        s = lbib.from_capillaries(_caps(), obs_capacity=cap)
        buf = torch.zeros((K, 3 * lbib.Solver.OBS_DTYPE.itemsize), dtype=torch.uint8).pin_memory()
        for k in range(K):
            s.advance(1)
            s.latest_observables_async(buf[k].data_ptr())
        s.advance(3)  # steps after the last read overwrite its slot too
        s.sync()
        bufs.append(buf.numpy().copy())
        s.close()
    assert np.array_equal(bufs[0], bufs[1])
    recs = bufs[1].view(lbib.Solver.OBS_DTYPE).reshape(K, 3)
    assert recs[1:, 0]["step"].tolist() == list(range(1, K))
