"""Failure detection without a GPU fault: the library's error paths driven by
host-side fault injection (nothing here traps, faults or hangs a device).

* A bounded device wait that gives up (a bulk-update block waiting for a
  tensor copy, a tensor-core kernel of the surrogate network) surfaces as
  LBIB_ERR_TIMEOUT at the next status check, and the context or network then
  refuses work until a trusted state is loaded again.  The injection sets the
  same status bit the waits set; the waits' own limits are left as they are.
* A device allocation that fails makes the allocating call return
  LBIB_ERR_OOM, and what it had allocated is given back: after destroying the
  object the device's free memory is where it started."""
import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


def test_wait_timeout_is_reported_and_the_context_refuses_steps_until_restored():
    cap = wl.small_capillary()
    ref = lbib.from_capillary(cap)
    ref.advance(15)
    s = lbib.from_capillary(cap)
    s.advance(5)
    saved = s.save_state()
    s.advance(3)
    s.inject_fault(lbib.LBIB_FAULT_WAIT_TIMEOUT)
    for call in (s.sync, lambda: s.advance(1), s.velocity):
        with pytest.raises(lbib.LbibError) as e:
            call()
        assert e.value.status == lbib.LBIB_ERR_TIMEOUT
    with pytest.raises(lbib.LbibError) as e:  # a faulted state is not saved
        s.save_state()
    assert e.value.status == lbib.LBIB_ERR_TIMEOUT
    s.load_state(saved)  # a trusted state clears the fault
    s.advance(10)
    s.sync()
    for b in range(len(cap.bodies)):
        assert np.array_equal(s.markers(b), ref.markers(b))
    ux, uy = s.velocity()
    rx, ry = ref.velocity()
    assert np.array_equal(ux, rx) and np.array_equal(uy, ry)
    with pytest.raises(lbib.LbibError) as e:
        s.inject_fault(99)
    assert e.value.status == lbib.LBIB_ERR_INVALID_ARG
    s.close()
    ref.close()


def test_network_wait_timeout_is_reported_until_parameters_are_set_again():
    n = 256
    net = lbib.Mlp(7, 3, width=64, n_hidden=2, max_batch=n, seed=3)
    x = torch.rand(n, 7, device="cuda")
    t = torch.rand(n, 3, device="cuda")
    y0 = torch.empty(n, 3, device="cuda")
    y1 = torch.empty(n, 3, device="cuda")
    net.forward(x.data_ptr(), n, y0.data_ptr())
    net.sync()
    params = net.get_params()
    net.inject_fault()
    with pytest.raises(lbib.LbibError) as e:
        net.sync()
    assert e.value.status == lbib.LBIB_ERR_TIMEOUT
    for call in (lambda: net.forward(x.data_ptr(), n, y1.data_ptr()),
                 lambda: net.train_step(x.data_ptr(), t.data_ptr(), n, 1e-3)):
        with pytest.raises(lbib.LbibError) as e:
            call()
        assert e.value.status == lbib.LBIB_ERR_TIMEOUT
    net.set_params(params)
    net.sync()
    net.forward(x.data_ptr(), n, y1.data_ptr())
    net.sync()
    assert torch.equal(y0, y1)
    net.close()


def _compact_capillary():
    """A 96 x 30 channel with a deformable cell and a rigid adhering ellipse."""
    cell = wl.circle(48, 30.0, 15.0, 9.0)
    part = wl.ellipse(24, 60.0, 0.1 + 2.5, 6.0, 2.5)
    adh = wl.Adhesion(24, 1.0, 0.2, 0.1, 0.085, 1e-3, 25.0)
    return wl.Capillary("compact", 96, 30, 1.0, 0.5, 0, "fp32", 0, [
        wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-3, beta=1e-2),
        wl.Body(wl.PARTICLE, wl.RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1, adhesion=adh),
    ])


def _run_small(cap):
    s = lbib.from_capillary(cap)
    try:
        s.advance(3)
        s.sync()
    finally:
        s.close()


def test_failed_allocations_return_oom_and_leak_nothing():
    """Fail the k-th allocation for every k a context makes (creation, set-up
    at the first step, step graphs): each attempt ends in LBIB_ERR_OOM and,
    once the object is destroyed, the device holds exactly what it held before."""
    cap = _compact_capillary()
    _run_small(cap)  # loads the library's device code once
    base = _free_bytes()
    failures = 0
    try:
        for k in range(200):
            lbib.inject_alloc_failure(k)
            try:
                _run_small(cap)
            except lbib.LbibError as e:
                assert e.status == lbib.LBIB_ERR_OOM, (k, str(e))
                failures += 1
                assert _free_bytes() == base, k
                continue
            break  # k is past the last allocation: the run needed no more
    finally:
        lbib.inject_alloc_failure(-1)
    assert failures >= 2  # creation and set-up (one allocation each) were both hit
    assert _free_bytes() == base
    _run_small(cap)  # the injection is spent: a normal run again


def test_failed_network_allocation_returns_oom_and_leaks_nothing():
    lbib.Mlp(7, 3, width=64, n_hidden=2, max_batch=512).close()
    base = _free_bytes()
    failures = 0
    try:
        for k in range(100):
            lbib.inject_alloc_failure(k)
            try:
                lbib.Mlp(7, 3, width=64, n_hidden=2, max_batch=512).close()
            except lbib.LbibError as e:
                assert e.status == lbib.LBIB_ERR_OOM, (k, str(e))
                failures += 1
                assert _free_bytes() == base, k
                continue
            break
    finally:
        lbib.inject_alloc_failure(-1)
    assert failures > 5
    assert _free_bytes() == base


def test_failed_allocation_in_the_autotuner_leaves_the_context_usable():
    cap = _compact_capillary()
    a = lbib.from_capillary(cap)
    b = lbib.from_capillary(cap)
    a.advance(4)
    b.advance(4)
    try:
        lbib.inject_alloc_failure(0)  # the autotuner's state snapshot
        with pytest.raises(lbib.LbibError) as e:
            a.autotune(steps_per_trial=2)
        assert e.value.status == lbib.LBIB_ERR_OOM
    finally:
        lbib.inject_alloc_failure(-1)
    a.advance(6)
    b.advance(6)
    assert np.array_equal(a.markers(0), b.markers(0))
    a.close()
    b.close()


def test_destroyed_contexts_memory_is_reused_then_released():
    """lbib_destroy returns a context's device memory to the library's pool,
    which keeps it for the next context of the process; a second context of
    the same size allocates nothing new from the device, and
    lbib_release_cached_memory gives the memory back to the device."""
    cap = wl.Capillary("long", 6000, 150, 1.0, 1e-2, 0, "fp32", 0, [])  # ~65 MB of populations
    lbib.release_cached_memory(0)
    free0 = _free_bytes()
    lbib.from_capillary(cap).close()
    free1 = _free_bytes()
    assert free0 - free1 > 60e6  # kept by the pool
    s = lbib.from_capillary(cap)
    s.advance(2)
    s.sync()
    assert _free_bytes() == free1  # the second context reused it
    s.close()
    lbib.release_cached_memory(0)
    assert _free_bytes() >= free0 - (2 << 20)
    with pytest.raises(lbib.LbibError) as e:
        lbib.release_cached_memory(-1)
    assert e.value.status == lbib.LBIB_ERR_INVALID_ARG
