"""The allocation-free lattice stepper, called through the C ABI.

lbib_lattice_advance_noalloc exists for callers that cannot allocate device
memory where they step the fluid (an external memory manager owns the device,
or an allocation would synchronise or fail there): it runs the library's bulk
lattice kernel with all scratch taken from one fixed device array.  This test
checks that its result equals the allocating path (create, write the
populations, advance, read them back) on two calls in a row with different
lattices, inputs and step counts, so that the previous call's leftovers in the
shared array cannot leak into the next.  It lives in a file of its own that
pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _params(nx, ny, bc, storage, tau=0.8, re=5.0, g=(0.0, 0.0)):
    return lbib.lbib_fluid_params(nx=nx, ny=ny, tau=tau, re=re, rho_out=1.0, gx=g[0], gy=g[1], bc_mode=bc,
                                  storage=storage, device=0)


def _allocating(nx, ny, bc, storage, f0, nsteps, g):
    s = lbib.Solver(nx, ny, tau=0.8, re=5.0, bc=bc, g=g, storage=storage)
    s.write_populations(f0)
    s.advance(nsteps)
    out = s.populations()
    s.close()
    return out


@pytest.mark.parametrize("storage", [lbib.LBIB_STORE_FP64, lbib.LBIB_STORE_FP32])
def test_noalloc_matches_the_allocating_path_on_two_calls_in_a_row(storage):
    torch = pytest.importorskip("torch")
    cases = [(100, 23, lbib.LBIB_BC_INLET_OUTLET, 7, (0.0, 0.0), 11),
             (64, 40, lbib.LBIB_BC_PERIODIC_FORCE, 4, (2e-5, -1e-5), 12)]
    for nx, ny, bc, nsteps, g, seed in cases:
        f0 = wl.random_populations(nx, ny, seed=seed, eps=1e-2)
        ref = _allocating(nx, ny, bc, storage, f0, nsteps, g)
        dev = torch.tensor(f0, dtype=torch.float64, device="cuda").contiguous()
        p = _params(nx, ny, bc, storage, g=g)
        lbib.lbib_lattice_advance_noalloc(p, dev.data_ptr(), nsteps)
        out = dev.cpu().numpy()
        # the same kernel on the same deviations: identical up to FMA-free
        # conversions, i.e. bit for bit here; the lattice tests' FP64 bound
        # (1e-14) is the stated tolerance
        assert np.abs(out - ref).max() <= 1e-14, (nx, ny, np.abs(out - ref).max())


def test_noalloc_rejects_lattices_beyond_its_fixed_scratch():
    lib = lbib.load()
    p = _params(4000, 2000, lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_STORE_FP32)
    st = lib.lbib_lattice_advance_noalloc(ctypes.byref(p), ctypes.c_void_p(16), 1)
    assert st == lbib.LBIB_ERR_UNSUPPORTED
    assert b"scratch" in lib.lbib_last_error(None)
