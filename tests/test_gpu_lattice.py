"""GPU parity of the lattice kernels (bulk + near, no membranes): one and
several steps from random post-collision populations, compared element by
element with the oracle, on lattices that span several 32 x 4 tiles and end in
ragged tiles, for both boundary modes and both storage precisions."""
import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SHAPES = [(37, 9), (64, 8), (100, 23), (3, 2)]


def _pair(nx, ny, bc, storage, f0, tau=0.8, re=5.0, g=(0.0, 0.0)):
    o = oracle.OracleSim(nx, ny, tau=tau, re=re, bc=bc, g=g)
    o.set_fpost(f0)
    s = lbib.Solver(nx, ny, tau=tau, re=re, bc=bc, g=g, storage=storage)
    s.write_populations(f0)
    return o, s


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
def test_lattice_step_fp64_matches_oracle(nx, ny, bc):
    f0 = wl.random_populations(nx, ny, seed=nx * 7 + ny, eps=1e-2)
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    o, s = _pair(nx, ny, bc, lbib.LBIB_STORE_FP64, f0, g=g)
    for n in (1, 4):
        o.step(n)
        s.advance(n)
        fo, fg = o.fpost(), s.populations()
        assert np.abs(fg - fo).max() < 1e-14, np.abs(fg - fo).max()
        r, ux, uy = o.macro()
        gux, guy = s.velocity()
        assert np.abs(gux - ux).max() < 1e-14 and np.abs(guy - uy).max() < 1e-14
        assert np.abs(s.density() - r).max() < 1e-14
    s.close()


@pytest.mark.parametrize("nx,ny", SHAPES[:3])
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
def test_lattice_step_fp32_matches_oracle(nx, ny, bc):
    """FP32 deviations from the rest weights: the error stays at the FP32
    rounding of the deviations, bounded here by 8 ulp of max |f - w| per step
    (a few 1e-9 for these 1e-2 perturbations), far below the rounding of
    absolute FP32 populations (~3e-8 per operation).

    The velocity bound 9 tol follows from u_x = j_x / rho with the populations
    each within tol (eps = 2^-24, tol = 48 eps dev, rho >= 1 - 9 dev = 0.91):
    j_x sums six populations (6 tol) in five FP32 roundings of partial sums
    of at most 3 dev, 6 dev (18 eps dev = 0.375 tol), so over rho 7.0 tol;
    rho - 1 carries at most 9 tol plus eight roundings of at most 9 dev
    (1.5 tol), which |u_x| <= 6 dev / rho = 0.066 scales to 0.78 tol; the
    reciprocal (one ulp after its Newton step) and the product add 0.3 tol.
    Sum 8.0 tol, below 9 tol (dev is at most 1e-2 here)."""
    f0 = wl.random_populations(nx, ny, seed=nx * 5 + ny, eps=1e-2)
    f0 = np.asarray(np.asarray(f0 - np.array([4/9] + [1/9]*4 + [1/36]*4)[:, None, None], np.float32),
                    np.float64) + np.array([4/9] + [1/9]*4 + [1/36]*4)[:, None, None]
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    o, s = _pair(nx, ny, bc, lbib.LBIB_STORE_FP32, f0, g=g)
    w = np.array([4/9] + [1/9]*4 + [1/36]*4)[:, None, None]
    dev = np.abs(f0 - w).max()
    o.step(5)
    s.advance(5)
    fo, fg = o.fpost(), s.populations()
    tol = 8 * 2.0**-24 * dev * 6
    assert np.abs(fg - fo).max() < tol, (np.abs(fg - fo).max(), tol)
    r, ux, uy = o.macro()
    gux, guy = s.velocity()
    assert np.abs(gux - ux).max() < 9 * tol and np.abs(guy - uy).max() < 9 * tol
    s.close()


def test_forced_poiseuille_on_gpu_reaches_the_closed_form():
    """Property at any size: the GPU's steady forced channel is the BGK
    bounce-back closed form (parabola + slip) at FP64."""
    tau, ny = 1.0, 12
    nu = (tau - 0.5) / 3
    gx = 8 * nu * 0.02 / ny**2
    s = lbib.Solver(40, ny, tau=tau, re=0.0, bc=lbib.LBIB_BC_PERIODIC_FORCE, g=(gx, 0.0))
    s.advance(int(6 * ny * ny / nu) + 2000)
    ux, uy = s.velocity()
    y = np.arange(ny) + 0.5
    exact = gx / (2 * nu) * y * (ny - y) + gx * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
    assert np.abs(ux - exact[:, None]).max() < 1e-11 * exact.max()
    s.close()


def test_mass_is_conserved_in_a_periodic_channel_fp32():
    nx, ny = 300, 50
    f0 = wl.random_populations(nx, ny, seed=11, eps=1e-3)
    s = lbib.Solver(nx, ny, tau=0.7, re=0.0, bc=lbib.LBIB_BC_PERIODIC_FORCE, storage=lbib.LBIB_STORE_FP32)
    s.write_populations(f0)
    m0 = s.populations().sum()
    s.advance(500)
    assert abs(s.populations().sum() - m0) < 1e-9 * m0
    s.close()


def test_injected_nan_is_reported_as_divergence():
    """Host-side fault injection: a NaN population surfaces as
    LBIB_ERR_DIVERGED at the next sync, and the context stays usable."""
    nx, ny = 40, 8
    f0 = wl.random_populations(nx, ny, seed=3)
    f0[2, 4, 17] = np.nan
    s = lbib.Solver(nx, ny, tau=1.0, re=1.0)
    s.write_populations(f0)
    s.advance(2)
    with pytest.raises(lbib.LbibError) as e:
        s.sync()
    assert e.value.status == lbib.LBIB_ERR_DIVERGED
    s.close()


# the TMA-staged bulk update (launch option bulk_tma): x-halo copies at both
# ends of the row pitch, zero-filled rows beyond the walls, wall / inlet /
# outlet nodes on the global path, and the forced variant (periodic mode)
_TMA = dict(lagrangian_threads=512, near_blocks=1, bulk_tiles_y=1, activation_stride=4,
            bulk_nodes_per_thread=1, observables_branch=0, chain_programmatic=0, near_update_blocks=1,
            bulk_tma=1)


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
def test_tma_staged_bulk_update_matches_oracle_fp64(nx, ny, bc):
    f0 = wl.random_populations(nx, ny, seed=nx * 3 + ny, eps=1e-2)
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    o, s = _pair(nx, ny, bc, lbib.LBIB_STORE_FP64, f0, g=g)
    s.set_launch_config(**_TMA)
    assert s.launch_config()["bulk_tma"] == 1
    for n in (1, 4):
        o.step(n)
        s.advance(n)
        assert np.abs(s.populations() - o.fpost()).max() < 1e-14
    s.close()


@pytest.mark.parametrize("storage", [lbib.LBIB_STORE_FP32, lbib.LBIB_STORE_BF16, lbib.LBIB_STORE_FP16])
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
def test_tma_staged_bulk_update_equals_direct_loads(storage, bc):
    nx, ny = 100, 23
    f0 = wl.random_populations(nx, ny, seed=11, eps=1e-2)
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    out = []
    for tma in (0, 1):
        s = lbib.Solver(nx, ny, tau=0.8, re=5.0, bc=bc, g=g, storage=storage)
        s.write_populations(f0)
        s.set_launch_config(**dict(_TMA, bulk_tma=tma))
        s.advance(6)
        out.append(s.populations())
        s.close()
    assert np.array_equal(out[0], out[1])


# the vectorised bulk update (bulk_nodes_per_thread = 4): shuffled x shifts,
# edge loads at warp ends, wall rows, Zou-He or periodic wrap in the lanes
# holding an instance's end columns, partial vectors at a ragged end
_VEC = dict(_TMA, bulk_tma=0, bulk_nodes_per_thread=4)


@pytest.mark.parametrize("nx,ny", SHAPES + [(130, 6), (261, 13)])
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
@pytest.mark.parametrize("rt", [1, 4])
def test_vector_bulk_update_matches_oracle_fp64(nx, ny, bc, rt):
    f0 = wl.random_populations(nx, ny, seed=nx * 11 + ny, eps=1e-2)
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    o, s = _pair(nx, ny, bc, lbib.LBIB_STORE_FP64, f0, g=g)
    s.set_launch_config(**dict(_VEC, bulk_tiles_y=rt))
    assert s.launch_config()["bulk_nodes_per_thread"] == 4
    for n in (1, 4):
        o.step(n)
        s.advance(n)
        assert np.abs(s.populations() - o.fpost()).max() < 1e-14
    s.close()


@pytest.mark.parametrize("storage", [lbib.LBIB_STORE_FP32, lbib.LBIB_STORE_BF16, lbib.LBIB_STORE_FP16])
@pytest.mark.parametrize("bc", [lbib.LBIB_BC_INLET_OUTLET, lbib.LBIB_BC_PERIODIC_FORCE])
@pytest.mark.parametrize("nx,ny", [(100, 23), (3, 2), (261, 13)])
def test_vector_bulk_update_equals_one_node_per_thread(storage, bc, nx, ny):
    f0 = wl.random_populations(nx, ny, seed=13 + nx, eps=1e-2)
    g = (2e-5, -1e-5) if bc == lbib.LBIB_BC_PERIODIC_FORCE else (0.0, 0.0)
    out = []
    for npt in (1, 4):
        s = lbib.Solver(nx, ny, tau=0.8, re=5.0, bc=bc, g=g, storage=storage)
        s.write_populations(f0)
        s.set_launch_config(**dict(_VEC, bulk_nodes_per_thread=npt))
        s.advance(6)
        out.append(s.populations())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_vector_bulk_update_in_a_ragged_batch_equals_lone_runs():
    """Instances of 37, 3, 130 and 261 columns side by side (each starting on
    a tile column): the vector lanes at an instance's end see the next
    instance's columns as neighbours, and must not take their values."""
    widths = [37, 3, 130, 261]
    ny = 11
    caps = [wl.Capillary(f"w{n}", n, ny, 0.9, 5.0, 0, "fp32", 0, []) for n in widths]
    f0 = [wl.random_populations(n, ny, seed=n, eps=1e-2) for n in widths]
    b = lbib.from_capillaries(caps)
    for k, f in enumerate(f0):
        b.write_populations(f, instance=k)
    b.set_launch_config(**_VEC)
    b.advance(5)
    for k, c in enumerate(caps):
        s = lbib.from_capillary(c)
        s.write_populations(f0[k])
        s.set_launch_config(**dict(_VEC, bulk_nodes_per_thread=1))
        s.advance(5)
        assert np.array_equal(b.populations(instance=k), s.populations()), c.name
        s.close()
    b.close()
