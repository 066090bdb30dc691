"""Pins of the oracle's storage-rounding mode: the precisions a library may
store the post-collision deviations g = f - w_i in (binary32, bfloat16 of
the binary32 value, binary16 of the binary32 value times 2^14, each rounded to
nearest with ties to even), checked against independent implementations
(numpy's float32 and float16 casts; the round-to-nearest-even bit recipe on
float32 words for bfloat16), and the mode's effect on a run: every stored
deviation is representable, and exact storage leaves the run unchanged.
CPU only."""
import numpy as np
import pytest

import oracle
from paper_2210_06043_gb300 import workloads as wl

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]


def _samples():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(scale=s, size=400) for s in (1e-9, 1e-6, 1e-4, 1e-2, 0.3)])
    # exact ties of each format: halfway between two neighbours
    ties = [1 + 2.0**-8, 1 + 3 * 2.0**-8, (1 + 2.0**-11) / 16384, (1 + 3 * 2.0**-11) / 16384, 2.0**-20 + 2.0**-45]
    return np.concatenate([x, ties, -np.array(ties), [0.0]])


def _bf16_rne(x32):
    u = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def test_binary32_storage_is_numpys_float32():
    for g in _samples():
        assert oracle.round_store(oracle.STORE_F32, g) == float(np.float32(g))


def test_binary16_storage_is_numpys_float16_of_the_scaled_binary32():
    for g in _samples():
        ref = float(np.float16(np.float32(g) * np.float32(16384))) / 16384
        assert oracle.round_store(oracle.STORE_F16, g) == ref, g


def test_bfloat16_storage_is_round_to_nearest_even_of_the_binary32():
    for g in _samples():
        assert oracle.round_store(oracle.STORE_BF16, g) == float(_bf16_rne(np.float32(g))), g
    assert oracle.round_store(oracle.STORE_BF16, 1 / 3) == 0.333984375


@pytest.mark.parametrize("kind,dtype", [(oracle.STORE_F32, np.float32), (oracle.STORE_F16, None),
                                        (oracle.STORE_BF16, None)])
def test_rounded_runs_store_only_representable_deviations(kind, dtype):
    cap = wl.small_capillary()
    s = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, bc=cap.bc, seed=cap.seed)
    s.set_storage_rounding(kind)
    s.step(3)
    g = (s.fpost() - W).ravel()
    again = np.array([oracle.round_store(kind, v) for v in g[:: max(1, g.size // 5000)]])
    assert np.array_equal(again, g[:: max(1, g.size // 5000)])
    if dtype is not None:
        assert np.array_equal(g.astype(dtype).astype(np.float64), g)


def test_exact_storage_leaves_the_run_unchanged():
    cap = wl.small_capillary()
    a = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, bc=cap.bc, seed=cap.seed)
    b = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, bc=cap.bc, seed=cap.seed)
    b.set_storage_rounding(oracle.STORE_EXACT)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.fpost(), b.fpost())
    with pytest.raises(ValueError):
        b.set_storage_rounding(7)
