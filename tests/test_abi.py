"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/lbib.h declares, and its ctypes structs match the header's layout.
CPU only: no compute call is made."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2210_06043_gb300 import build, lbib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("lbib.h", "lbib_mlp.h")]


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbib_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbib_create", "lbib_add_membrane", "lbib_set_adhesion", "lbib_advance", "lbib_sync",
                     "lbib_read_velocity", "lbib_read_observables", "lbib_read_markers", "lbib_save_state",
                     "lbib_load_state", "lbib_destroy", "lbib_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbib_\w+)", out))
    assert set(declared_functions()) <= exported


def _c_layout():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbib.h"
#include "lbib_mlp.h"
#define O(t, f) printf("%s.%s %zu\n", #t, #f, offsetof(t, f))
#define S(t) printf("%s.sizeof %zu\n", #t, sizeof(t))
int main(void) {
  S(lbib_fluid_params); O(lbib_fluid_params, tau); O(lbib_fluid_params, bc_mode);
  O(lbib_fluid_params, obs_capacity); O(lbib_fluid_params, cuda_stream); O(lbib_fluid_params, seed);
  O(lbib_fluid_params, transfer);
  S(lbib_membrane_desc); O(lbib_membrane_desc, xy); O(lbib_membrane_desc, xy_ref); O(lbib_membrane_desc, density_ratio);
  S(lbib_adhesion_params); O(lbib_adhesion_params, sigma); O(lbib_adhesion_params, xi);
  S(lbib_obs); O(lbib_obs, n_l); O(lbib_obs, n_bound); O(lbib_obs, status);
  S(lbib_launch_config); O(lbib_launch_config, near_blocks); O(lbib_launch_config, bulk_tiles_y);
  O(lbib_launch_config, activation_stride); O(lbib_launch_config, bulk_nodes_per_thread);
  O(lbib_launch_config, observables_branch); O(lbib_launch_config, chain_programmatic);
  O(lbib_launch_config, near_update_blocks); O(lbib_launch_config, bulk_tma);
  S(lbib_mlp_desc); O(lbib_mlp_desc, cuda_stream); O(lbib_mlp_desc, seed); O(lbib_mlp_desc, out_scale);
  return 0;
}
'''
    d = os.path.join(ROOT, "paper_2210_06043_gb300", "_build")
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "layout.c")
    exe = os.path.join(d, "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.strip().splitlines())


def test_ctypes_structs_match_the_header():
    lay = _c_layout()
    for cls in (lbib.lbib_fluid_params, lbib.lbib_membrane_desc, lbib.lbib_adhesion_params, lbib.lbib_obs,
                lbib.lbib_launch_config, lbib.lbib_mlp_desc):
        name = cls.__name__
        assert int(lay[f"{name}.sizeof"]) == ctypes.sizeof(cls), name
        for key, val in lay.items():
            t, f = key.split(".")
            if t == name and f != "sizeof":
                assert getattr(cls, f).offset == int(val), key


def test_create_reports_errors_through_the_boundary():
    """Invalid parameters are rejected before any device work; a missing GPU
    surfaces as an error status with a message, never a crash."""
    lib = lbib.load()
    p = lbib.lbib_fluid_params(nx=2, ny=10, tau=1.0, re=0.01, rho_out=1.0)
    h = ctypes.c_void_p()
    assert lib.lbib_create(ctypes.byref(p), ctypes.byref(h)) == lbib.LBIB_ERR_INVALID_ARG
    assert b"nx" in lib.lbib_last_error(None)
    p = lbib.lbib_fluid_params(nx=16, ny=8, tau=0.5, re=0.01, rho_out=1.0)
    assert lib.lbib_create(ctypes.byref(p), ctypes.byref(h)) == lbib.LBIB_ERR_INVALID_ARG
    p = lbib.lbib_fluid_params(nx=16, ny=8, tau=1.0, re=0.01, rho_out=1.0, storage=7)
    assert lib.lbib_create(ctypes.byref(p), ctypes.byref(h)) == lbib.LBIB_ERR_INVALID_ARG
    p = lbib.lbib_fluid_params(nx=16, ny=8, tau=1.0, re=0.01, rho_out=1.0, transfer=2)
    assert lib.lbib_create(ctypes.byref(p), ctypes.byref(h)) == lbib.LBIB_ERR_INVALID_ARG
    assert b"transfer" in lib.lbib_last_error(None)
    p = lbib.lbib_fluid_params(nx=16, ny=8, tau=1.0, re=0.01, rho_out=1.0, device=0)
    st = lib.lbib_create(ctypes.byref(p), ctypes.byref(h))
    if st == lbib.LBIB_OK:  # a GPU is present
        lib.lbib_destroy(h)
    else:
        assert st == lbib.LBIB_ERR_CUDA and lib.lbib_last_error(None)


def test_create_batch_reports_errors_through_the_boundary():
    lib = lbib.load()
    p = lbib.lbib_fluid_params(nx=0, ny=10, tau=1.0, re=0.01, rho_out=1.0)
    h = ctypes.c_void_p()
    nx = np.array([40, 2, 50], dtype=np.int32)
    assert lib.lbib_create_batch(ctypes.byref(p), 3, nx.ctypes.data, None, ctypes.byref(h)) == \
        lbib.LBIB_ERR_INVALID_ARG
    assert lib.lbib_create_batch(ctypes.byref(p), 0, nx.ctypes.data, None, ctypes.byref(h)) == \
        lbib.LBIB_ERR_INVALID_ARG
    assert lib.lbib_create_batch(ctypes.byref(p), 2, None, None, ctypes.byref(h)) == lbib.LBIB_ERR_INVALID_ARG
    # 9 * (sum of padded widths) * ny must stay below 2^31
    big = np.full(4, 1 << 23, dtype=np.int32)
    assert lib.lbib_create_batch(ctypes.byref(p), 4, big.ctypes.data, None, ctypes.byref(h)) == \
        lbib.LBIB_ERR_UNSUPPORTED


def test_bounds_checked_build_compiles_and_exports_every_declared_symbol():
    """The debug build with the index checks compiled in (-DLBIB_CHECKED) is a
    separate library with the same boundary; lbib picks it with LBIB_CHECKED=1."""
    path = build.build(checked=True)
    assert path.endswith("liblbib_checked.so") and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(declared_functions()) <= set(re.findall(r"\bT (lbib_\w+)", out))
    env_before = os.environ.get("LBIB_CHECKED")
    try:
        os.environ["LBIB_CHECKED"] = "1"
        assert lbib.library_path() == path
        os.environ["LBIB_CHECKED"] = "0"
        assert lbib.library_path() == build.LIB
    finally:
        if env_before is None:
            os.environ.pop("LBIB_CHECKED", None)
        else:
            os.environ["LBIB_CHECKED"] = env_before
