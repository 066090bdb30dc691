"""ctypes binding of the C ABI in ``include/lbib.h`` (same names, argument
marshalling only: every step of the time step runs in the library's CUDA
kernels).  Loading fails loudly if the library cannot be built or loaded; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

# ------------------------------------------------------------------ enums
LBIB_OK, LBIB_ERR_INVALID_ARG, LBIB_ERR_UNSUPPORTED, LBIB_ERR_CUDA = 0, 1, 2, 3
LBIB_ERR_OOM, LBIB_ERR_DIVERGED, LBIB_ERR_TIMEOUT, LBIB_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "OOM", 5: "DIVERGED",
                6: "TIMEOUT", 7: "STATE"}
LBIB_BC_INLET_OUTLET, LBIB_BC_PERIODIC_FORCE = 0, 1
LBIB_TRANSFER_PESKIN, LBIB_TRANSFER_MLS = 0, 1
LBIB_STORE_FP64, LBIB_STORE_FP32, LBIB_STORE_BF16, LBIB_STORE_FP16 = 0, 1, 2, 3
STORAGE_CODES = {"fp64": LBIB_STORE_FP64, "fp32": LBIB_STORE_FP32, "bf16": LBIB_STORE_BF16, "fp16": LBIB_STORE_FP16}
LBIB_CELL, LBIB_PARTICLE = 0, 1
LBIB_DEFORMABLE, LBIB_RIGID, LBIB_FIXED = 0, 1, 2
LBIB_FAULT_WAIT_TIMEOUT = 1
FIELDS = ("x", "y", "xp", "yp", "uvx", "uvy", "fsx", "fsy", "fbx", "fby", "fax", "fay",
          "fpx", "fpy", "fwx", "fwy", "fhx", "fhy", "ftx", "fty", "vx", "vy",
          "mx", "my", "mfx", "mfy", "mds")


class lbib_fluid_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("re", ctypes.c_double), ("rho_out", ctypes.c_double), ("gx", ctypes.c_double),
                ("gy", ctypes.c_double), ("bc_mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("device", ctypes.c_int32), ("obs_capacity", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("transfer", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lbib_membrane_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("motion", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("xy", ctypes.POINTER(ctypes.c_double)),
                ("xy_ref", ctypes.POINTER(ctypes.c_double)), ("ca", ctypes.c_double),
                ("beta", ctypes.c_double), ("ka", ctypes.c_double), ("density_ratio", ctypes.c_double)]


class lbib_adhesion_params(ctypes.Structure):
    _fields_ = [("n_ligands", ctypes.c_int32), ("reserved", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("y_cr", ctypes.c_double), ("y_eq", ctypes.c_double), ("kf_dt", ctypes.c_double),
                ("kr0_dt", ctypes.c_double), ("xi", ctypes.c_double)]


class lbib_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t_star", ctypes.c_double), ("delta_p", ctypes.c_double),
                ("r", ctypes.c_double), ("n_l", ctypes.c_double), ("n_bound", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class lbib_launch_config(ctypes.Structure):
    _fields_ = [("lagrangian_threads", ctypes.c_int32), ("near_blocks", ctypes.c_int32),
                ("bulk_tiles_y", ctypes.c_int32), ("activation_stride", ctypes.c_int32),
                ("bulk_nodes_per_thread", ctypes.c_int32), ("observables_branch", ctypes.c_int32),
                ("chain_programmatic", ctypes.c_int32), ("near_update_blocks", ctypes.c_int32),
                ("bulk_tma", ctypes.c_int32)]


class lbib_mlp_desc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("width", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("device", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("in_shift", ctypes.POINTER(ctypes.c_float)), ("in_scale", ctypes.POINTER(ctypes.c_float)),
                ("out_shift", ctypes.POINTER(ctypes.c_float)), ("out_scale", ctypes.POINTER(ctypes.c_float))]


_P = ctypes.c_void_p
_SIGS = {
    "lbib_create": [ctypes.POINTER(lbib_fluid_params), ctypes.POINTER(_P)],
    "lbib_add_membrane": [_P, ctypes.POINTER(lbib_membrane_desc), ctypes.POINTER(ctypes.c_int32)],
    "lbib_set_adhesion": [_P, ctypes.c_int32, ctypes.POINTER(lbib_adhesion_params)],
    "lbib_advance": [_P, ctypes.c_int64],
    "lbib_sync": [_P],
    "lbib_step_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "lbib_read_velocity": [_P, _P, _P, ctypes.c_size_t],
    "lbib_read_density": [_P, _P, ctypes.c_size_t],
    "lbib_read_velocity_device": [_P, _P, _P, ctypes.c_size_t, ctypes.c_int32],
    "lbib_read_populations": [_P, _P, ctypes.c_size_t],
    "lbib_write_populations": [_P, _P, ctypes.c_size_t],
    "lbib_read_observables": [_P, ctypes.POINTER(lbib_obs), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "lbib_read_markers": [_P, ctypes.c_int32, _P, ctypes.c_size_t],
    "lbib_read_body_field": [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t],
    "lbib_read_bonds": [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t],
    "lbib_state_size": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "lbib_save_state": [_P, _P, ctypes.c_size_t],
    "lbib_load_state": [_P, _P, ctypes.c_size_t],
    "lbib_set_profiling": [_P, ctypes.c_int32],
    "lbib_read_kernel_times": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float)],
    "lbib_describe": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                      ctypes.POINTER(ctypes.c_int32)],
    "lbib_lattice_advance_noalloc": [ctypes.POINTER(lbib_fluid_params), _P, ctypes.c_int64],
    "lbib_create_batch": [ctypes.POINTER(lbib_fluid_params), ctypes.c_int32, _P, _P, ctypes.POINTER(_P)],
    "lbib_add_membrane_to": [_P, ctypes.c_int32, ctypes.POINTER(lbib_membrane_desc), ctypes.POINTER(ctypes.c_int32)],
    "lbib_read_instance_velocity": [_P, ctypes.c_int32, _P, _P, ctypes.c_size_t],
    "lbib_read_instance_populations": [_P, ctypes.c_int32, _P, ctypes.c_size_t],
    "lbib_write_instance_populations": [_P, ctypes.c_int32, _P, ctypes.c_size_t],
    "lbib_read_instance_observables": [_P, ctypes.c_int32, ctypes.POINTER(lbib_obs), ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)],
    "lbib_read_latest_observables": [_P, ctypes.POINTER(lbib_obs), ctypes.c_size_t],
    "lbib_read_latest_observables_async": [_P, _P, ctypes.c_size_t],
    "lbib_get_launch_config": [_P, ctypes.POINTER(lbib_launch_config)],
    "lbib_set_launch_config": [_P, ctypes.POINTER(lbib_launch_config)],
    "lbib_autotune": [_P, ctypes.c_int32, ctypes.POINTER(lbib_launch_config)],
    "lbib_mlp_create": [ctypes.POINTER(lbib_mlp_desc), ctypes.POINTER(_P)],
    "lbib_mlp_forward": [_P, _P, ctypes.c_int32, _P],
    "lbib_mlp_train_step": [_P, _P, _P, ctypes.c_int32, ctypes.c_float, _P],
    "lbib_mlp_gradients": [_P, _P, _P, ctypes.c_int32, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_float)],
    "lbib_mlp_backward": [_P, _P, _P, ctypes.c_int32, _P, ctypes.c_size_t, _P],
    "lbib_mlp_apply_gradient": [_P, _P, ctypes.c_size_t, ctypes.c_float, ctypes.c_float],
    "lbib_mlp_param_count": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "lbib_mlp_get_params": [_P, _P, ctypes.c_size_t],
    "lbib_mlp_set_params": [_P, _P, ctypes.c_size_t],
    "lbib_mlp_sync": [_P],
    "lbib_mlp_inject_fault": [_P, ctypes.c_int32],
    "lbib_inject_fault": [_P, ctypes.c_int32],
    "lbib_release_cached_memory": [ctypes.c_int32],
    "lbib_add_membranes": [_P, ctypes.c_int32, _P, _P, _P, _P],
}

_lib = None
_lock = threading.Lock()


def checked() -> bool:
    """True when LBIB_CHECKED=1 in the environment: the process loads the
    bounds-checked debug build (liblbib_checked.so) instead of liblbib.so."""
    return os.environ.get("LBIB_CHECKED", "0") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load() -> ctypes.CDLL:
    """Build (if stale) and load liblbib.so (the checked build with
    LBIB_CHECKED=1); raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=checked())
            lib = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.lbib_last_error.argtypes = [_P]
            lib.lbib_last_error.restype = ctypes.c_char_p
            lib.lbib_destroy.argtypes = [_P]
            lib.lbib_destroy.restype = None
            lib.lbib_mlp_destroy.argtypes = [_P]
            lib.lbib_mlp_destroy.restype = None
            lib.lbib_inject_alloc_failure.argtypes = [ctypes.c_int64]
            lib.lbib_inject_alloc_failure.restype = None
            _lib = lib
        return _lib


class LbibError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbib {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, ctx) -> None:
    if status != LBIB_OK:
        msg = load().lbib_last_error(ctx).decode(errors="replace")
        raise LbibError(status, msg)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------ one-to-one wrappers

def lbib_create(params: lbib_fluid_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lbib_create(ctypes.byref(params), ctypes.byref(h)), None)
    return h


def lbib_create_batch(params: lbib_fluid_params, nx, seeds=None) -> ctypes.c_void_p:
    nxa = np.ascontiguousarray(np.asarray(nx, dtype=np.int32))
    sa = None if seeds is None else np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    h = ctypes.c_void_p()
    _check(load().lbib_create_batch(ctypes.byref(params), len(nxa), _vp(nxa), None if sa is None else _vp(sa),
                                    ctypes.byref(h)), None)
    return h


def lbib_add_membrane(ctx, desc: lbib_membrane_desc) -> int:
    i = ctypes.c_int32()
    _check(load().lbib_add_membrane(ctx, ctypes.byref(desc), ctypes.byref(i)), ctx)
    return i.value


def lbib_add_membrane_to(ctx, instance: int, desc: lbib_membrane_desc) -> int:
    i = ctypes.c_int32()
    _check(load().lbib_add_membrane_to(ctx, int(instance), ctypes.byref(desc), ctypes.byref(i)), ctx)
    return i.value


def lbib_set_adhesion(ctx, body: int, params: lbib_adhesion_params) -> None:
    _check(load().lbib_set_adhesion(ctx, body, ctypes.byref(params)), ctx)


def lbib_advance(ctx, nsteps: int) -> None:
    _check(load().lbib_advance(ctx, int(nsteps)), ctx)


def lbib_sync(ctx) -> None:
    _check(load().lbib_sync(ctx), ctx)


def lbib_destroy(ctx) -> None:
    load().lbib_destroy(ctx)


def lbib_lattice_advance_noalloc(params: lbib_fluid_params, f_device_ptr: int, nsteps: int) -> None:
    """Allocation-free lattice stepping of a membrane-free channel on a caller
    device buffer of 9 nx ny doubles (see include/lbib.h)."""
    _check(load().lbib_lattice_advance_noalloc(ctypes.byref(params), ctypes.c_void_p(f_device_ptr),
                                                int(nsteps)), None)


def _config_dict(c: lbib_launch_config) -> dict:
    return dict(lagrangian_threads=c.lagrangian_threads, near_blocks=c.near_blocks, bulk_tiles_y=c.bulk_tiles_y,
                activation_stride=c.activation_stride, bulk_nodes_per_thread=c.bulk_nodes_per_thread,
                observables_branch=c.observables_branch, chain_programmatic=c.chain_programmatic,
                near_update_blocks=c.near_update_blocks, bulk_tma=c.bulk_tma)


class Solver:
    """A context plus its geometry, driven through the C ABI.  ``nx`` is one
    channel length (a single capillary) or a sequence of them (a batch of
    capillaries sharing ny and the fluid parameters, one Philox seed each:
    ``seeds`` or seed + i)."""

    def __init__(self, nx, ny, tau=1.0, re=1e-2, rho_out=1.0, bc=LBIB_BC_INLET_OUTLET, g=(0.0, 0.0),
                 storage=LBIB_STORE_FP64, device=0, seed=0, stream: Optional[int] = None, obs_capacity=0,
                 seeds=None, transfer=0):
        self.lib = load()
        batch = np.ndim(nx) > 0
        nxs = [int(v) for v in (nx if batch else [nx])]
        p = lbib_fluid_params(nx=nxs[0], ny=int(ny), tau=float(tau), re=float(re), rho_out=float(rho_out),
                              gx=float(g[0]), gy=float(g[1]), bc_mode=int(bc), storage=int(storage),
                              device=int(device), obs_capacity=int(obs_capacity),
                              cuda_stream=stream, seed=int(seed) & (2**64 - 1), transfer=int(transfer))
        self.nxs, self.ny = nxs, int(ny)
        self.nx = nxs[0]
        self.ctx = lbib_create_batch(p, nxs, seeds) if batch else lbib_create(p)
        self.nv = []
        self.nlig = {}

    # lifetime
    def close(self):
        if getattr(self, "ctx", None):
            lbib_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, status):
        _check(status, self.ctx)

    # set-up
    def add_membrane(self, kind, motion, xy, xy_ref=None, ca=1e-3, beta=0.0, ka=1.0, density_ratio=1.0,
                     instance=0) -> int:
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1))
        ref = None if xy_ref is None else np.ascontiguousarray(np.asarray(xy_ref, dtype=np.float64).reshape(-1))
        d = lbib_membrane_desc(kind=int(kind), motion=int(motion), nv=len(xy) // 2, xy=_dp(xy),
                               xy_ref=_dp(ref) if ref is not None else None, ca=float(ca), beta=float(beta),
                               ka=float(ka), density_ratio=float(density_ratio))
        i = lbib_add_membrane_to(self.ctx, instance, d)
        self.nv.append(len(xy) // 2)
        return i

    def set_adhesion(self, body, n_lig, sigma, y_cr, y_eq, kf_dt, kr0_dt, xi=0.0):
        a = lbib_adhesion_params(n_ligands=int(n_lig), sigma=float(sigma), y_cr=float(y_cr), y_eq=float(y_eq),
                                 kf_dt=float(kf_dt), kr0_dt=float(kr0_dt), xi=float(xi))
        lbib_set_adhesion(self.ctx, int(body), a)
        self.nlig[int(body)] = int(n_lig)

    # stepping
    def advance(self, n=1):
        lbib_advance(self.ctx, n)

    def sync(self):
        lbib_sync(self.ctx)

    def inject_fault(self, kind=LBIB_FAULT_WAIT_TIMEOUT):
        """Failure-detection tests: raise a bounded-wait timeout in stream order."""
        self._c(self.lib.lbib_inject_fault(self.ctx, int(kind)))

    def step_count(self) -> int:
        s = ctypes.c_int64()
        self._c(self.lib.lbib_step_count(self.ctx, ctypes.byref(s)))
        return s.value

    # reads
    def velocity(self, instance=0):
        ux = np.zeros((self.ny, self.nxs[instance])); uy = np.zeros_like(ux)
        self._c(self.lib.lbib_read_instance_velocity(self.ctx, int(instance), _vp(ux), _vp(uy), ux.size))
        return ux, uy

    def density(self):
        r = np.zeros((self.ny, self.nx))
        self._c(self.lib.lbib_read_density(self.ctx, _vp(r), r.size))
        return r

    def velocity_device(self, ux_ptr: int, uy_ptr: int, n: int, dtype: int):
        self._c(self.lib.lbib_read_velocity_device(self.ctx, ctypes.c_void_p(ux_ptr), ctypes.c_void_p(uy_ptr),
                                                   n, dtype))

    def populations(self, instance=0):
        f = np.zeros((9, self.ny, self.nxs[instance]))
        self._c(self.lib.lbib_read_instance_populations(self.ctx, int(instance), _vp(f), f.size))
        return f

    def write_populations(self, f, instance=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nxs[instance])
        self._c(self.lib.lbib_write_instance_populations(self.ctx, int(instance), _vp(f), f.size))

    def observables(self, cap=1 << 16, instance=0):
        buf = (lbib_obs * cap)()
        n = ctypes.c_size_t()
        self._c(self.lib.lbib_read_instance_observables(self.ctx, int(instance), buf, cap, ctypes.byref(n)))
        return [dict(step=o.step, t_star=o.t_star, delta_p=o.delta_p, r=o.r, n_l=o.n_l, n_bound=o.n_bound,
                     status=o.status) for o in buf[:n.value]]

    def latest_observables(self):
        """Record of the last completed step of every instance (one copy)."""
        buf = (lbib_obs * len(self.nxs))()
        self._c(self.lib.lbib_read_latest_observables(self.ctx, buf, len(self.nxs)))
        return [dict(step=o.step, t_star=o.t_star, delta_p=o.delta_p, r=o.r, n_l=o.n_l, n_bound=o.n_bound,
                     status=o.status) for o in buf]

    # numpy layout of lbib_obs (48 bytes)
    OBS_DTYPE = np.dtype([("step", "<i8"), ("t_star", "<f8"), ("delta_p", "<f8"), ("r", "<f8"), ("n_l", "<f8"),
                          ("n_bound", "<i4"), ("status", "<i4")])

    def latest_observables_async(self, out_ptr: int):
        """Enqueues the copy of every instance's newest record into host memory
        at out_ptr (n_instances records of OBS_DTYPE, ideally page-locked) and
        returns at once; valid after sync()."""
        self._c(self.lib.lbib_read_latest_observables_async(self.ctx, ctypes.c_void_p(out_ptr), len(self.nxs)))

    def markers(self, body):
        xy = np.zeros(2 * self.nv[body])
        self._c(self.lib.lbib_read_markers(self.ctx, int(body), _vp(xy), xy.size))
        return xy.reshape(-1, 2)

    def body_field(self, body, field):
        out = np.zeros(self.nv[body])
        self._c(self.lib.lbib_read_body_field(self.ctx, int(body), FIELDS.index(field), _vp(out), out.size))
        return out

    def bonds(self, body):
        n = self.nlig[int(body)]
        bound = np.zeros(n, np.int32); ax = np.zeros(n); ay = np.zeros(n); mg = np.zeros(n)
        self._c(self.lib.lbib_read_bonds(self.ctx, int(body), _vp(bound), _vp(ax), _vp(ay), _vp(mg), n))
        return bound, ax, ay, mg

    def state_size(self) -> int:
        n = ctypes.c_size_t()
        self._c(self.lib.lbib_state_size(self.ctx, ctypes.byref(n)))
        return n.value

    def save_state(self) -> bytearray:
        buf = bytearray(self.state_size())
        arr = (ctypes.c_char * len(buf)).from_buffer(buf)
        self._c(self.lib.lbib_save_state(self.ctx, ctypes.cast(arr, ctypes.c_void_p), len(buf)))
        return buf

    def load_state(self, buf: bytearray):
        arr = (ctypes.c_char * len(buf)).from_buffer(buf)
        self._c(self.lib.lbib_load_state(self.ctx, ctypes.cast(arr, ctypes.c_void_p), len(buf)))

    def set_profiling(self, on: bool):
        self._c(self.lib.lbib_set_profiling(self.ctx, 1 if on else 0))

    def kernel_times(self):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        self._c(self.lib.lbib_read_kernel_times(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def launch_config(self) -> dict:
        c = lbib_launch_config()
        self._c(self.lib.lbib_get_launch_config(self.ctx, ctypes.byref(c)))
        return _config_dict(c)

    def set_launch_config(self, lagrangian_threads, near_blocks, bulk_tiles_y, activation_stride=4,
                          bulk_nodes_per_thread=1, observables_branch=0, chain_programmatic=0,
                          near_update_blocks=0, bulk_tma=0):
        """near_update_blocks 0 keeps the current grid of the near lattice update."""
        if not near_update_blocks:
            near_update_blocks = self.launch_config()["near_update_blocks"]
        c = lbib_launch_config(lagrangian_threads=int(lagrangian_threads), near_blocks=int(near_blocks),
                               bulk_tiles_y=int(bulk_tiles_y), activation_stride=int(activation_stride),
                               bulk_nodes_per_thread=int(bulk_nodes_per_thread),
                               observables_branch=int(observables_branch),
                               chain_programmatic=int(chain_programmatic),
                               near_update_blocks=int(near_update_blocks), bulk_tma=int(bulk_tma))
        self._c(self.lib.lbib_set_launch_config(self.ctx, ctypes.byref(c)))

    def autotune(self, steps_per_trial=20) -> dict:
        """Times candidate launch configurations on this context's state and
        keeps the fastest; the state is unchanged (see include/lbib.h)."""
        c = lbib_launch_config()
        self._c(self.lib.lbib_autotune(self.ctx, int(steps_per_trial), ctypes.byref(c)))
        return _config_dict(c)

    def describe(self):
        k, n, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._c(self.lib.lbib_describe(self.ctx, ctypes.byref(k), ctypes.byref(n), ctypes.byref(t)))
        return dict(kernels_per_step=k.value, near_tiles=n.value, tiles=t.value)


def from_capillary(cap, storage=None, device=0, stream=None, obs_capacity=0) -> Solver:
    """A Solver holding the lattice and bodies of a workloads.Capillary."""
    st = storage
    if st is None:
        st = STORAGE_CODES[cap.storage]
    s = Solver(cap.nx, cap.ny, tau=cap.tau, re=cap.re, rho_out=cap.rho_out, bc=cap.bc, g=cap.g, storage=st,
               device=device, seed=cap.seed, stream=stream, obs_capacity=obs_capacity, transfer=cap.transfer)
    _add_bodies(s, cap, 0)
    return s


class Mlp:
    """The surrogate network of include/lbib_mlp.h.  Device arrays are passed
    as raw pointers (e.g. ``tensor.data_ptr()`` of contiguous float32 CUDA
    tensors); this class only marshals arguments."""

    def __init__(self, n_in, n_out, width=256, n_hidden=3, max_batch=65536, device=0, stream=None, seed=0,
                 in_shift=None, in_scale=None, out_shift=None, out_scale=None):
        self.lib = load()
        keep = []

        def fp(v):
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
            keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

        d = lbib_mlp_desc(n_in=int(n_in), width=int(width), n_hidden=int(n_hidden), n_out=int(n_out),
                          max_batch=int(max_batch), device=int(device), cuda_stream=stream,
                          seed=int(seed) & (2**64 - 1), in_shift=fp(in_shift), in_scale=fp(in_scale),
                          out_shift=fp(out_shift), out_scale=fp(out_scale))
        h = ctypes.c_void_p()
        _check(self.lib.lbib_mlp_create(ctypes.byref(d), ctypes.byref(h)), None)
        self.net = h
        self.n_in, self.n_out, self.width, self.n_hidden = int(n_in), int(n_out), int(width), int(n_hidden)

    def close(self):
        if getattr(self, "net", None):
            self.lib.lbib_mlp_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(st, None)

    def sync(self):
        self._c(self.lib.lbib_mlp_sync(self.net))

    def inject_fault(self, kind=LBIB_FAULT_WAIT_TIMEOUT):
        """Failure-detection tests: raise a bounded-wait timeout in stream order."""
        self._c(self.lib.lbib_mlp_inject_fault(self.net, int(kind)))

    def forward(self, x_ptr: int, batch: int, y_ptr: int):
        self._c(self.lib.lbib_mlp_forward(self.net, ctypes.c_void_p(x_ptr), int(batch), ctypes.c_void_p(y_ptr)))

    def train_step(self, x_ptr: int, t_ptr: int, batch: int, lr: float, loss_ptr: Optional[int] = None):
        self._c(self.lib.lbib_mlp_train_step(self.net, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(batch),
                                             float(lr), ctypes.c_void_p(loss_ptr) if loss_ptr else None))

    def param_count(self) -> int:
        n = ctypes.c_size_t()
        self._c(self.lib.lbib_mlp_param_count(self.net, ctypes.byref(n)))
        return n.value

    def gradients(self, x_ptr: int, t_ptr: int, batch: int):
        g = np.zeros(self.param_count(), np.float32)
        loss = ctypes.c_float()
        self._c(self.lib.lbib_mlp_gradients(self.net, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(batch),
                                            _vp(g), g.size, ctypes.byref(loss)))
        return g, loss.value

    def backward(self, x_ptr: int, t_ptr: int, batch: int, grad_ptr: int, n: int, loss_ptr: Optional[int] = None):
        """Gradient of the batch loss into the device array at grad_ptr (n floats), no update."""
        self._c(self.lib.lbib_mlp_backward(self.net, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(batch),
                                           ctypes.c_void_p(grad_ptr), int(n),
                                           ctypes.c_void_p(loss_ptr) if loss_ptr else None))

    def apply_gradient(self, grad_ptr: int, n: int, scale: float, lr: float):
        """One Adam step with scale * the device gradient at grad_ptr."""
        self._c(self.lib.lbib_mlp_apply_gradient(self.net, ctypes.c_void_p(grad_ptr), int(n), float(scale),
                                                 float(lr)))

    def get_params(self):
        p = np.zeros(self.param_count(), np.float32)
        self._c(self.lib.lbib_mlp_get_params(self.net, _vp(p), p.size))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        self._c(self.lib.lbib_mlp_set_params(self.net, _vp(p), p.size))

    def layers(self, p=None):
        """Split a flat parameter vector into [(W, b), ...] (hidden layers, then output)."""
        p = self.get_params() if p is None else p
        dims = [self.n_in] + [self.width] * self.n_hidden + [self.n_out]
        out, k = [], 0
        for i, o in zip(dims[:-1], dims[1:]):
            W = p[k:k + o * i].reshape(o, i)
            k += o * i
            b = p[k:k + o]
            k += o
            out.append((W, b))
        return out


def _add_bodies(s: Solver, cap, instance: int) -> None:
    _add_all(s, [(instance, b) for b in cap.bodies])


# numpy images of lbib_membrane_desc and lbib_adhesion_params (same fields, same offsets),
# so a batch's descriptors are filled as arrays rather than one ctypes object each
_MEMBRANE_DT = np.dtype([("kind", "<i4"), ("motion", "<i4"), ("nv", "<i4"), ("reserved", "<i4"), ("xy", "<u8"),
                         ("xy_ref", "<u8"), ("ca", "<f8"), ("beta", "<f8"), ("ka", "<f8"),
                         ("density_ratio", "<f8")], align=True)
_ADHESION_DT = np.dtype([("n_ligands", "<i4"), ("reserved", "<i4"), ("sigma", "<f8"), ("y_cr", "<f8"),
                         ("y_eq", "<f8"), ("kf_dt", "<f8"), ("kr0_dt", "<f8"), ("xi", "<f8")], align=True)
assert _MEMBRANE_DT.itemsize == ctypes.sizeof(lbib_membrane_desc)
assert _ADHESION_DT.itemsize == ctypes.sizeof(lbib_adhesion_params)


def _addr(a: np.ndarray) -> int:
    return a.__array_interface__["data"][0]


class _Records:
    """lbib_add_membranes' arguments for a list of (instance, workloads.Body):
    the descriptors (one array, filled a field at a time), every body's
    vertices (and stress-free vertices) copied into one array the descriptors
    point into, the adhesion records and a pointer per body (0: none).  The
    library copies what the pointers reach during the call; `keep` holds the
    arrays until then."""

    def __init__(self, items):
        n = len(items)
        bodies = [b for _, b in items]
        self.inst = np.fromiter((int(i) for i, _ in items), np.int32, n)
        xys = [np.ascontiguousarray(b.xy, dtype=np.float64).reshape(-1) for b in bodies]
        sizes = np.fromiter((x.size for x in xys), np.int64, n)
        self.nv = sizes // 2
        d = np.zeros(n, _MEMBRANE_DT)
        d["kind"] = [int(b.kind) for b in bodies]
        d["motion"] = [int(b.motion) for b in bodies]
        d["nv"] = self.nv
        flat = np.concatenate(xys) if n else np.zeros(0)
        d["xy"] = _addr(flat) + 8 * (np.cumsum(sizes) - sizes)
        with_ref = [k for k, b in enumerate(bodies) if b.xy_ref is not None]
        flat_ref = np.zeros(0)
        if with_ref:
            refs = [np.ascontiguousarray(bodies[k].xy_ref, dtype=np.float64).reshape(-1) for k in with_ref]
            rsz = np.fromiter((r.size for r in refs), np.int64, len(refs))
            flat_ref = np.concatenate(refs)
            d["xy_ref"][with_ref] = _addr(flat_ref) + 8 * (np.cumsum(rsz) - rsz)
        d["ca"] = [float(b.ca) for b in bodies]
        d["beta"] = [float(b.beta) for b in bodies]
        d["ka"] = [float(b.ka) for b in bodies]
        d["density_ratio"] = [float(b.density_ratio) for b in bodies]
        self.descs = d
        self.with_adh = [k for k, b in enumerate(bodies) if b.adhesion is not None]
        ads = [bodies[k].adhesion for k in self.with_adh]
        adh = np.zeros(len(ads), _ADHESION_DT)
        if ads:
            adh["n_ligands"] = [int(a.n_lig) for a in ads]
            for f, attr in (("sigma", "sigma"), ("y_cr", "y_cr"), ("y_eq", "y_eq"), ("kf_dt", "kf_dt"),
                            ("kr0_dt", "kr0_dt"), ("xi", "xi")):
                adh[f] = [float(getattr(a, attr)) for a in ads]
        self.adh = adh
        self.n_lig = [int(a.n_lig) for a in ads]
        self.adh_ptr = np.zeros(n, np.uint64)
        if ads:
            self.adh_ptr[self.with_adh] = _addr(adh) + _ADHESION_DT.itemsize * np.arange(len(ads), dtype=np.uint64)
        self.keep = (flat, flat_ref, adh)


def _add_all(s: Solver, items) -> None:
    """Every (instance, workloads.Body) of `items` in one lbib_add_membranes call."""
    n = len(items)
    if n == 0:
        return
    r = _Records(items)
    ids = np.zeros(n, np.int32)
    s._c(s.lib.lbib_add_membranes(s.ctx, n, _vp(r.inst), _vp(r.descs), _vp(r.adh_ptr), _vp(ids)))
    s.nv.extend(int(v) for v in r.nv)
    for k, nl in zip(r.with_adh, r.n_lig):
        s.nlig[int(ids[k])] = nl


def from_capillaries(caps, storage=None, device=0, stream=None, obs_capacity=0) -> Solver:
    """One batched Solver holding every workloads.Capillary of ``caps`` as its
    instances (same ny, tau, Re, boundary mode, body force and storage; each
    keeps its own length, bodies and seed)."""
    c0 = caps[0]
    for c in caps:
        if (c.ny, c.tau, c.re, c.rho_out, c.bc, tuple(c.g), c.storage, c.transfer) != \
                (c0.ny, c0.tau, c0.re, c0.rho_out, c0.bc, tuple(c0.g), c0.storage, c0.transfer):
            raise ValueError("instances of a batch share ny and the fluid parameters")
    st = storage
    if st is None:
        st = STORAGE_CODES[c0.storage]
    s = Solver([c.nx for c in caps], c0.ny, tau=c0.tau, re=c0.re, rho_out=c0.rho_out, bc=c0.bc, g=c0.g,
               storage=st, device=device, stream=stream, obs_capacity=obs_capacity, seeds=[c.seed for c in caps],
               transfer=c0.transfer)
    _add_all(s, [(k, b) for k, c in enumerate(caps) for b in c.bodies])
    return s


def inject_alloc_failure(after: int) -> None:
    """Failure-detection tests: the (after + 1)-th device allocation the
    library makes from now on fails as out of memory (once); after < 0 cancels."""
    load().lbib_inject_alloc_failure(int(after))


def release_cached_memory(device: int = 0) -> None:
    """Give the device memory the library keeps for the next context back
    to the device (waits for the device)."""
    _check(load().lbib_release_cached_memory(int(device)), None)


def roofline_bytes_per_node(storage: int) -> int:
    """Algorithmic DRAM bytes of one lattice-node update: 9 populations read and
    written once each."""
    return 2 * 9 * {LBIB_STORE_FP64: 8, LBIB_STORE_FP32: 4, LBIB_STORE_BF16: 2, LBIB_STORE_FP16: 2}[storage]


__all__ = [n for n in dir() if n.startswith("lbib_") or n.startswith("LBIB_")] + [
    "Solver", "Mlp", "from_capillary", "from_capillaries", "load", "library_path", "LbibError", "roofline_bytes_per_node", "FIELDS",
    "inject_alloc_failure", "release_cached_memory"]
