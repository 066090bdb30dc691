"""FP64 CPU oracle of the hybrid LBM-IBM time step (ctypes wrapper).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2210_06043_gb300``; the two meet only
through the seeded input generators of ``paper_2210_06043_gb300.workloads``,
which hold no arithmetic of the method.

The C source ``lbib_oracle.c`` states, equation by equation, what each function
follows in the paper (Coclite et al., J. Fluids Struct.).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbib_oracle.so")
_lock = threading.Lock()
_lib = None

BC_INLET_OUTLET, BC_PERIODIC_FORCE = 0, 1
CELL, PARTICLE = 0, 1
DEFORMABLE, RIGID, FIXED = 0, 1, 2
TRANSFER_PESKIN, TRANSFER_MLS = 0, 1
STORE_EXACT, STORE_F32, STORE_BF16, STORE_F16 = 0, 1, 2, 3

# order of the per-vertex arrays exposed by orc_get_body
BODY_FIELDS = (
    "x", "y", "xp", "yp", "uvx", "uvy", "fsx", "fsy", "fbx", "fby", "fax", "fay",
    "fpx", "fpy", "fwx", "fwy", "fhx", "fhy", "ftx", "fty", "vx", "vy",
    "mx", "my", "mfx", "mfy", "mds",
)
BODY_SCALARS = (
    "A0", "P0", "ks", "kb", "mv", "mass", "inertia", "xc", "yc", "ang",
    "area", "perim", "cx", "cy", "sigma", "nl0",
)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        U64, I64 = ctypes.c_uint64, ctypes.c_int64
        sig = {
            "orc_lattice": (None, [P, P, P, P]),
            "orc_equilibrium": (None, [D, D, D, P]),
            "orc_guo_term": (None, [D, D, D, D, D, P]),
            "orc_stream_bc": (None, [I, I, I, D, D, P, P]),
            "orc_phi": (D, [D]),
            "orc_dphi": (D, [D]),
            "orc_mls_weight": (D, [D]),
            "orc_interp": (D, [I, I, P, D, D, P, P, P, I, I]),
            "orc_spread": (None, [I, I, I, P, P, P, P, P, P, P, I]),
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_bond_uniform": (D, [U64, I64, ctypes.c_uint32]),
            "orc_polygon": (None, [I, P, P, P]),
            "orc_stretch_energy": (D, [I, P, P, P, D]),
            "orc_membrane_forces": (None, [I, P, P, P, P, D, D, D, D, D, P, P, P, P, P, P]),
            "orc_repulsion_magnitude": (D, [D]),
            "orc_rigid_bdf2": (D, [D, D, D]),
            "orc_create": (P, [I, I, D, D, D, I, D, D, U64]),
            "orc_destroy": (None, [P]),
            "orc_set_repulsion_cutoff": (None, [P, D]),
            "orc_set_transfer": (I, [P, I]),
            "orc_add_body": (I, [P, I, I, I, P, P, D, D, D, D]),
            "orc_set_adhesion": (I, [P, I, I, D, D, D, D, D, D]),
            "orc_set_fpost": (None, [P, P]),
            "orc_get_fpost": (None, [P, P]),
            "orc_get_macro": (None, [P, P, P, P]),
            "orc_set_macro": (None, [P, P, P, P]),
            "orc_get_force": (None, [P, P, P]),
            "orc_umax": (D, [P]),
            "orc_step_count": (I64, [P]),
            "orc_diverged": (I, [P]),
            "orc_get_obs": (None, [P, P]),
            "orc_get_body": (I, [P, I, I, P]),
            "orc_get_body_scalars": (None, [P, I, P]),
            "orc_get_bonds": (I, [P, I, P, P, P, P]),
            "orc_body_traction": (None, [P, I, P, P]),
            "orc_step": (None, [P]),
            "orc_run": (None, [P, I64]),
            "orc_set_threads": (I, [I]),
            "orc_round_store": (D, [I, D]),
            "orc_set_storage_rounding": (I, [P, I]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> int:
    """Host threads of the node loops (the results do not depend on it);
    returns the count in use."""
    return _load().orc_set_threads(int(n))


# ------------------------------------------------------------ pieces (pins)

def lattice():
    """(ex, ey, w, opp) of Eq. 3 as built by the oracle."""
    lib = _load()
    ex = np.zeros(9, np.int32); ey = np.zeros(9, np.int32)
    w = np.zeros(9); opp = np.zeros(9, np.int32)
    lib.orc_lattice(_p(ex), _p(ey), _p(w), _p(opp))
    return ex, ey, w, opp


def equilibrium(rho, ux, uy):
    out = np.zeros(9)
    _load().orc_equilibrium(rho, ux, uy, _p(out))
    return out


def guo_term(ux, uy, fx, fy, tau):
    out = np.zeros(9)
    _load().orc_guo_term(ux, uy, fx, fy, tau, _p(out))
    return out


def stream_bc(fpost, bc=BC_INLET_OUTLET, umax=0.0, rho_out=1.0):
    """Eq. 1 left-hand side plus boundary conditions on a [9, ny, nx] array."""
    fpost = _f64(fpost)
    _, ny, nx = fpost.shape
    out = np.zeros_like(fpost)
    _load().orc_stream_bc(nx, ny, bc, umax, rho_out, _p(fpost), _p(out))
    return out


def phi(r):
    return _load().orc_phi(float(r))


def dphi(r):
    return _load().orc_dphi(float(r))


def mls_weight(r):
    return _load().orc_mls_weight(float(r))


def interp(field, X, Y, renorm=False, kind=TRANSFER_PESKIN):
    """(W, value, d/dX, d/dY) of the interpolant: Peskin velocity-type
    (stencil truncated at the walls) or, with renorm, density-type; or, with
    kind=TRANSFER_MLS, the moving-least-squares fit (W = the sum of its shape
    functions, gradients its linear coefficients)."""
    field = _f64(field)
    ny, nx = field.shape
    v = ctypes.c_double(); gx = ctypes.c_double(); gy = ctypes.c_double()
    W = _load().orc_interp(nx, ny, _p(field), float(X), float(Y), ctypes.byref(v),
                           ctypes.byref(gx), ctypes.byref(gy), int(bool(renorm)), int(kind))
    return W, v.value, gx.value, gy.value


def spread(nx, ny, X, Y, Fx, Fy, ds, kind=TRANSFER_PESKIN):
    X, Y, Fx, Fy, ds = map(_f64, (X, Y, Fx, Fy, ds))
    ox = np.zeros((ny, nx)); oy = np.zeros((ny, nx))
    _load().orc_spread(nx, ny, len(X), _p(X), _p(Y), _p(Fx), _p(Fy), _p(ds), _p(ox), _p(oy), int(kind))
    return ox, oy


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def bond_uniform(seed, step, site):
    return _load().orc_bond_uniform(int(seed), int(step), int(site))


def round_store(kind, g):
    """A deviation as stored in precision `kind` (STORE_*)."""
    return _load().orc_round_store(int(kind), float(g))


def polygon(xy):
    """{A, P, cx, cy, Jc} of a closed chain given as an (nv, 2) array."""
    xy = _f64(xy)
    x = _f64(xy[:, 0]); y = _f64(xy[:, 1])
    out = np.zeros(5)
    _load().orc_polygon(len(x), _p(x), _p(y), _p(out))
    return dict(zip(("A", "P", "cx", "cy", "Jc"), out))


def stretch_energy(xy, l0, ks):
    xy = _f64(xy); x = _f64(xy[:, 0]); y = _f64(xy[:, 1]); l0 = _f64(l0)
    return _load().orc_stretch_energy(len(x), _p(x), _p(y), _p(l0), ks)


def membrane_forces(xy, l0, th0, A0, ks, kb, ka, pref=1.0 / 3.0):
    """Per-vertex (F^s, F^b, F^a), each (nv, 2)."""
    xy = _f64(xy); x = _f64(xy[:, 0]); y = _f64(xy[:, 1])
    l0 = _f64(l0); th0 = _f64(th0)
    nv = len(x)
    o = [np.zeros(nv) for _ in range(6)]
    _load().orc_membrane_forces(nv, _p(x), _p(y), _p(l0), _p(th0), A0, ks, kb, ka, pref,
                                *[_p(a) for a in o])
    return (np.stack([o[0], o[1]], 1), np.stack([o[2], o[3]], 1), np.stack([o[4], o[5]], 1))


def repulsion_magnitude(d):
    return _load().orc_repulsion_magnitude(float(d))


def rigid_bdf2(u1, u2, acc):
    return _load().orc_rigid_bdf2(u1, u2, acc)


# --------------------------------------------------------------- the sim

class OracleSim:
    """One capillary instance stepped by the oracle."""

    def __init__(self, nx, ny, tau=1.0, re=1e-2, rho_out=1.0, bc=BC_INLET_OUTLET,
                 g=(0.0, 0.0), seed=0):
        self._lib = _load()
        self.nx, self.ny = int(nx), int(ny)
        h = self._lib.orc_create(self.nx, self.ny, float(tau), float(re), float(rho_out), int(bc),
                                 float(g[0]), float(g[1]), int(seed) & (2**64 - 1))
        if not h:
            raise ValueError("oracle rejected the lattice parameters")
        self._h = ctypes.c_void_p(h)
        self.nv = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def umax(self):
        return self._lib.orc_umax(self._h)

    @property
    def step_count(self):
        return self._lib.orc_step_count(self._h)

    @property
    def diverged(self):
        return bool(self._lib.orc_diverged(self._h))

    def set_repulsion_cutoff(self, d):
        self._lib.orc_set_repulsion_cutoff(self._h, float(d))

    def set_storage_rounding(self, kind):
        """Round the stored deviations to precision `kind` (STORE_*) after every
        collision, and the current state at once."""
        if self._lib.orc_set_storage_rounding(self._h, int(kind)) != 0:
            raise ValueError("unknown storage kind")

    def set_transfer(self, kind):
        if self._lib.orc_set_transfer(self._h, int(kind)) != 0:
            raise ValueError("unknown transfer kernel")

    def add_body(self, kind, motion, xy, xy_ref=None, ca=1e-3, beta=0.0, ka=1.0, density_ratio=1.0):
        xy = _f64(np.asarray(xy).reshape(-1))
        ref = None if xy_ref is None else _f64(np.asarray(xy_ref).reshape(-1))
        bid = self._lib.orc_add_body(self._h, int(kind), int(motion), len(xy) // 2, _p(xy),
                                     None if ref is None else _p(ref), float(ca), float(beta),
                                     float(ka), float(density_ratio))
        if bid < 0:
            raise ValueError("oracle rejected the body")
        self.nv.append(len(xy) // 2)
        return bid

    def set_adhesion(self, body, n_lig, sigma, y_cr, y_eq, kf_dt, kr0_dt, xi=0.0):
        r = self._lib.orc_set_adhesion(self._h, int(body), int(n_lig), float(sigma), float(y_cr),
                                       float(y_eq), float(kf_dt), float(kr0_dt), float(xi))
        if r != 0:
            raise ValueError("oracle rejected the adhesion parameters")

    def step(self, n=1):
        self._lib.orc_run(self._h, int(n))

    def fpost(self):
        out = np.zeros((9, self.ny, self.nx))
        self._lib.orc_get_fpost(self._h, _p(out))
        return out

    def set_fpost(self, f):
        f = _f64(f)
        assert f.shape == (9, self.ny, self.nx)
        self._lib.orc_set_fpost(self._h, _p(f))

    def macro(self):
        r = np.zeros((self.ny, self.nx)); ux = np.zeros_like(r); uy = np.zeros_like(r)
        self._lib.orc_get_macro(self._h, _p(r), _p(ux), _p(uy))
        return r, ux, uy

    def set_macro(self, rho, ux, uy):
        self._lib.orc_set_macro(self._h, _p(_f64(rho)), _p(_f64(ux)), _p(_f64(uy)))

    def force_field(self):
        fx = np.zeros((self.ny, self.nx)); fy = np.zeros_like(fx)
        self._lib.orc_get_force(self._h, _p(fx), _p(fy))
        return fx, fy

    def body(self, b, field):
        out = np.zeros(self.nv[b])
        self._lib.orc_get_body(self._h, int(b), BODY_FIELDS.index(field), _p(out))
        return out

    def body_xy(self, b):
        return np.stack([self.body(b, "x"), self.body(b, "y")], 1)

    def body_scalars(self, b):
        out = np.zeros(len(BODY_SCALARS))
        self._lib.orc_get_body_scalars(self._h, int(b), _p(out))
        return dict(zip(BODY_SCALARS, out))

    def bonds(self, b, n_lig):
        bound = np.zeros(n_lig, np.int32); ax = np.zeros(n_lig); ay = np.zeros(n_lig)
        margin = np.zeros(n_lig)
        self._lib.orc_get_bonds(self._h, int(b), _p(bound), _p(ax), _p(ay), _p(margin))
        return bound, ax, ay, margin

    def traction(self, b):
        fx = np.zeros(self.nv[b]); fy = np.zeros(self.nv[b])
        self._lib.orc_body_traction(self._h, int(b), _p(fx), _p(fy))
        return fx, fy

    def obs(self):
        out = np.zeros(6)
        self._lib.orc_get_obs(self._h, _p(out))
        return dict(zip(("step", "t_star", "delta_p", "r", "n_l", "n_bound"), out))
