"""Seeded synthetic inputs: membrane meshes and capillary configurations.

This module produces inputs only (vertex coordinates, parameter sets and random
population fields).  It holds none of the time-step arithmetic and is the one
module that both the CUDA library's tests and the CPU oracle's tests draw their
inputs from.

Geometry follows the problem statement of Coclite et al. (Sec. 3.1): a channel
of height H = 7.5 um whose lattice resolution is set by ``ny`` nodes across; a
deformable cell of 7 um released on the centre line at x = 5 um; a particle of
length b = 2 um and thickness h deposited on the lower wall at x = 12.5 um with
a 12.5 nm gap.  The biconcave shape is the parametrisation of Eq. 20, read as
x = alpha sin q, y = (alpha / 2)(0.207 + 2.003 sin^2 q - 1.123 sin^4 q) cos q
with alpha the 3.5 um cell radius, turned so that its long axis spans the
channel height (the 7 um cell is "slightly smaller than the height of the
channel").
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Optional

import numpy as np

H_UM = 7.5  # channel height, Sec. 3.1
CELL_RADIUS_UM = 3.5  # Sec. 3.1
CELL_X_UM, CELL_Y_UM = 5.0, 3.75  # release point, Sec. 3.1
PARTICLE_X_UM, PARTICLE_GAP_UM = 12.5, 0.0125  # Sec. 3.1
PARTICLE_LENGTH_UM = 2.0  # b, Sec. 3.1
Y_CR_UM = 0.025  # critical bond length, Sec. 2.5

CELL, PARTICLE = 0, 1
DEFORMABLE, RIGID, FIXED = 0, 1, 2


def _resample_closed(pts: np.ndarray, n: int) -> np.ndarray:
    """n points equally spaced in arc length along a densely sampled closed curve."""
    closed = np.vstack([pts, pts[:1]])
    seg = np.hypot(np.diff(closed[:, 0]), np.diff(closed[:, 1]))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    target = np.arange(n) * s[-1] / n
    x = np.interp(target, s, closed[:, 0])
    y = np.interp(target, s, closed[:, 1])
    return np.stack([x, y], 1)


def _ccw(xy: np.ndarray) -> np.ndarray:
    x, y = xy[:, 0], xy[:, 1]
    a2 = np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    return xy if a2 > 0 else xy[::-1].copy()


def circle(n: int, cx: float, cy: float, r: float, phase: float = 0.0) -> np.ndarray:
    t = phase + 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], 1)


def ellipse(n: int, cx: float, cy: float, a: float, b: float, dense: int = 20000) -> np.ndarray:
    """Counter-clockwise ellipse with semi-axes a (x) and b (y), equal arc spacing,
    vertex 0 at the lowest point."""
    t = -0.5 * np.pi + 2.0 * np.pi * np.arange(dense) / dense
    pts = np.stack([a * np.cos(t), b * np.sin(t)], 1)
    return _ccw(_resample_closed(pts, n)) + np.array([cx, cy])


def rectangle(n: int, cx: float, cy: float, b: float, h: float) -> np.ndarray:
    """Counter-clockwise b x h rectangle, n vertices equally spaced in arc
    length starting mid-base (exact points on the polygonal path)."""
    corners = np.array([[0.0, -h / 2], [b / 2, -h / 2], [b / 2, h / 2], [-b / 2, h / 2],
                        [-b / 2, -h / 2], [0.0, -h / 2]])
    seg = np.hypot(*np.diff(corners, axis=0).T)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    t = np.arange(n) * s[-1] / n
    pts = np.stack([np.interp(t, s, corners[:, 0]), np.interp(t, s, corners[:, 1])], 1)
    return _ccw(pts) + np.array([cx, cy])


def biconcave(n: int, cx: float, cy: float, alpha: float, across: bool = True,
              dense: int = 20000) -> np.ndarray:
    """Eq. 20 shape (reading above), equal arc spacing, counter-clockwise.
    across=True turns the long axis to the y direction."""
    q = -0.5 * np.pi + 2.0 * np.pi * np.arange(dense) / dense
    s = np.sin(q)
    x = alpha * s
    y = 0.5 * alpha * (0.207 + 2.003 * s**2 - 1.123 * s**4) * np.cos(q)
    pts = np.stack([x, y], 1)
    if across:
        pts = np.stack([-y, x], 1)
    return _ccw(_resample_closed(pts, n)) + np.array([cx, cy])


def random_populations(nx: int, ny: int, seed: int = 0, eps: float = 1e-3) -> np.ndarray:
    """w_i (1 + e), e ~ U(-eps, eps): [9, ny, nx] post-collision populations."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rng = np.random.default_rng(seed)
    return w[:, None, None] * (1.0 + rng.uniform(-eps, eps, size=(9, ny, nx)))


@dataclasses.dataclass
class Adhesion:
    n_lig: int
    sigma: float  # in units rho_ref nu_ref^2 / H (Sec. 2.5); inf => fixed particle
    y_cr: float  # lattice units
    y_eq: float
    kf_dt: float
    kr0_dt: float
    xi: float  # force sensitivity of the reverse rate, 1 / lattice length^2


@dataclasses.dataclass
class Body:
    kind: int
    motion: int
    xy: np.ndarray
    ca: float
    beta: float
    ka: float = 1.0
    density_ratio: float = 1.0
    xy_ref: Optional[np.ndarray] = None
    adhesion: Optional[Adhesion] = None


@dataclasses.dataclass
class Capillary:
    name: str
    nx: int
    ny: int
    tau: float
    re: float
    steps: int
    storage: str  # "fp64" | "fp32"
    seed: int
    bodies: List[Body]
    bc: int = 0  # 0 inlet/outlet, 1 periodic + body force
    g: tuple = (0.0, 0.0)
    rho_out: float = 1.0
    transfer: int = 0  # 0 Peskin delta, 1 moving least squares

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def markers(self) -> int:
        return int(sum(len(b.xy) for b in self.bodies))


def _bond_defaults(ny: int, n_lig: int, sigma: float) -> Adhesion:
    dx = H_UM / ny
    y_cr = Y_CR_UM / dx
    y_eq = 0.5 * y_cr  # Sec. 2.5
    # k_f / k_r0 = 8.5e3 (Sec. 3.1); the per-step values are this project's choice
    return Adhesion(n_lig=n_lig, sigma=sigma, y_cr=y_cr, y_eq=y_eq, kf_dt=0.085, kr0_dt=1e-5,
                    xi=1.0 / (y_eq * y_eq))


def small_capillary(seed: int = 0) -> Capillary:
    """240 x 60 nodes (H = 60 dx), Re = 1e-2, tau = 1, biconcave 7 um cell with
    128 markers (spring + bending), rigid 2 x 0.5 um elliptical particle with 32
    markers bonded to the lower wall by 40 ligand sites; 2000 steps in FP64."""
    nx, ny = 240, 60
    dx = H_UM / ny
    cell = biconcave(128, CELL_X_UM / dx, CELL_Y_UM / dx, CELL_RADIUS_UM / dx)
    a, b = 0.5 * PARTICLE_LENGTH_UM / dx, 0.5 * 0.5 / dx
    part = ellipse(32, PARTICLE_X_UM / dx, PARTICLE_GAP_UM / dx + b, a, b)
    bodies = [
        Body(CELL, DEFORMABLE, cell, ca=1e-3, beta=1e-2),
        Body(PARTICLE, RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1,
             adhesion=_bond_defaults(ny, 40, 1.0)),
    ]
    return Capillary("capillary 240x60, biconcave cell + rigid ellipse, fp64", nx, ny, 1.0, 1e-2,
                     2000, "fp64", seed, bodies)


def production_capillary(seed: int = 0) -> Capillary:
    """1200 x 150 nodes (H = 150 dx), Re = 1e-2, tau = 1, globular 7 um cell
    with 256 markers, soft discoidal 2 x 1 um particle (Ca = 1e-3, aspect ratio
    0.5) with 96 markers and 200 ligand sites; FP32 populations, 2e5 steps."""
    nx, ny = 1200, 150
    dx = H_UM / ny
    cell = circle(256, CELL_X_UM / dx, CELL_Y_UM / dx, CELL_RADIUS_UM / dx)
    a, b = 0.5 * PARTICLE_LENGTH_UM / dx, 0.5 * 1.0 / dx
    part = ellipse(96, PARTICLE_X_UM / dx, PARTICLE_GAP_UM / dx + b, a, b)
    bodies = [
        Body(CELL, DEFORMABLE, cell, ca=1e-3, beta=0.0),
        Body(PARTICLE, DEFORMABLE, part, ca=1e-3, beta=1e-2, density_ratio=1.1,
             adhesion=_bond_defaults(ny, 200, 1.0)),
    ]
    return Capillary("capillary 1200x150, globular cell + soft ellipse (AR 0.5), fp32", nx, ny, 1.0,
                     1e-2, 200000, "fp32", seed, bodies)


# parameter sweep of Sec. 3.1: particle aspect ratio h / b, particle capillary
# number (0: rigid), cell shape, and two bond-kinetics seeds
SWEEP_AR = (0.25, 0.5, 0.75, 1.0)
SWEEP_CA = (0.0, 1e-4, 5e-4, 1e-3)
SWEEP_CELLS = ("globular", "biconcave")
SWEEP_SEEDS = (0, 1)


def sweep_capillary(nx: int, ny: int, ar: float, ca: float, cell: str, seed: int,
                    storage: str = "fp32", cell_markers: int = 256, particle_markers: int = 96,
                    n_lig: int = 200) -> Capillary:
    """One capillary of the sweep: a 7 um cell (globular or biconcave) at the
    release point and a 2 um particle of thickness ar * 2 um on the lower wall
    (rigid when ca == 0, else deformable with that Ca), 200 ligand sites."""
    dx = H_UM / ny
    if cell == "globular":
        c = circle(cell_markers, CELL_X_UM / dx, CELL_Y_UM / dx, CELL_RADIUS_UM / dx)
        body_c = Body(CELL, DEFORMABLE, c, ca=1e-3, beta=0.0)
    else:
        c = biconcave(cell_markers, CELL_X_UM / dx, CELL_Y_UM / dx, CELL_RADIUS_UM / dx)
        body_c = Body(CELL, DEFORMABLE, c, ca=1e-3, beta=1e-2)
    a, b = 0.5 * PARTICLE_LENGTH_UM / dx, 0.5 * ar * PARTICLE_LENGTH_UM / dx
    part = ellipse(particle_markers, PARTICLE_X_UM / dx, PARTICLE_GAP_UM / dx + b, a, b)
    if ca == 0.0:
        body_p = Body(PARTICLE, RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1,
                      adhesion=_bond_defaults(ny, n_lig, 1.0))
    else:
        body_p = Body(PARTICLE, DEFORMABLE, part, ca=ca, beta=1e-2, density_ratio=1.1,
                      adhesion=_bond_defaults(ny, n_lig, 1.0))
    name = f"{nx}x{ny} {cell} cell, particle AR {ar} Ca {ca}, seed {seed}"
    return Capillary(name, nx, ny, 1.0, 1e-2, 200000, storage, seed, [body_c, body_p])


def sweep_capillaries(seed: int = 0, ny: int = 150, nx_range=(600, 1600), storage: str = "fp32") -> List[Capillary]:
    """The 64-capillary sweep: every combination of SWEEP_AR x SWEEP_CA x
    SWEEP_CELLS x SWEEP_SEEDS, channel lengths drawn uniformly from nx_range
    (inclusive) with numpy's default generator seeded by ``seed``."""
    rng = np.random.default_rng(seed)
    combos = list(itertools.product(SWEEP_AR, SWEEP_CA, SWEEP_CELLS, SWEEP_SEEDS))
    lengths = rng.integers(nx_range[0], nx_range[1] + 1, size=len(combos))
    return [sweep_capillary(int(n), ny, ar, ca, cell, s, storage)
            for n, (ar, ca, cell, s) in zip(lengths, combos)]


def scaled(cap: Capillary, nx: int, ny: int) -> Capillary:
    """The same bodies and parameters on a resized lattice (bodies kept in place)."""
    return dataclasses.replace(cap, nx=nx, ny=ny, name=f"{cap.name} on {nx}x{ny}")


def reduced_area(xy: np.ndarray) -> float:
    """4 pi A / P^2 (the swelling ratio quoted in Sec. 3.1)."""
    x, y = xy[:, 0], xy[:, 1]
    A = 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    P = np.sum(np.hypot(np.roll(x, -1) - x, np.roll(y, -1) - y))
    return 4.0 * math.pi * A / P**2


# Sec. 3.1 compares square particles with circular ones whose diameter equals
# the squares' thickness: d = 0.5, 1.0, 1.5 and 2.0 um
COMPARISON_D_UM = (0.5, 1.0, 1.5, 2.0)
LIGAND_DENSITY_PER_UM = 40.0  # ~ the 200 sites of the 2 x 1 um particle's 4.8 um perimeter


def particle_shape(shape: str, n: int, d_um: float, ny: int) -> np.ndarray:
    """A particle of thickness d_um resting on the lower wall at the release
    point of the particles of Sec. 3.1: a d x d square or a circle of diameter
    d, in lattice units of a channel ny nodes high."""
    dx = H_UM / ny
    d = d_um / dx
    cx, cy = PARTICLE_X_UM / dx, PARTICLE_GAP_UM / dx + 0.5 * d
    if shape == "square":
        return rectangle(n, cx, cy, d, d)
    if shape == "circle":
        return circle(n, cx, cy, 0.5 * d, phase=-0.5 * np.pi)
    raise ValueError("shape is 'square' or 'circle'")


def particle_comparison_capillary(shape: str, d_um: float, nx: int = 1200, ny: int = 150, ca: float = 0.0,
                                  seed: int = 0, storage: str = "fp32", markers: Optional[int] = None) -> Capillary:
    """The globular 7 um cell over a square or circular particle of thickness
    d_um adhering to the lower wall (sigma = 1), rigid when ca == 0, with
    ligand sites at LIGAND_DENSITY_PER_UM along the perimeter and (by default)
    one marker per lattice spacing of perimeter."""
    dx = H_UM / ny
    perim_um = (4.0 if shape == "square" else math.pi) * d_um
    if markers is None:
        markers = max(32, int(math.ceil(perim_um / dx)))
    part = particle_shape(shape, markers, d_um, ny)
    n_lig = max(4, int(round(LIGAND_DENSITY_PER_UM * perim_um)))
    cell = circle(256, CELL_X_UM / dx, CELL_Y_UM / dx, CELL_RADIUS_UM / dx)
    motion = RIGID if ca == 0.0 else DEFORMABLE
    bodies = [Body(CELL, DEFORMABLE, cell, ca=1e-3, beta=0.0),
              Body(PARTICLE, motion, part, ca=ca, beta=0.0 if ca == 0.0 else 1e-2, density_ratio=1.1,
                   adhesion=_bond_defaults(ny, n_lig, 1.0))]
    return Capillary(f"{nx}x{ny} globular cell, {shape} particle d = {d_um} um, Ca {ca}", nx, ny, 1.0, 1e-2,
                     200000, storage, seed, bodies)


def particle_comparison_capillaries(ca: float = 0.0, nx: int = 1200, ny: int = 150, seed: int = 0,
                                    storage: str = "fp32") -> List[Capillary]:
    """Square and circular particles of every COMPARISON_D_UM (8 capillaries)."""
    return [particle_comparison_capillary(s, d, nx, ny, ca, seed, storage)
            for s in ("square", "circle") for d in COMPARISON_D_UM]
