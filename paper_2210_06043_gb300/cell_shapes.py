"""Bullet- and parachute-shaped cells (Sec. 3.1): the shapes that the
circular and the biconcave cell settle into in the capillary's plane
Poiseuille flow.  The paper transports these deformed shapes with the circular
and biconcave shapes as their stress-free configurations, so they are
generated here by the solver itself: the cell alone, released on the centre
line, is advanced until its shape (seen from its centroid) stops changing.

The channel is finite, so a long run is relayed: when the cell nears the
outlet, the current shape is placed back near the inlet in a fresh channel
(undisturbed inflow, same stress-free shape) and the run continues.  At the
low Reynolds numbers of the paper the flow around the cell re-forms within a
viscous time, so the relay does not change the shape the run converges to.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import lbib
from . import workloads as wl


def _centroid(xy: np.ndarray):
    x, y = xy[:, 0], xy[:, 1]
    c = x * np.roll(y, -1) - np.roll(x, -1) * y
    a = 0.5 * c.sum()
    return np.array([((x + np.roll(x, -1)) * c).sum() / (6 * a), ((y + np.roll(y, -1)) * c).sum() / (6 * a)]), a


@dataclasses.dataclass
class SteadyShape:
    xy: np.ndarray      # vertices about the area centroid, lattice units of the run
    steps: int          # solver steps taken
    converged: bool     # the last check moved no vertex by more than tol * R
    change: float       # that last move / R (R = radius of the reference's area)
    relays: int         # times the cell was placed back near the inlet


def steady_shape(ref_xy: np.ndarray, ny: int, ca: float = 1e-3, beta: float = 0.0, re: float = 0.2,
                 nx: Optional[int] = None, storage: int = lbib.LBIB_STORE_FP32, check_tstar: float = 0.05,
                 tol: float = 2e-3, max_tstar: float = 20.0, device: int = 0, stream=None,
                 transfer: int = lbib.LBIB_TRANSFER_PESKIN) -> SteadyShape:
    """Runs a deformable cell with stress-free shape ref_xy (counter-clockwise,
    lattice units of a channel ny nodes high, any position) alone in the
    inlet/outlet capillary at Reynolds number re (tau = 1) until no vertex
    moves by more than tol * R relative to the centroid between two checks
    check_tstar apart in t u_max / H (or until max_tstar).  The shape depends
    on Ca and the confinement, not on re, while re stays small (Stokes
    regime); a larger re only takes fewer steps.  Returns the shape about its
    area centroid."""
    ref = np.asarray(ref_xy, np.float64)
    c0, a0 = _centroid(ref)
    ref = ref - c0
    R = math.sqrt(abs(a0) / math.pi)
    nx = int(nx or 8 * ny)
    steps_per_t = ny * ny * 6.0 / re  # H / u_max with u_max = re nu / H, nu = 1/6
    check_every = max(1, int(round(check_tstar * steps_per_t)))
    max_steps = int(max_tstar * steps_per_t)
    start = np.array([1.5 * ny, 0.5 * ny])
    shape = ref.copy()
    steps = relays = 0
    prev = None
    change = float("inf")
    while steps < max_steps:
        cap = wl.Capillary("steady cell shape", nx, ny, 1.0, re, max_steps, "fp64", 0,
                           [wl.Body(wl.CELL, wl.DEFORMABLE, shape + start, ca=ca, beta=beta, xy_ref=ref + start)],
                           transfer=transfer)
        s = lbib.from_capillary(cap, storage=storage, device=device, stream=stream)
        try:
            while steps < max_steps:
                s.advance(check_every)
                steps += check_every
                m = s.markers(0)
                c, _ = _centroid(m)
                shape = m - c
                if prev is not None:
                    change = float(np.abs(shape - prev).max()) / R
                    if change < tol:
                        return SteadyShape(shape, steps, True, change, relays)
                prev = shape
                if c[0] > nx - 1.5 * ny:
                    relays += 1
                    break
        finally:
            s.close()
    return SteadyShape(shape, steps, False, change, relays)


def bullet_cell(n: int, ny: int, **kw) -> SteadyShape:
    """The steady shape of the circular 7 um cell (Sec. 3.1) in a channel ny
    nodes high, n vertices."""
    dx = wl.H_UM / ny
    return steady_shape(wl.circle(n, 0.0, 0.0, wl.CELL_RADIUS_UM / dx), ny, **kw)


def parachute_cell(n: int, ny: int, **kw) -> SteadyShape:
    """The steady shape of the biconcave cell of Eq. 20 (Sec. 3.1)."""
    dx = wl.H_UM / ny
    kw.setdefault("beta", 1e-2)
    return steady_shape(wl.biconcave(n, 0.0, 0.0, wl.CELL_RADIUS_UM / dx), ny, **kw)


def rescale(xy: np.ndarray, from_ny: int, to_ny: int, n: Optional[int] = None) -> np.ndarray:
    """A shape generated in a channel from_ny nodes high, in lattice units of a
    channel to_ny nodes high (same physical size: coordinates scale by
    to_ny / from_ny), resampled to n vertices equally spaced in arc length
    (n = the input's count by default), counter-clockwise, about its area
    centroid.  Lets a shape generated on a coarse lattice serve a fine one."""
    xy = np.asarray(xy, np.float64) * (float(to_ny) / float(from_ny))
    n = int(n or len(xy))
    dense = wl._resample_closed(xy, max(20000, 8 * n))
    out = wl._ccw(wl._resample_closed(dense, n))
    c, _ = _centroid(out)
    return out - c
