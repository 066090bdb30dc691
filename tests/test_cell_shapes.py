"""Host-side helpers of the generated cell shapes (paper_2210_06043_gb300/
cell_shapes.py): rescaling between lattice resolutions keeps the shape (its
reduced area and its aspect ratio), the area scales with the square of the
resolution, and the result is counter-clockwise about its area centroid."""
import math

import numpy as np

from paper_2210_06043_gb300 import cell_shapes as cs
from paper_2210_06043_gb300 import workloads as wl


def _area(xy):
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def test_rescale_keeps_the_shape():
    src = wl.biconcave(64, 3.0, -2.0, 14.0)  # a 30-node channel's biconcave cell, off centre
    out = cs.rescale(src, 30, 150, n=256)
    assert out.shape == (256, 2)
    assert _area(out) > 0  # counter-clockwise
    c, a = cs._centroid(out)
    assert np.abs(c).max() < 1e-9
    assert math.isclose(a, _area(src) * 25.0, rel_tol=2e-3)
    assert math.isclose(wl.reduced_area(out), wl.reduced_area(src), rel_tol=2e-3)
    ext = lambda p: (p[:, 0].max() - p[:, 0].min()) / (p[:, 1].max() - p[:, 1].min())
    assert math.isclose(ext(out), ext(src), rel_tol=1e-2)
    seg = np.hypot(*np.diff(np.vstack([out, out[:1]]), axis=0).T)
    assert seg.max() / seg.min() < 1.01  # equally spaced in arc length
