"""Host logic of the surrogate's inputs and statistics (surrogate.py), on CPU:

* ``initial_bonds`` (N0, the normalisation of N_L, from an interpolated table of
  particle polygons and a candidate-site shortcut) equals the count obtained
  site by site on the exact polygon ``capillary_for`` builds, under the
  adhesion rule include/lbib.h states (n sites at arc lengths (k + 1/2) P / n
  along the chain; bonded at t = 0 when the gap to the nearer wall is below
  y_cr).  The GPU test checks the same count against the library itself.
* ``seed_statistics`` against its definition on a synthetic set with known
  spread, and ``replicate``'s seeds."""
import math

import numpy as np
import pytest

from paper_2210_06043_gb300 import surrogate as sg


def _n0_site_by_site(p):
    body = sg.capillary_for(p).bodies[1]
    xy = np.asarray(body.xy, np.float64)
    n, y_cr = body.adhesion.n_lig, body.adhesion.y_cr
    closed = np.vstack([xy, xy[:1]])
    cum = np.concatenate([[0.0], np.cumsum(np.hypot(*np.diff(closed, axis=0).T))])
    count = 0
    for k in range(n):
        s = (k + 0.5) * cum[-1] / n
        l = 0
        while l < len(xy) - 1 and s > cum[l + 1]:
            l += 1
        t = min(1.0, max(0.0, (s - cum[l]) / (cum[l + 1] - cum[l])))
        py = closed[l, 1] + t * (closed[l + 1, 1] - closed[l, 1])
        count += min(py, sg.NY - py) < y_cr
    return count


def test_initial_bonds_equal_the_site_by_site_count():
    pts = sg.sample_points(160, seed=21)
    # the ends of the aspect-ratio range and one point outside it (exact construction)
    pts += [sg.Point(sg.AR_RANGE[0], -3.5, False, "globular", 10.0), sg.Point(sg.AR_RANGE[1], -3.5, True, "biconcave",
                                                                             50.0),
            sg.Point(1.2, -3.5, True, "globular", 30.0)]
    got = sg.initial_bonds(pts)
    want = np.array([_n0_site_by_site(p) for p in pts])
    assert np.array_equal(got, want), np.flatnonzero(got != want)
    assert got.min() >= 1 and len(np.unique(got)) > 5  # a step function with many levels
    assert sg.initial_bonds([]).shape == (0,)


def test_features_rows():
    pts = sg.sample_points(3, seed=2)
    t = np.array([0.1, 0.5])
    X = sg.features_many(pts, t)
    assert X.shape == (6, len(sg.FEATURES))
    n0 = sg.initial_bonds(pts)
    assert np.array_equal(X[::2, sg.FEATURES.index("initial_bonds")], n0.astype(np.float32))
    assert np.allclose(X[:, sg.FEATURES.index("inverse_initial_bonds")], np.repeat(1.0 / n0, 2))
    assert np.allclose(X[:, -1], np.tile(t, 3))
    assert np.array_equal(sg.features(pts[1], t), X[2:4])


def test_seed_statistics_and_replicates():
    rng = np.random.default_rng(0)
    n, R, T = 50, 4, 30
    mean = rng.normal(size=(n, 1, T, 3))
    sd = np.array([0.5, 2.0, 0.1])
    Y = (mean + sd * rng.normal(size=(n, R, T, 3))).reshape(n * R, T, 3)
    m, spread, floor = sg.seed_statistics(Y, R)
    assert np.allclose(m, Y.reshape(n, R, T, 3).mean(1))
    assert np.allclose(spread, sd, rtol=0.1)  # 4500 samples per output
    assert np.allclose(floor, spread / math.sqrt(R))
    with pytest.raises(ValueError):
        sg.seed_statistics(Y, 1)
    pts = sg.sample_points(2, seed=3)
    reps = sg.replicate(pts, 3)
    assert [r.seed for r in reps] == [pts[0].seed * 3 + j for j in range(3)] + [pts[1].seed * 3 + j for j in range(3)]
    assert all(r.aspect_ratio == pts[i // 3].aspect_ratio for i, r in enumerate(reps))
