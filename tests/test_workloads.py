"""The seeded input recipes (paper_2512_06143_gb300/workloads.py) produce what they state: the
configured sizes, ranges and mean stored entries per row (library k-d tree counts, independent of
both the oracle and the CUDA path)."""
import math

import numpy as np
import pytest

scipy_spatial = pytest.importorskip("scipy.spatial")

from paper_2512_06143_gb300 import workloads as W  # noqa: E402


def _mean_entries(X, r, rows=4000, seed=0):
    tree = scipy_spatial.cKDTree(X)
    idx = np.random.default_rng(seed).choice(X.shape[0], size=min(rows, X.shape[0]), replace=False)
    # the pattern is d < r (strict) plus the diagonal; the k-d tree counts d <= r, and ties at
    # exactly r have probability zero for these continuous inputs
    return float(np.mean([len(v) for v in tree.query_ball_point(X[idx], r)]))


def test_clusters_3d_frozen_radius_gives_about_100_entries_per_row():
    w = W.clusters_3d(0)
    X = w["X"]
    assert X.shape == (1_000_000, 3) and X.min() >= 0.0 and X.max() <= 1.0
    assert w["hyper"]["r"] == W.FROZEN_R[("clusters_3d", 0)] and w["hyper"]["sigma2"] == 4e-4
    assert w["hyper"]["centers"].shape == (8, 3)
    assert _mean_entries(X, w["hyper"]["r"]) == pytest.approx(100.0, rel=0.05)


def test_sphere_4d_recipe_at_reduced_size():
    w = W.sphere_4d(0, n=200_000)
    X = w["X"]
    assert X.shape == (200_000, 4) and X.min() >= 0.0 and X.max() <= 1.0
    # latitude uniform on the sphere: sin(lat) = 2 u - 1 is uniform on [-1, 1]
    sinlat = np.sin(X[:, 1] * math.pi - math.pi / 2)
    assert abs(sinlat.mean()) < 0.01 and sinlat.var() == pytest.approx(1.0 / 3.0, rel=0.02)
    assert _mean_entries(X, w["hyper"]["r"]) == pytest.approx(60.0, rel=0.06)


def test_batch_recipe():
    ws = W.batch(0)
    assert len(ws) == 256
    ns = np.array([w["X"].shape[0] for w in ws])
    ds = np.array([w["hyper"]["d"] for w in ws])
    assert ns.min() >= 2048 and ns.max() <= 65536 and set(ds.tolist()) == {1, 2, 3}
    for w in ws[:8]:
        got = _mean_entries(w["X"], w["hyper"]["r"], rows=1000)
        assert got == pytest.approx(w["target_nnz"], rel=0.25)   # boundary effects at small n


def test_generators_are_seeded():
    a, b = W.clusters_3d(1, n=5000), W.clusters_3d(1, n=5000)
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["y"], b["y"])
    assert not np.array_equal(a["X"], W.clusters_3d(2, n=5000)["X"])
