"""Seeded synthetic workloads shaped like the paper's experiments (inputs only).

This module is the single place both the CUDA path's tests/benchmark and the CPU oracle get
their inputs from.  It generates point clouds X, observations y and kernel hyperparameters with
numpy's PCG64 generator; it contains none of the method's arithmetic (no kernel values, no
pattern decisions, no solves).  The one derived quantity, the Wendland support radius r tuned to
a target mean number of stored entries per row, is found with a library k-d tree neighbour
count on a row sample and frozen per (workload, seed) in ``FROZEN_R``.

Workloads (the datasets of the paper are not available; these stand in for them):
  * ``small_2d``   -- N = 4096, d = 2, X ~ U[0,1]^2, y = sin(6 x1) cos(4 x2) + N(0, 0.01^2),
                      L = 4 bumps (centers ~ U[0,1]^2, radii 0.4, amplitude 1, beta 1),
                      Wendland C2 with r = 0.05, sigma^2 = 1e-4: plain FP64, exact log-det.
  * ``clusters_3d``-- N = 1,000,000, d = 3, 50 Gaussian clusters (sigma 0.03, centers ~ U[0,1]^3)
                      clipped to [0,1]^3, y = sin(2 pi x1) + sin(4 pi x2 + 1) + sin(6 pi x3 + 2)
                      + N(0, 0.02^2), L = 8 bumps (radii 0.4), r tuned for ~100 entries per row,
                      sigma^2 = 4e-4 (the generic synthetic data of App. B.6, at N = 1e6).
  * ``batch``      -- 256 independent problems, N log-uniform in [2048, 65536], d in {1, 2, 3},
                      target entries per row log-uniform in [10, 200], X ~ U[0,1]^d, L = 4 bumps
                      (radii 0.4), y = the clusters_3d function on the first d coordinates,
                      sigma^2 = 1e-4.
  * ``sphere_4d``  -- N = 10,000,000, d = 4: (longitude/2pi, (latitude + pi/2)/pi, time, elevation)
                      with points uniform on the sphere, time ~ U[0,1] and elevation a smooth
                      16-mode random Fourier field of (lon, lat) scaled to [0,1]; L = 8 bumps
                      (radii 0.3), r tuned for ~60 entries per row, sigma^2 = 4e-4 (the shape of
                      the 10-million-point temperature run, Sec. 5.5 / App. B.5).
  * ``f1_1d``      -- the 1-D test function of Sec. 5.1, f1(x) = sin 5x + cos 20x
                      + 2 (x - 0.4)^2 cos 400x, on N uniform points in [0, 1].
"""
from __future__ import annotations

import math

import numpy as np

# r frozen per (workload, seed) by ``tune_r`` (bisection on a 10^4-row sample to the target
# mean entries per row, diagonal included, +-3%).
FROZEN_R = {
    ("clusters_3d", 0): 0.0105222,
    ("sphere_4d", 0): 0.0158314,
}


def _hyper(d, r, sigma2, centers, radii, amps, beta=1.0, w0=0.0, kind=0, family=0, ell=None, G=None):
    h = dict(d=int(d), r=float(r), sigma2=float(sigma2),
             centers=np.ascontiguousarray(centers, np.float64).reshape(-1, d),
             radii=np.ascontiguousarray(radii, np.float64),
             amps=np.ascontiguousarray(amps, np.float64), beta=float(beta), w0=float(w0),
             kind=int(kind))
    if family:
        h.update(family=int(family), ell=np.ascontiguousarray(ell, np.float64).reshape(d),
                 G=np.ascontiguousarray(G, np.float64).reshape(-1, d))
    return h


def tune_r(X: np.ndarray, target: float, seed: int = 0, sample: int = 10000,
           rel_tol: float = 0.03) -> float:
    """Radius whose mean neighbour count (the point itself included) on a row sample is within
    rel_tol of target.  Uses scipy's k-d tree (a library neighbour search)."""
    from scipy.spatial import cKDTree
    n, d = X.shape
    rng = np.random.default_rng(seed + 7919)
    idx = rng.choice(n, size=min(sample, n), replace=False)
    tree = cKDTree(X)
    q = X[idx]
    vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
    r = (target / (n * vol)) ** (1.0 / d)
    lo, hi = r * 0.05, r * 20.0
    for _ in range(60):
        cnt = tree.query_ball_point(q, r, return_length=True).mean()
        if abs(cnt - target) <= rel_tol * target * 0.5:
            break
        if cnt < target:
            lo = r
        else:
            hi = r
        r = 0.5 * (lo + hi)
    return float(f"{r:.6g}")


def small_2d(seed: int = 0, n: int = 4096) -> dict:
    rng = np.random.default_rng(seed)
    X = rng.random((n, 2))
    y = np.sin(6 * X[:, 0]) * np.cos(4 * X[:, 1]) + rng.normal(0.0, 0.01, n)
    L = 4
    hyp = _hyper(2, 0.05, 1e-4, rng.random((L, 2)), np.full(L, 0.4), np.ones(L))
    return dict(name="small_2d", X=X, y=y, hyper=hyp)


def _clusters(rng, n, d, k=50, sigma=0.03):
    cent = rng.random((k, d))
    lab = rng.integers(0, k, n)
    X = cent[lab] + rng.normal(0.0, sigma, (n, d))
    return np.clip(X, 0.0, 1.0)


def _sines(X, rng, noise):
    f = np.sin(2 * np.pi * X[:, 0])
    if X.shape[1] > 1:
        f = f + np.sin(4 * np.pi * X[:, 1] + 1.0)
    if X.shape[1] > 2:
        f = f + np.sin(6 * np.pi * X[:, 2] + 2.0)
    return f + rng.normal(0.0, noise, X.shape[0])


def clusters_3d(seed: int = 0, n: int = 1_000_000, target_nnz: float = 100.0,
                r: float | None = None) -> dict:
    rng = np.random.default_rng(seed)
    X = _clusters(rng, n, 3)
    y = _sines(X, rng, 0.02)
    L = 8
    centers = rng.random((L, 3))
    if r is None:
        r = FROZEN_R.get(("clusters_3d", seed)) if n == 1_000_000 and target_nnz == 100.0 else None
        if r is None:
            r = tune_r(X, target_nnz, seed)
    hyp = _hyper(3, r, 4e-4, centers, np.full(L, 0.4), np.ones(L))
    return dict(name="clusters_3d", X=X, y=y, hyper=hyp)


def _fourier_field(rng, lon, lat, modes=16):
    f = np.zeros_like(lon)
    for _ in range(modes):
        kx, ky = rng.integers(1, 6, 2)
        ph = rng.random(2) * 2 * np.pi
        amp = rng.normal() / (kx + ky)
        f += amp * np.sin(kx * lon + ph[0]) * np.cos(ky * lat + ph[1])
    f -= f.min()
    mx = f.max()
    return f / mx if mx > 0 else f


def sphere_4d(seed: int = 0, n: int = 10_000_000, target_nnz: float = 60.0,
              r: float | None = None) -> dict:
    rng = np.random.default_rng(seed)
    lon = rng.random(n) * 2 * np.pi
    lat = np.arcsin(rng.random(n) * 2.0 - 1.0)
    t = rng.random(n)
    fr = np.random.default_rng(seed + 1)
    e = _fourier_field(fr, lon, lat)
    X = np.stack([lon / (2 * np.pi), (lat + np.pi / 2) / np.pi, t, e], axis=1)
    y = (np.sin(2 * np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1]) + 0.5 * np.sin(2 * np.pi * X[:, 2])
         + 0.5 * X[:, 3] + rng.normal(0.0, 0.02, n))
    L = 8
    centers = rng.random((L, 4))
    if r is None:
        r = FROZEN_R.get(("sphere_4d", seed)) if n == 10_000_000 and target_nnz == 60.0 else None
        if r is None:
            r = tune_r(X, target_nnz, seed)
    hyp = _hyper(4, r, 4e-4, centers, np.full(L, 0.3), np.ones(L))
    return dict(name="sphere_4d", X=X, y=y, hyper=hyp)


def batch(seed: int = 0, count: int = 256, n_range=(2048, 65536), nnz_range=(10.0, 200.0)) -> list:
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = int(rng.integers(1, 4))
        target = math.exp(rng.uniform(math.log(nnz_range[0]), math.log(nnz_range[1])))
        X = rng.random((n, d))
        y = _sines(X, rng, 0.02)
        vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        r = (target / (n * vol)) ** (1.0 / d)
        L = 4
        hyp = _hyper(d, r, 1e-4, rng.random((L, d)), np.full(L, 0.4), np.ones(L))
        out.append(dict(name=f"batch[{b}]", X=X, y=y, hyper=hyp, target_nnz=target))
    return out


def f1(x):
    """Sec. 5.1's 1-D test function."""
    x = np.asarray(x, np.float64)
    return np.sin(5 * x) + np.cos(20 * x) + 2 * (x - 0.4) ** 2 * np.cos(400 * x)


def f1_1d(seed: int = 0, n: int = 2000, r: float = 0.02) -> dict:
    rng = np.random.default_rng(seed)
    X = np.sort(rng.random(n))[:, None]
    y = f1(X[:, 0]) + rng.normal(0.0, 0.01, n)
    L = 2
    hyp = _hyper(1, r, 1e-4, rng.random((L, 1)), np.full(L, 0.4), np.ones(L), w0=1.0)
    return dict(name="f1_1d", X=X, y=y, hyper=hyp)


def random_small(seed: int, n: int, d: int, L: int = 3, r: float | None = None, kind: int = 0,
                 w0: float = 0.0, sigma2: float = 1e-3, clustered: bool = False) -> dict:
    """Small random problems for parity tests (any d in 1..4)."""
    rng = np.random.default_rng(seed)
    X = _clusters(rng, n, d, k=max(1, n // 200), sigma=0.05) if clustered else rng.random((n, d))
    y = _sines(X, rng, 0.02)
    if r is None:
        vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        r = (30.0 / (n * vol)) ** (1.0 / d)
    hyp = _hyper(d, r, sigma2, rng.random((L, d)), rng.uniform(0.3, 0.6, L), rng.uniform(0.5, 1.5, L),
                 w0=w0, kind=kind)
    return dict(name=f"random_small[{seed}]", X=X, y=y, hyper=hyp)


def random_wendconv(seed: int, n: int, d: int, L: int = 3, r: float | None = None, kind: int = 0,
                    sigma2: float = 1e-3, clustered: bool = False, stationary: bool = False) -> dict:
    """Problems for the Wendland convolution kernel (Eq. 6): the length-scale field's base
    factors ell ~ U(0.7, 1.4)^d and bump weights G ~ U(0, 1.5)^(L x d), the signal field
    w0 = 1 plus amplitudes U(0.2, 1) on bumps of radius U(0.3, 0.6).  stationary=True sets
    G = 0, ell = 1, amplitudes 0 (the kernel is then Eq. 3's plain taper)."""
    rng = np.random.default_rng(seed)
    X = _clusters(rng, n, d, k=max(1, n // 200), sigma=0.05) if clustered else rng.random((n, d))
    y = _sines(X, rng, 0.02)
    if r is None:
        vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        r = (30.0 / (n * vol)) ** (1.0 / d)
    centers, radii = rng.random((L, d)), rng.uniform(0.3, 0.6, L)
    ell, G, amps = rng.uniform(0.7, 1.4, d), rng.uniform(0.0, 1.5, (L, d)), rng.uniform(0.2, 1.0, L)
    if stationary:
        ell, G, amps = np.ones(d), np.zeros((L, d)), np.zeros(L)
    hyp = _hyper(d, r, sigma2, centers, radii, amps, w0=1.0, kind=kind, family=1, ell=ell, G=G)
    return dict(name=f"random_wendconv[{seed}]", X=X, y=y, hyper=hyp)


def random_farfield(seed: int, n: int, d: int, L: int = 4, r: float | None = None, radius: float = 0.12,
                    lc: float = 0.3, w0: float = 1.0, sigma2: float = 1e-3) -> dict:
    """Problems for the far-field kernel (Sec. 4.5): a local Wendland term of amplitude w0 plus the
    bumps' far-field term on a squared-exponential core of length lc; small bumps (radius
    `radius`, centers U[0,1]^d, amplitudes U(0.5, 1.5)) keep the far-field blocks sparse."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = _sines(X, rng, 0.02)
    if r is None:
        vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        r = (30.0 / (n * vol)) ** (1.0 / d)
    hyp = _hyper(d, r, sigma2, rng.random((L, d)), np.full(L, radius), rng.uniform(0.5, 1.5, L), w0=w0)
    hyp.update(family=2, ell=np.array([lc]), G=np.zeros((L, d)))
    return dict(name=f"random_farfield[{seed}]", X=X, y=y, hyper=hyp)


def f1_1d_wendconv(seed: int = 0, n: int = 2000, r: float = 0.02) -> dict:
    """Sec. 5.1's 1-D test with the Wendland convolution kernel (the paper's choice for it)."""
    rng = np.random.default_rng(seed)
    X = np.sort(rng.random(n))[:, None]
    y = f1(X[:, 0]) + rng.normal(0.0, 0.01, n)
    L = 3
    hyp = _hyper(1, r, 1e-4, rng.random((L, 1)), np.full(L, 0.3), rng.uniform(0.2, 0.8, L), w0=1.0,
                 family=1, ell=np.ones(1), G=rng.uniform(0.0, 2.0, (L, 1)))
    return dict(name="f1_1d_wendconv", X=X, y=y, hyper=hyp)


def perturbed_hypers(hyper: dict, count: int, seed: int) -> list:
    """`count` hyperparameter sets drawn around `hyper` (inputs for gradient checks at random
    theta): centers shifted by U(-0.1, 0.1) per coordinate, bump radii and amplitudes scaled by
    log-uniform factors in [0.8, 1.25] and [0.5, 2], r by [0.9, 1.1] and sigma^2 by [0.5, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    L, d = np.asarray(hyper["radii"]).shape[0], hyper["d"]

    def lu(lo, hi, size=None):
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size))

    for _ in range(count):
        out.append(_hyper(d, hyper["r"] * lu(0.9, 1.1), hyper["sigma2"] * lu(0.5, 2.0),
                          np.asarray(hyper["centers"]) + rng.uniform(-0.1, 0.1, (L, d)),
                          np.asarray(hyper["radii"]) * lu(0.8, 1.25, L),
                          np.asarray(hyper["amps"]) * lu(0.5, 2.0, L),
                          beta=hyper["beta"], w0=hyper["w0"], kind=hyper["kind"]))
    return out


def checksums(X: np.ndarray, y: np.ndarray) -> list:
    """Order-sensitive sums of the inputs, to confirm that another machine's generator produced
    the same X and y (up to the last-bit differences of its math library)."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    wgt = np.linspace(1.0, 2.0, X.shape[0])
    return [float(v) for v in np.concatenate([X.sum(0), (X * wgt[:, None]).sum(0), [y.sum(), (y * wgt).sum()]])]
