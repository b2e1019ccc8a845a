"""Pins of the oracle's far-field kernel (Sec. 4.5, family 2): w0 phi(|D|/r) + kappa(|D|) sum_l
b_l(xi) b_l(xj) with a squared-exponential core kappa.  Zero amplitudes reduce it to the plain
taper bit for bit; pairs sharing a bump are stored at any distance; the two-point closed form;
symmetry and positive semi-definiteness; the exact gradient against finite differences."""
import math

import numpy as np
import pytest

from paper_2512_06143_gb300 import workloads as W


def test_zero_amplitudes_reduce_to_the_plain_taper(orc):
    w = W.random_farfield(1000, 500, 2)
    h2 = orc.Hyper(**{**w["hyper"], "amps": np.zeros(4)})
    h0 = orc.Hyper(d=2, r=h2.r, sigma2=h2.sigma2, centers=np.zeros((0, 2)), radii=np.zeros(0), amps=np.zeros(0),
                   w0=h2.w0)
    assert np.array_equal(orc.dense_A(w["X"], h2), orc.dense_A(w["X"], h0))


def test_pairs_sharing_a_bump_are_stored_at_any_distance(orc):
    X = np.array([[0.1, 0.1], [0.12, 0.1], [0.9, 0.9], [0.1, 0.35], [0.5, 0.5]])
    h = orc.Hyper(d=2, r=0.05, sigma2=0.0, centers=np.array([[0.1, 0.22]]), radii=np.array([0.2]),
                  amps=np.array([1.3]), w0=0.7, family=2, ell=np.array([0.25]))
    c = orc.assemble(X, h, "brute")
    rows = {i: set(c.col[c.rowptr[i]:c.rowptr[i + 1]].tolist()) for i in range(5)}
    # points 0, 1 and 3 lie inside the bump; 0-1 are also within r; 2 and 4 are outside
    assert rows[0] == {0, 1, 3} and rows[3] == {0, 1, 3} and rows[2] == {2} and rows[4] == {4}
    b = orc.bumps(h, X[0])[0], orc.bumps(h, X[3])[0]
    q = float(np.sum((X[0] - X[3]) ** 2))
    K = orc.dense_A(X, h)
    assert K[0, 3] == pytest.approx(math.exp(-q / (2 * 0.25 ** 2)) * b[0] * b[1], rel=1e-14)
    t = 0.02 / 0.05
    b0, b1 = orc.bumps(h, X[0])[0], orc.bumps(h, X[1])[0]
    expect = 0.7 * (1 - t) ** 4 * (4 * t + 1) + math.exp(-0.02 ** 2 / (2 * 0.25 ** 2)) * b0 * b1
    assert K[0, 1] == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_symmetric_and_psd(orc, d):
    w = W.random_farfield(1010 + d, 400, d, radius={1: 0.05, 2: 0.15, 3: 0.25}[d])
    K = orc.dense_A(w["X"], orc.Hyper(**{**w["hyper"], "sigma2": 0.0}))
    assert np.array_equal(K, K.T)
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-10 * ev.max()


def test_exact_gradient_matches_finite_differences(orc):
    w = W.random_farfield(1020, 220, 2, L=3, radius=0.2, sigma2=5e-3, r=0.1)
    h = orc.Hyper(**w["hyper"])
    g = orc.grad_exact(w["X"], w["y"], h)
    fd = orc.lml_fd_grad(w["X"], w["y"], h, step=1e-5)
    assert g.shape == (h.nparams,) == (3 * 4 + 4,)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max() + 1e-9
