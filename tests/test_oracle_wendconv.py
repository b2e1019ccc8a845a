"""Pins of the oracle's Wendland convolution kernel (Eq. 6, Sec. 4.2, family 1): the stationary
reduction to Eq. 3 (bit for bit), the constant anisotropic case in closed form, symmetry and
positive semi-definiteness with non-constant fields (Paciorek's construction), the prefactor bound
and the support rule, and the exact gradient against central finite differences of the LML."""
import math

import numpy as np
import pytest

from paper_2512_06143_gb300 import workloads as W


def test_stationary_fields_reduce_to_the_plain_taper_bit_for_bit(orc):
    for d in (1, 2, 3):
        w = W.random_wendconv(900 + d, 400, d, stationary=True)
        h1 = orc.Hyper(**w["hyper"])
        h0 = orc.Hyper(d=d, r=h1.r, sigma2=h1.sigma2, centers=np.zeros((0, d)), radii=np.zeros(0),
                       amps=np.zeros(0), w0=1.0)
        A1, A0 = orc.dense_A(w["X"], h1), orc.dense_A(w["X"], h0)
        assert np.array_equal(A1, A0)
        c1, c0 = orc.assemble(w["X"], h1, "brute"), orc.assemble(w["X"], h0, "brute")
        assert np.array_equal(c1.col, c0.col) and np.array_equal(c1.rowptr, c0.rowptr)


def test_constant_anisotropic_length_scales_closed_form(orc):
    rng = np.random.default_rng(5)
    X = rng.random((250, 3))
    ell = np.array([0.6, 1.3, 2.0])
    r = 0.2
    h = orc.Hyper(d=3, r=r, sigma2=0.0, centers=rng.random((2, 3)), radii=np.array([0.4, 0.5]),
                  amps=np.zeros(2), w0=1.0, family=1, ell=ell, G=np.zeros((2, 3)))
    K = orc.dense_A(X, h)
    D = X[:, None, :] - X[None, :, :]
    t = np.sqrt(np.sum(D * D / (ell * ell), axis=2)) / r
    expect = np.where(t < 1.0, (1 - t) ** 4 * (4 * t + 1), 0.0)
    np.testing.assert_allclose(K, expect, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d,kind", [(1, 0), (2, 0), (3, 1), (4, 0)])
def test_symmetric_psd_prefactor_and_support(orc, d, kind):
    w = W.random_wendconv(910 + d, 350, d, kind=kind, r={1: 0.05, 2: 0.15, 3: 0.3, 4: 0.45}[d])
    h = orc.Hyper(**{**w["hyper"], "sigma2": 0.0})
    K = orc.dense_A(w["X"], h)
    assert np.array_equal(K, K.T)
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-10 * ev.max()
    pv = orc.point_values(w["X"], h)
    s, lam = pv[:, 0], pv[:, 1:]
    X = w["X"]
    for i in range(0, 350, 17):
        for j in range(0, 350, 5):
            q = orc.lib().orc_wc_q(d, X[i].ctypes.data, X[j].ctypes.data, lam[i].ctypes.data, lam[j].ctypes.data)
            if i != j and q >= h.r * h.r:
                assert K[i, j] == 0.0
            else:
                # |S_i|^(1/4) |S_j|^(1/4) / |(S_i + S_j)/2|^(1/2) <= 1 (arithmetic-geometric mean)
                phi = orc.phi(h.kind, d, math.sqrt(q) / h.r)
                assert abs(K[i, j]) <= abs(s[i] * s[j]) * phi * (1 + 1e-14) + 1e-300
    np.testing.assert_allclose(np.diag(K), s * s, rtol=1e-15)


@pytest.mark.parametrize("d", [1, 2])
def test_exact_gradient_matches_finite_differences(orc, d):
    w = W.random_wendconv(920 + d, 220, d, L=2, sigma2=5e-3, r={1: 0.04, 2: 0.2}[d])
    h = orc.Hyper(**w["hyper"])
    g = orc.grad_exact(w["X"], w["y"], h)
    fd = orc.lml_fd_grad(w["X"], w["y"], h, step=1e-5)
    assert g.shape == (h.nparams,) == (2 * (2 * d + 2) + d + 3,)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max() + 1e-9
