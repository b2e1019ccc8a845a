"""Pins of the oracle's posterior (Eq. 2, Sec. 3) against facts that do not use its formula:
closed-form identities at the training points, the joint-Gaussian conditional taken from a dense
assembly of training and test points together (library solve), the single-point closed form, a
test point outside every support, and the bounds 0 <= var <= k(x*, x*)."""
import numpy as np
import pytest

from paper_2512_06143_gb300 import workloads as W


def _problem(orc, seed, n=300, d=2, w0=0.0, kind=0):
    w = W.random_small(seed, n, d, L=3, sigma2=2e-3, w0=w0, kind=kind, r={1: 0.05, 2: 0.2, 3: 0.3}[d])
    return w, orc.Hyper(**w["hyper"])


@pytest.mark.parametrize("d,w0,kind", [(1, 0.0, 0), (2, 0.0, 0), (3, 0.5, 1)])
def test_posterior_at_training_points_closed_forms(orc, d, w0, kind):
    # K A^{-1} y = (A - s2 I) A^{-1} y = y - s2 a, and
    # diag(K A^{-1} K) = diag(A - 2 s2 I + s2^2 A^{-1})  =>  var_i = s2 - s2^2 (A^{-1})_ii
    w, h = _problem(orc, 500 + d, d=d, w0=w0, kind=kind)
    p = orc.posterior(w["X"], w["y"], h, w["X"])
    s2 = h.sigma2
    np.testing.assert_allclose(p["mean"], w["y"] - s2 * p["a"], rtol=0, atol=1e-10 * np.abs(w["y"]).max())
    Ainv = np.linalg.inv(p["A"])
    np.testing.assert_allclose(p["var"], s2 - s2 * s2 * np.diag(Ainv), rtol=0, atol=1e-11)


def test_posterior_is_the_joint_gaussian_conditional(orc):
    w, h = _problem(orc, 510, n=250, d=2)
    rng = np.random.default_rng(9)
    Xs = rng.random((60, 2))
    p = orc.posterior(w["X"], w["y"], h, Xs)
    n = w["X"].shape[0]
    J = orc.dense_A(np.vstack([w["X"], Xs]), h)       # K of the union + s2 on every diagonal
    Att, Ast = J[:n, :n], J[n:, :n]
    Kss = J[n:, n:] - h.sigma2 * np.eye(Xs.shape[0])
    mean = Ast @ np.linalg.solve(Att, w["y"])
    var = np.diag(Kss) - np.einsum("ij,ji->i", Ast, np.linalg.solve(Att, Ast.T))
    np.testing.assert_allclose(p["mean"], mean, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(p["var"], var, rtol=1e-9, atol=1e-12)
    assert np.all(p["var"] >= -1e-12) and np.all(p["var"] <= orc.prior_var(Xs, h) + 1e-12)


def test_posterior_single_training_point(orc):
    h = orc.Hyper(d=2, r=0.5, sigma2=0.1, centers=np.array([[0.5, 0.5]]), radii=np.array([2.0]),
                  amps=np.array([1.3]), beta=1.0)
    X = np.array([[0.4, 0.45]])
    y = np.array([0.7])
    Xs = np.array([[0.5, 0.6], [0.41, 0.45], [3.0, 3.0]])
    p = orc.posterior(X, y, h, Xs)
    k11 = orc.kernel(h, X[0], X[0])
    for i, xs in enumerate(Xs):
        ks = orc.kernel(h, xs, X[0]) if np.sum((xs - X[0]) ** 2) < h.r ** 2 else 0.0
        kss = orc.kernel(h, xs, xs)
        assert p["mean"][i] == pytest.approx(ks * y[0] / (k11 + h.sigma2), rel=1e-13, abs=1e-15)
        assert p["var"][i] == pytest.approx(kss - ks * ks / (k11 + h.sigma2), rel=1e-13, abs=1e-15)


def test_posterior_outside_every_support(orc):
    w, h = _problem(orc, 520, n=200, d=2, w0=0.25)
    Xs = np.array([[5.0, 5.0], [-3.0, 0.5]])
    p = orc.posterior(w["X"], w["y"], h, Xs)
    assert np.all(p["mean"] == 0.0)
    # phi(0) = 1 and the bumps vanish far away: k(x*, x*) = sum_l b_l(x*)^2 + w0 = w0
    np.testing.assert_allclose(p["var"], 0.25, rtol=1e-15)
    b = orc.bumps(h, w["X"][0])
    assert orc.prior_var(w["X"][:1], h)[0] == pytest.approx(float(np.sum(b * b)) + 0.25, rel=1e-14)


# ------------------------------------------------------------------------------------------------
# MINRES (the paper's solver, App. B.6) pins: the library's dense solve, an indefinite system
# (what CG cannot do), the residual-norm recurrence against the true residual, the minimal-residual
# property against CG's iterates, and exactness on an operator with few distinct eigenvalues.
# ------------------------------------------------------------------------------------------------
def test_minres_solves_spd_and_indefinite_systems(orc):
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(60, 60)))
    for ev in (np.linspace(0.1, 10.0, 60), np.concatenate([-np.linspace(0.5, 3.0, 20), np.linspace(0.2, 5.0, 40)])):
        M = (Q * ev) @ Q.T
        b = rng.normal(size=60)
        x, it, hist = orc.minres(lambda v: M @ v, b, tol=1e-12, maxit=500)
        np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-9, atol=1e-10)
        assert hist[-1] <= 1e-12 * np.linalg.norm(b) * 1.0001


def test_minres_residual_recurrence_and_minimality(orc):
    w = W.random_small(530, 400, 2, L=2, sigma2=1e-2, r=0.12)
    h = orc.Hyper(**w["hyper"])
    A = orc.dense_A(w["X"], h)
    b = w["y"]
    for k in (1, 2, 5, 12, 30):
        x, it, hist = orc.minres(lambda v: A @ v, b, tol=0.0, maxit=k)
        assert it == k
        true = np.linalg.norm(b - A @ x)
        assert abs(true - hist[-1]) <= 1e-9 * np.linalg.norm(b)
        # minimal residual over the Krylov space: no larger than CG's residual after k steps
        xc, _, _, _, _ = orc.cg(orc.CSR(400, *_dense_csr(A)), b, tol=0.0, maxit=k)
        assert true <= np.linalg.norm(b - A @ xc) * (1 + 1e-9)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_minres_exact_with_few_distinct_eigenvalues(orc):
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(50, 50)))
    M = (Q * np.repeat([0.5, 2.0, -1.0], [20, 20, 10])) @ Q.T
    b = rng.normal(size=50)
    x, it, hist = orc.minres(lambda v: M @ v, b, tol=1e-13, maxit=50)
    assert it <= 3 + 1
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-11)


def _dense_csr(A):
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), A[rows, cols].astype(np.float64)
