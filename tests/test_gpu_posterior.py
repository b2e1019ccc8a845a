"""Posterior mean and latent variance (Eq. 2, Sec. 3) through the C ABI (gp2s_posterior) against
the oracle's dense posterior: test points inside, on and outside the training cloud, all d, both
Wendland kinds, FP64 and mixed precision.

Bars: mean within 1e-8 of max |mean| (the cross-covariance in FP64; the y solve refined to
tol_refine = 1e-12, since a solve stopped at a relative residual tol leaves up to
tol |y| / sigma^2 in a = A^{-1} y, which at the default 1e-8 can reach the bar); variance within
1e-6 k(x*, x*) (the solve in the problem's vector precision to tol_probe = 1e-7, its energy form
second order in the solution error)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_06143_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06143_gb300 as gp
    from paper_2512_06143_gb300 import build
    build.build()
    gp.load()
    return gp


def _test_points(rng, X, ns):
    d = X.shape[1]
    inside = rng.random((ns // 2, d))
    on = X[rng.choice(X.shape[0], ns // 4, replace=False)]
    outside = rng.random((ns - ns // 2 - ns // 4, d)) * 3.0 - 1.0
    return np.vstack([inside, on, outside])


@pytest.mark.parametrize("d,kind,w0,precision", [(1, 0, 0.0, "mixed"), (2, 0, 0.0, "mixed"), (3, 1, 0.5, "mixed"),
                                                 (4, 0, 0.0, "mixed"), (2, 0, 0.3, "fp64"), (3, 0, 0.0, "fp64")])
def test_posterior_matches_oracle(gp, d, kind, w0, precision):
    import oracle
    w = W.random_small(600 + d, 3000, d, L=3, sigma2=1e-3, kind=kind, w0=w0, clustered=(d == 3))
    h = gp.Hyper(**w["hyper"])
    prec = gp.PREC_MIXED if precision == "mixed" else gp.PREC_FP64
    opts = gp.default_opts(precision=prec, logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=30, tol_probe=1e-7,
                           tol_refine=1e-12)
    ctx = gp.Context(0)
    ctx.lml(torch.tensor(w["X"], device="cuda"), torch.tensor(w["y"], device="cuda"), h, opts)
    Xs = _test_points(np.random.default_rng(d), w["X"], 150)
    mean, var, info = ctx.posterior(torch.tensor(Xs, device="cuda"))
    p = oracle.posterior(w["X"], w["y"], oracle.Hyper(**w["hyper"]), Xs)
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    # pairs inside the support (explicit zeros included: outside every bump with w0 = 0 the kernel
    # value is 0 inside the support), with d2 summed left to right in FP64 as the pattern test does
    d2 = np.zeros((len(Xs), w["X"].shape[0]))
    for k in range(d):
        dk = Xs[:, k][:, None] - w["X"][:, k][None, :]
        d2 = d2 + dk * dk
    assert info["n_test"] == len(Xs) and info["cross_entries"] == int(np.count_nonzero(d2 < h.r * h.r))
    assert np.abs(mean - p["mean"]).max() <= 1e-8 * np.abs(p["mean"]).max()
    kss = oracle.prior_var(Xs, oracle.Hyper(**w["hyper"]))
    assert np.all(np.abs(var - p["var"]) <= 1e-6 * kss + 1e-12)
    # outside the cloud: no neighbours, mean 0 and the prior variance exactly
    far = np.all((Xs < -0.3) | (Xs > 1.3), axis=1)
    assert np.all(mean[far] == 0.0) and np.allclose(var[far], kss[far], rtol=1e-14)


def test_posterior_host_buffers_mean_only_and_errors(gp):
    import oracle
    w = W.small_2d(0)
    h = gp.Hyper(**w["hyper"])
    ctx = gp.Context(0)
    with pytest.raises(gp.GP2SError) as e:
        ctx.posterior(np.zeros((3, 2)))
    assert e.value.status == gp.ENOTREADY
    ctx.lml(w["X"], w["y"], h, gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_EXACT))
    Xs = np.random.default_rng(1).random((700, 2))
    mean, var, info = ctx.posterior(Xs, variance=False)
    assert var is None and info["batches"] == 0
    p = oracle.posterior(w["X"], w["y"], oracle.Hyper(**w["hyper"]), Xs)
    assert np.abs(mean - p["mean"]).max() <= 1e-8 * np.abs(p["mean"]).max()
    m0, v0, i0 = ctx.posterior(np.zeros((0, 2)))
    assert m0.shape == (0,) and i0["n_test"] == 0


# ------------------------------------------------------------------------------------------------
# MINRES (opts.solver = SOLVER_MINRES, App. B.6's solver) for the y column
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_minres_solve_matches_oracle(gp, precision):
    import oracle
    w = W.random_small(620, 5000, 2, L=3, sigma2=1e-3)
    h = gp.Hyper(**w["hyper"])
    prec = gp.PREC_MIXED if precision == "mixed" else gp.PREC_FP64
    ctx = gp.Context(0)
    opts = gp.default_opts(precision=prec, solver=gp.SOLVER_MINRES, logdet=gp.LOGDET_EXACT)
    ctx.assemble(torch.tensor(w["X"], device="cuda"), h, opts)
    a, info = ctx.solve(torch.tensor(w["y"], device="cuda"))
    a = a.cpu().numpy()
    ho = oracle.Hyper(**w["hyper"])
    csr = oracle.assemble(w["X"], ho)
    assert info["relres"] <= 1e-8
    assert np.linalg.norm(w["y"] - csr.matmat(a)) <= 1e-8 * np.linalg.norm(w["y"])
    # the same algorithm on the same Jacobi-scaled system: the oracle's MINRES reaches the first
    # stop (0.1 tol_refine on the scaled residual) within a step or two of the GPU's
    D = csr.diag()
    s = 1.0 / np.sqrt(D)
    _, k_oracle, _ = oracle.minres(csr.scaled(s), s * w["y"], tol=1e-9)
    if info["outer"] == 0:
        assert abs(info["iters"] - k_oracle) <= 2
    lml_m, i_m = ctx.lml(w["X"], w["y"], h, opts)
    e = oracle.lml_exact(w["X"], w["y"], ho)
    assert i_m["quad"] == pytest.approx(e["quad"], rel=1e-8)
    assert lml_m == pytest.approx(e["lml"], rel=1e-9)


def test_minres_with_probe_columns_and_gradient(gp):
    import oracle
    w = W.random_small(621, 4000, 2, L=3, sigma2=1e-3)
    h = gp.Hyper(**w["hyper"])
    opts = gp.default_opts(probes=32, lanczos_steps=50, seed=5, tol_probe=1e-6, solver=gp.SOLVER_MINRES,
                           logdet=gp.LOGDET_SLQ)
    lml, g, info = gp.Context(0).lml_grad(w["X"], w["y"], h, opts)
    s = oracle.lml_slq(w["X"], w["y"], oracle.Hyper(**w["hyper"]), m=32, k=50, seed=5)
    assert info["relres"] <= 1e-8
    assert info["logdet"] == pytest.approx(s["logdet"], rel=1e-3)
    assert info["quad"] == pytest.approx(s["quad"], rel=1e-7)
    assert np.abs(g - s["grad"]).max() <= 1e-6 * np.abs(s["grad"]).max()
