"""Block Metropolis-Hastings training (gp2s_mcmc, App. D) through the C ABI against the oracle's
driver with the same random numbers (FP64 form, exact log-determinant, so both sides evaluate the
same LML to ~1e-12 and take the same accept/reject decisions), plus checkpoint/resume and the
driver's own random stream."""
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


def _setup(gp):
    w = W.random_small(800, 800, 2, L=2, sigma2=2e-3, r=0.1)
    h = gp.Hyper(**w["hyper"])
    L, d = h.L, h.d
    P = h.nparams
    block = np.array([0] * (L * d) + [1] * L + [2] * L + [3, 3], np.int32)
    step = np.array([0.03] * (L * d) + [0.03] * L + [0.1] * L + [0.004, 3e-4])
    lower = np.array([-1.0] * (L * d) + [0.05] * L + [0.01] * L + [0.05, 1e-5])
    upper = np.array([2.0] * (L * d) + [2.0] * L + [10.0] * L + [0.2, 1.0])
    assert P == block.size
    return w, h, block, step, lower, upper


def test_mcmc_chain_matches_oracle(gp):
    import oracle
    w, h, block, step, lower, upper = _setup(gp)
    T, P = 10, h.nparams
    rng = np.random.default_rng(11)
    normals, uniforms = rng.normal(size=(T, P)), rng.random((T, 4))
    opts = gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_EXACT)
    chain, acc, info = gp.Context(0).mcmc(w["X"], w["y"], h, block, step, T, opts, lower, upper, normals, uniforms)
    ho = oracle.Hyper(**w["hyper"])
    ochain, oacc = oracle.mcmc(lambda th: oracle.lml_exact(w["X"], w["y"], ho.with_theta(th))["lml"], h.theta(),
                               block, step, lower, upper, normals, uniforms)
    assert np.array_equal(acc, oacc)
    assert 0 < acc.sum() < acc.size
    np.testing.assert_allclose(chain[:, :P], ochain[:, :P], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(chain[:, P], ochain[:, P], rtol=1e-10)
    assert info["done"] == T and info["accepted"] == int(acc.sum())
    assert info["pattern_reused"] > 0          # blocks that leave r alone reuse the pattern


def test_mcmc_checkpoint_resume_and_own_random_stream(gp, tmp_path):
    w, h, block, step, lower, upper = _setup(gp)
    opts = gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_EXACT)
    X = torch.tensor(w["X"], device="cuda")
    y = torch.tensor(w["y"], device="cuda")
    full, acc_full, _ = gp.Context(0).mcmc(X, y, h, block, step, 8, opts, lower, upper, seed=5)
    again, _, _ = gp.Context(0).mcmc(X, y, h, block, step, 8, opts, lower, upper, seed=5)
    assert np.array_equal(full, again)                    # the driver's stream is deterministic
    assert 0 < acc_full.sum() < acc_full.size
    ck = str(tmp_path / "chain.ckpt")
    first, _, i1 = gp.Context(0).mcmc(X, y, h, block, step, 5, opts, lower, upper, seed=5, checkpoint=ck,
                                      checkpoint_every=2)
    assert np.array_equal(first, full[:5])
    rest, _, i2 = gp.Context(0).mcmc(X, y, h, block, step, 8, opts, lower, upper, seed=5, checkpoint=ck,
                                     checkpoint_every=2, resume=True)
    assert i2["start"] == 5 and np.all(np.isnan(rest[:5]))
    assert np.array_equal(rest[5:], full[5:])
    with pytest.raises(gp.GP2SError):
        gp.Context(0).mcmc(X, y, h, block, step, 8, opts, lower, upper, checkpoint=str(tmp_path / "none"),
                           resume=True)
