"""Pattern reuse across evaluations (opts.pattern_cache = 0, the default): when X and r are the
same as in the last assembly, only the bump tables and values are recomputed.  The result must be
bit-identical to a fresh assembly of the same hyperparameters, and any change of X, r, the
support option or the precision must rebuild the pattern."""
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


def test_reused_pattern_gives_bit_identical_results(gp):
    w = W.random_small(700, 20000, 3, L=4, sigma2=1e-3, clustered=True)
    X = torch.tensor(w["X"], device="cuda")
    y = torch.tensor(w["y"], device="cuda")
    h1 = gp.Hyper(**w["hyper"])
    th = h1.theta()
    th2 = th.copy()
    th2[:h1.L * h1.d] += 0.05            # move the bump centers, keep r and sigma2
    th2[h1.L * h1.d + h1.L:h1.L * h1.d + 2 * h1.L] *= 1.3
    h2 = h1.with_theta(th2)
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=50, seed=4)
    ctx = gp.Context(0)
    _, _, i1 = ctx.lml_grad(X, y, h1, opts)
    assert i1["pattern_reused"] == 0
    lml_c, g_c, i2 = ctx.lml_grad(X, y, h2, opts)
    assert i2["pattern_reused"] == 1 and i2["nnz"] == i1["nnz"]
    lml_f, g_f, i3 = gp.Context(0).lml_grad(X, y, h2, opts)
    assert i3["pattern_reused"] == 0
    assert lml_c == lml_f and np.array_equal(g_c, g_f)
    assert i2["iters_y"] == i3["iters_y"] and i2["iters_probes"] == i3["iters_probes"]


def test_changes_that_rebuild_the_pattern(gp):
    w = W.random_small(701, 6000, 2, L=3, sigma2=1e-3)
    X = torch.tensor(w["X"], device="cuda")
    y = torch.tensor(w["y"], device="cuda")
    h = gp.Hyper(**w["hyper"])
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=30)
    ctx = gp.Context(0)
    ctx.lml(X, y, h, opts)
    assert ctx.lml(X, y, h, opts)[1]["pattern_reused"] == 1
    hr = gp.Hyper(**{**w["hyper"], "r": w["hyper"]["r"] * 1.01})
    assert ctx.lml(X, y, hr, opts)[1]["pattern_reused"] == 0
    assert ctx.lml(X, y, hr, opts)[1]["pattern_reused"] == 1
    X2 = X.clone()
    X2[17, 1] += 1e-12
    assert ctx.lml(X2, y, hr, opts)[1]["pattern_reused"] == 0
    assert ctx.lml(X2, y, hr, gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=30,
                                               exact_support=1))[1]["pattern_reused"] == 0
    assert ctx.lml(X2, y, hr, gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=30,
                                               pattern_cache=1))[1]["pattern_reused"] == 0
    assert ctx.lml(X2, y, hr, gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=30,
                                               precision=gp.PREC_FP64))[1]["pattern_reused"] == 0
