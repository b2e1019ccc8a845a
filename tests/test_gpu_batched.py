"""Batched form (gp2s_lml_batched): many uneven problems in one call must give, problem by problem,
exactly what single gp2s_lml calls give (same kernels, deterministic reductions), and agree with the
FP64 oracle's SLQ with identical probes."""
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


def _problems(gp, seed, count, device):
    out = []
    for w in W.batch(seed, count=count, n_range=(1500, 6000), nnz_range=(10.0, 80.0)):
        X = torch.tensor(w["X"], device=device) if device else w["X"]
        y = torch.tensor(w["y"], device=device) if device else w["y"]
        out.append((X, y, gp.Hyper(**w["hyper"]), w))
    return out


@pytest.mark.parametrize("device", ["cuda", None])
def test_batched_equals_single_calls(gp, device):
    probs = _problems(gp, 7, 10, device)
    ctx = gp.Context(0)
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=50, seed=4)
    lml_b, infos = ctx.lml_batched([(X, y, h) for X, y, h, _ in probs], opts)
    ref = gp.Context(0)
    for b, (X, y, h, _) in enumerate(probs):
        v, info = ref.lml(X, y, h, opts)
        assert lml_b[b] == v, b
        assert infos[b]["nnz"] == info["nnz"] and infos[b]["relres"] <= 1e-8


def test_batched_matches_oracle(gp):
    import oracle
    probs = _problems(gp, 8, 4, "cuda")
    ctx = gp.Context(0)
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=60, seed=9)
    lml_b, infos = ctx.lml_batched([(X, y, h) for X, y, h, _ in probs], opts)
    for b, (_, _, _, w) in enumerate(probs):
        s = oracle.lml_slq(w["X"], w["y"], oracle.Hyper(**w["hyper"]), m=32, k=60, seed=9, grad=False)
        assert infos[b]["logdet"] == pytest.approx(s["logdet"], rel=1e-3)
        assert infos[b]["quad"] == pytest.approx(s["quad"], rel=1e-7)
        # the LML inherits the log-det's 1e-3 (relative to log|A|, which can be much larger than
        # the LML itself) and the quadratic form's 1e-7, each with the factor 1/2 of the LML (Sec. 3)
        tol = 0.5e-3 * abs(s["logdet"]) + 0.5e-7 * abs(s["quad"])
        assert abs(lml_b[b] - s["lml"]) <= tol


def test_batched_reports_a_failing_problem(gp):
    probs = _problems(gp, 9, 3, "cuda")
    bad = probs[1][2].with_theta(probs[1][2].theta())
    bad.r = -1.0
    ctx = gp.Context(0)
    with pytest.raises(gp.GP2SError) as e:
        ctx.lml_batched([(probs[0][0], probs[0][1], probs[0][2]), (probs[1][0], probs[1][1], bad),
                         (probs[2][0], probs[2][1], probs[2][2])], gp.default_opts(probes=32))
    assert e.value.status == gp.EINVAL
    assert "problem 1" in str(e.value)
