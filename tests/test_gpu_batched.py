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


@pytest.mark.parametrize("device,probes", [("cuda", 32), (None, 16)])
def test_batched_equals_single_calls(gp, device, probes):
    """Problem by problem the batched result is the single call's with the block size the
    autotuner chose (graph replay does not change results)."""
    probs = _problems(gp, 7, 10, device)
    ctx = gp.Context(0)
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=probes, lanczos_steps=50, seed=4)
    lml_b, infos = ctx.lml_batched([(X, y, h) for X, y, h, _ in probs], opts)
    ref = gp.Context(0)
    for b, (X, y, h, _) in enumerate(probs):
        assert infos[b]["batch_config"] in (0, 1, 2, 3)
        v, info = ref.lml(X, y, h, gp.default_opts(logdet=gp.LOGDET_SLQ, probes=probes, lanczos_steps=50, seed=4,
                                                   bj_block=infos[b]["bj_block"]))
        assert lml_b[b] == v, b
        assert infos[b]["nnz"] == info["nnz"] and infos[b]["relres"] <= 1e-8


def test_autotuner_tries_every_configuration_then_keeps_the_best(gp, monkeypatch):
    # n in [4100, 8000]: one size class per d, about ten problems each, so that the first call
    # tries all four configurations in every class
    probs = []
    for w in W.batch(10, count=30, n_range=(4100, 8000), nnz_range=(10.0, 80.0)):
        probs.append((torch.tensor(w["X"], device="cuda"), torch.tensor(w["y"], device="cuda"),
                      gp.Hyper(**w["hyper"]), w))
    ctx = gp.Context(0)
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=16, lanczos_steps=40)
    _, infos = ctx.lml_batched([(X, y, h) for X, y, h, _ in probs], opts)
    cfg = [i["batch_config"] for i in infos]
    assert set(cfg) <= {0, 1, 2, 3} and len(set(cfg)) >= 2
    # a second call on the same context starts from the tuned table: one configuration per class
    _, infos2 = ctx.lml_batched([(X, y, h) for X, y, h, _ in probs], opts)
    by_class = {}
    for (X, y, h, w), i in zip(probs, infos2):
        by_class.setdefault((h.d, int(np.log2(X.shape[0]))), set()).add(i["batch_config"])
    assert all(len(v) == 1 for v in by_class.values())
    monkeypatch.setenv("GP2S_BATCH_TUNE", "0")
    _, infos3 = gp.Context(0).lml_batched([(X, y, h) for X, y, h, _ in probs[:4]], opts)
    assert all(i["batch_config"] == -1 for i in infos3)


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


def test_batch_problems_at_full_range_match_oracle(gp):
    """Three problems of the 256-problem batch itself (the largest, 64,877 points; the densest rows,
    ~197 per row; the largest 1-D one), 16 probes x 100 steps, in one batched call with other
    problems, mixed precision and the plain FP64 form, against the oracle's stored results with
    identical probes (tests/golden/oracle_batch0_p*.json)."""
    import json
    import os
    ws = W.batch(0)
    picks = (100, 32, 116)
    refs = {}
    for p in picks:
        with open(os.path.join(os.path.dirname(__file__), "golden", f"oracle_batch0_p{p}.json")) as f:
            refs[p] = json.load(f)
        np.testing.assert_allclose(W.checksums(ws[p]["X"], ws[p]["y"]), refs[p]["checksums"], rtol=1e-10, atol=0)
    sel = list(picks) + [0, 1, 2, 3, 4]
    probs = [(torch.tensor(ws[i]["X"], device="cuda"), torch.tensor(ws[i]["y"], device="cuda"),
              gp.Hyper(**ws[i]["hyper"])) for i in sel]
    ctx = gp.Context(0)
    for opts in (gp.default_opts(logdet=gp.LOGDET_SLQ, probes=16, lanczos_steps=100),
                 gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_SLQ, probes=16, lanczos_steps=100,
                                 precond=1)):
        lml_b, infos = ctx.lml_batched(probs, opts)
        for k, p in enumerate(picks):
            r = refs[p]
            assert infos[k]["nnz"] == r["nnz"]
            assert infos[k]["logdet"] == pytest.approx(r["logdet"], rel=1e-3)
            assert infos[k]["quad"] == pytest.approx(r["quad"], rel=1e-7)
            assert abs(lml_b[k] - r["lml"]) <= 0.5e-3 * abs(r["logdet"]) + 0.5e-7 * abs(r["quad"])
