"""CUDA path vs the FP64 oracle at the benchmark's own configurations, through the C ABI.

The oracle needs minutes per case at these sizes, so its results are stored in
tests/golden/oracle_<case>.json by tests/golden/make_oracle_large.py (which calls only the oracle
and the seeded input generators).  Every test regenerates the inputs, checks them against the
stored checksums, and runs the GPU with the stored hyperparameters and identical probes:

  * 150,000 points of the clustered 3-D generator (L = 8, 42 parameters, 64 probes x 100 steps,
    DEFAULT options: mixed precision, tol_probe 1e-5, block-Jacobi with 128-row blocks, the
    multi-segment SpMM reduction), at the base hyperparameters and at one drawn set;
  * 20,000 points of the same generator at 8 drawn hyperparameter sets (the gradient check at
    random theta);
  * 150,000 points of the 4-D sphere x time x elevation generator (32 probes);
  * the 10,000,000-point 4-D workload itself: log-det, quadratic term, LML and gradient against
    the oracle's run over all 10M points (its CG to 1e-8), and the y solve's residual on sampled
    rows of the oracle's A.

Bars (the LML's follows from the other two, since it is a difference of large terms):
  log-determinant 1e-3 relative (identical probes), quadratic term y^T A^{-1} y 1e-7 relative,
  |dLML| <= 1/2 1e-3 |logdet| + 1/2 1e-7 |y^T a|, gradient max |dg| <= 1e-4 max |g|.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_06143_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06143_gb300 as gp
    from paper_2512_06143_gb300 import build
    build.build()
    gp.load()
    return gp


@pytest.fixture(scope="module")
def ctx(gp):
    return gp.Context(0)


def _case(name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as f:
        ref = json.load(f)
    gen = {"clusters_3d": W.clusters_3d, "sphere_4d": W.sphere_4d}[ref["workload"]]
    w = gen(0, n=ref["n"], target_nnz=ref["target"])
    np.testing.assert_allclose(W.checksums(w["X"], w["y"]), ref["checksums"], rtol=1e-10, atol=0,
                               err_msg="the generator gave other inputs than the stored case")
    return ref, w


def _compare(gp, ctx, name, **opt_kw):
    ref, w = _case(name)
    h = gp.Hyper(**ref["hyper"])
    opts = gp.default_opts(probes=ref["probes"], lanczos_steps=ref["steps"], seed=ref["seed"], **opt_kw)
    lml, g, info = ctx.lml_grad(torch.tensor(w["X"], device="cuda"), torch.tensor(w["y"], device="cuda"), h, opts)
    assert info["nnz"] == ref["nnz"]
    assert info["relres"] <= 1e-8
    assert info["logdet"] == pytest.approx(ref["logdet"], rel=1e-3)
    assert info["quad"] == pytest.approx(ref["quad"], rel=1e-7)
    assert abs(lml - ref["lml"]) <= 0.5e-3 * abs(ref["logdet"]) + 0.5e-7 * abs(ref["quad"])
    gref = np.asarray(ref["grad"])
    assert g.shape == gref.shape
    err = np.abs(g - gref).max() / np.abs(gref).max()
    assert err <= 1e-4, err
    return info, err


@pytest.mark.parametrize("t", [0, 1])
def test_clusters_3d_150k_default_options_match_oracle(gp, ctx, t):
    info, err = _compare(gp, ctx, f"clusters_3d_150k_t{t}")
    # the paths that only turn on at this size: 128-row block-Jacobi blocks and the SpMM's
    # multi-segment reduction of its partial dots
    assert info["bj_block"] == 128
    assert info["spmm_seg_tiles"] > 1


@pytest.mark.parametrize("t", range(8))
def test_clusters_3d_20k_gradient_at_random_theta(gp, ctx, t):
    _compare(gp, ctx, f"clusters_3d_20k_t{t}", logdet=gp.LOGDET_SLQ)


def test_reliable_updates_of_the_y_column_match_oracle(gp, monkeypatch):
    """The y column's reliable updates (on by default from 2^18 rows) forced on for the 150k-point
    clustered case: the solve stops at its true FP64 residual with no restarted refinement step,
    and log-det, quadratic term, LML and gradient meet the same bars against the oracle."""
    monkeypatch.setenv("GP2S_RELIABLE_MIN_ROWS", "0")
    info, err = _compare(gp, gp.Context(0), "clusters_3d_150k_t0")
    assert info["outer"] == 0
    monkeypatch.setenv("GP2S_RELIABLE_Y", "0")
    info0, _ = _compare(gp, gp.Context(0), "clusters_3d_150k_t0")
    assert info0["outer"] >= 1


def test_sphere_4d_150k_default_options_match_oracle(gp, ctx):
    info, err = _compare(gp, ctx, "sphere_4d_150k")
    assert info["spmm_seg_tiles"] > 1


def test_sphere_4d_10m_full_size_matches_oracle(gp, ctx):
    """The whole 10M-point evaluation with default options (mixed precision, 32 probes x 100
    steps, reliable updates of the y column) against the oracle's FP64 run on the same 10M points
    with identical probes."""
    info, err = _compare(gp, ctx, "sphere_4d_10m")
    assert info["n"] == 10_000_000 and info["outer"] == 0


def test_solve_sphere_4d_full_size_sampled_residual_rows(gp, ctx):
    """10M-point 4-D workload, mixed precision with FP64 refinement: y - A a on sampled rows, the
    rows of A from the oracle's brute force over all 10M points, within 1e-8 |y| each."""
    import oracle
    w = W.sphere_4d(0)
    h = gp.Hyper(**w["hyper"])
    ctx.assemble(torch.tensor(w["X"], device="cuda"), h, gp.default_opts())
    a, info = ctx.solve(torch.tensor(w["y"], device="cuda"))
    assert info["relres"] <= 1e-8
    a = a.cpu().numpy()
    rows = np.random.default_rng(4).choice(len(a), 32, replace=False)
    ynorm = np.linalg.norm(w["y"])
    for r, (oc, ov) in zip(rows, oracle.rows_brute(w["X"], oracle.Hyper(**w["hyper"]), rows)):
        assert abs(w["y"][r] - float(ov @ a[oc])) <= 1e-8 * ynorm


def test_probe_solves_below_the_fp32_floor(gp, ctx):
    """tol_probe below the FP32 rounding level: every probe column stops by the exhausted-Krylov
    rule (its recursively updated FP32 residual reaches 1e-6 |b| before its true residual need),
    and the SLQ log-determinant and Hutchinson gradient still meet their bars against the oracle
    with identical probes (the oracle's FP64 CG runs to 1e-10)."""
    import oracle
    w = W.random_small(320, 8000, 3, L=4, sigma2=1e-4, clustered=True)
    h = gp.Hyper(**w["hyper"])
    opts = gp.default_opts(logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=80, seed=9, tol_probe=1e-9)
    lml, g, info = ctx.lml_grad(w["X"], w["y"], h, opts)
    assert info["iters_probes"] < opts.max_iter
    s = oracle.lml_slq(w["X"], w["y"], oracle.Hyper(**w["hyper"]), m=32, k=80, seed=9)
    assert info["logdet"] == pytest.approx(s["logdet"], rel=1e-3)
    assert np.abs(g - s["grad"]).max() <= 1e-4 * np.abs(s["grad"]).max()
