"""The far-field kernel (Sec. 4.5; kernel family FARFIELD) through the C ABI against the FP64 oracle:
the pattern (Euclidean ball or a shared bump) bit for bit, FP64 values to 1e-12 and FP32 values to
1e-6 of the largest, the exact LML, and the SLQ log-determinant and Hutchinson gradient with
identical probes."""
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


@pytest.fixture(scope="module")
def ctx(gp):
    return gp.Context(0)


@pytest.mark.parametrize("d,radius", [(1, 0.03), (2, 0.08), (3, 0.15)])
def test_assembly_matches_oracle(gp, ctx, d, radius):
    import oracle
    w = W.random_farfield(1100 + d, 4000, d, L=5, radius=radius)
    h = gp.Hyper(**w["hyper"])
    info = ctx.assemble(torch.tensor(w["X"], device="cuda"), h, gp.default_opts())
    c = ctx.csr()
    rp = c["rowptr"].cpu().numpy().astype(np.int64)
    col = c["col"].cpu().numpy().astype(np.int64)
    perm = c["perm"].cpu().numpy().astype(np.int64)
    s = c["dscale"].cpu().numpy()
    n = rp.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    A64 = c["val64"].cpu().numpy() / (s[rows] * s[col])
    A32 = c["val32"].cpu().numpy().astype(np.float64) / (s[rows] * s[col])
    key = perm[rows] * n + perm[col]
    order = np.argsort(key, kind="stable")
    ocsr = oracle.assemble(w["X"], oracle.Hyper(**w["hyper"]), "brute")
    okey = np.repeat(np.arange(n), np.diff(ocsr.rowptr)).astype(np.int64) * n + ocsr.col.astype(np.int64)
    assert info["nnz"] == ocsr.nnz and np.array_equal(key[order], okey)
    amax = np.abs(ocsr.val).max()
    assert np.abs(A64[order] - ocsr.val).max() <= 1e-12 * amax
    assert np.abs(A32[order] - ocsr.val).max() <= 1e-6 * amax
    for i in range(0, n, 53):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    # far pairs exist: more entries than the Euclidean ball alone
    euclid = oracle.assemble(w["X"], oracle.Hyper(**{**w["hyper"], "family": 0, "amps": w["hyper"]["amps"]}), "brute")
    assert ocsr.nnz > euclid.nnz


def test_exact_lml_matches_oracle(gp, ctx):
    import oracle
    w = W.random_farfield(1110, 3000, 2, L=4, radius=0.1)
    h = gp.Hyper(**w["hyper"])
    lml, info = ctx.lml(w["X"], w["y"], h, gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_EXACT))
    e = oracle.lml_exact(w["X"], w["y"], oracle.Hyper(**w["hyper"]))
    assert info["logdet"] == pytest.approx(e["logdet"], rel=1e-10)
    assert info["quad"] == pytest.approx(e["quad"], rel=1e-8)
    assert lml == pytest.approx(e["lml"], rel=1e-9)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_slq_and_gradient_match_oracle_with_identical_probes(gp, ctx, precision):
    import oracle
    w = W.random_farfield(1120, 4000, 2, L=4, radius=0.1, sigma2=1e-2)
    h = gp.Hyper(**w["hyper"])
    prec = gp.PREC_MIXED if precision == "mixed" else gp.PREC_FP64
    tol = 1e-6 if precision == "mixed" else 1e-11
    opts = gp.default_opts(precision=prec, logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=50, seed=7,
                           tol_probe=tol, tol_refine=min(1e-8, tol), precond=2 if precision == "mixed" else 1)
    lml, g, info = ctx.lml_grad(w["X"], w["y"], h, opts)
    s = oracle.lml_slq(w["X"], w["y"], oracle.Hyper(**w["hyper"]), m=32, k=50, seed=7, tol=1e-12)
    assert info["logdet"] == pytest.approx(s["logdet"], rel=1e-3)
    assert info["quad"] == pytest.approx(s["quad"], rel=1e-7)
    assert g.shape == s["grad"].shape == (h.nparams,)
    assert np.abs(g - s["grad"]).max() <= 1e-5 * np.abs(s["grad"]).max()
