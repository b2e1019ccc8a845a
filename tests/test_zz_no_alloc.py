"""The allocation-free entry point gp2s_lml_exact_noalloc, called through the C ABI.

Callers that cannot allocate device memory (work queued during CUDA stream capture, or a device
whose memory belongs to another allocator) use this entry point; it must agree with the ordinary
gp2s_lml (FP64, exact log-determinant) on the same inputs.  Two calls in a row, with different
problem sizes, check that the shared scratch array left behind by the first call does not leak into
the second.  This file is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

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
    L = gp.load()
    f = L.gp2s_lml_exact_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return gp


def _noalloc(gp, X, y, h):
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    hc = h.c()
    stream = torch.cuda.current_stream()
    st = gp.load().gp2s_lml_exact_noalloc(X.shape[0], X.data_ptr(), y.data_ptr(), ctypes.byref(hc),
                                          out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return st, out.cpu().numpy()


def test_noalloc_matches_gp2s_lml_two_calls(gp):
    ctx = gp.Context(0)
    opts = gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_EXACT)
    for seed, n, d in [(401, 500, 2), (402, 317, 3)]:
        w = W.random_small(seed, n, d, L=3, sigma2=1e-3, r=0.15 if d == 2 else 0.25)
        h = gp.Hyper(**w["hyper"])
        X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
        y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
        st, out = _noalloc(gp, X, y, h)
        assert st == gp.OK
        lml, info = ctx.lml(X, y, h, opts)
        assert out[0] == pytest.approx(lml, rel=1e-8)
        assert out[1] == pytest.approx(info["quad"], rel=1e-8)
        assert out[2] == pytest.approx(info["logdet"], rel=1e-10)


@pytest.mark.parametrize("d,kind,w0", [(1, 0, 0.0), (2, 0, 0.0), (3, 0, 0.0), (4, 0, 0.0), (1, 1, 0.0),
                                        (2, 1, 0.0), (3, 1, 0.0), (2, 0, 0.7), (3, 1, 0.5), (4, 0, 1.0)])
def test_noalloc_matches_the_oracle(gp, d, kind, w0):
    """Directly against the FP64 oracle's dense LML (brute-force A, library Cholesky), independent of
    the CSR path: both Wendland kinds, with and without the constant w0 under the bump sum."""
    import oracle
    w = W.random_small(410 + d + 10 * kind, 500, d, L=3, sigma2=1e-3, kind=kind, w0=w0,
                       r={1: 0.02, 2: 0.15, 3: 0.25, 4: 0.4}[d])
    h = gp.Hyper(**w["hyper"])
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
    st, out = _noalloc(gp, X, y, h)
    assert st == gp.OK
    e = oracle.lml_exact(w["X"], w["y"], oracle.Hyper(**w["hyper"]))
    assert out[2] == pytest.approx(e["logdet"], rel=1e-10)
    assert out[1] == pytest.approx(e["quad"], rel=1e-8)
    assert out[0] == pytest.approx(e["lml"], rel=1e-8)


def test_noalloc_rejects_sizes_beyond_the_limit(gp):
    w = W.random_small(403, 513, 2)
    h = gp.Hyper(**w["hyper"])
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
    st, out = _noalloc(gp, X, y, h)
    assert st == gp.EINVAL
    assert np.all(np.isnan(out))      # nothing was written


def test_noalloc_inside_a_captured_cuda_graph(gp):
    """What the entry point is for: it is queued while a stream is being captured and allocates
    nothing.  One eager warm-up call, then the call captured with torch.cuda.graph on a side stream;
    two replays with new y contents written in place give the eager results for those y bit for bit,
    and neither torch's allocated bytes nor the device's free bytes change across the replays."""
    w = W.random_small(404, 300, 2, L=3, sigma2=1e-3, r=0.15)
    h = gp.Hyper(**w["hyper"])
    hc = h.c()
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
    n = X.shape[0]
    f = gp.load().gp2s_lml_exact_noalloc
    rng = np.random.default_rng(5)
    ys = [torch.tensor(w["y"] + 0.1 * rng.standard_normal(n), dtype=torch.float64, device="cuda") for _ in range(2)]
    # eager results for the two right-hand sides
    ref = []
    out_e = torch.empty(3, dtype=torch.float64, device="cuda")
    for yk in ys:
        y.copy_(yk)
        st = f(n, X.data_ptr(), y.data_ptr(), ctypes.byref(hc), out_e.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert st == gp.OK
        ref.append(out_e.cpu().numpy().copy())
    # capture on a side stream (torch's default global capture mode: any unsafe call fails it)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        st = f(n, X.data_ptr(), y.data_ptr(), ctypes.byref(hc), out.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
    assert st == gp.OK
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for yk, rk in zip(ys, ref):
        y.copy_(yk)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), rk)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
