"""gp2s on GB300: exact sparse-kernel Gaussian-process log marginal likelihood (gp2Scale, arXiv
2512.06143) in hand-written CUDA for sm_103a.

This module is argument marshalling only: it loads the in-tree ``libgp2s.so`` (C ABI of
``include/gp2s.h``) with ctypes and passes tensor pointers, sizes and the current CUDA stream.
Every step of the computation runs in the library's kernels.  There is no CPU fallback: if the
library is missing or fails to load, every call raises.

    import torch, paper_2512_06143_gb300 as gp
    ctx = gp.Context()                                   # device 0, torch's current stream
    lml, grad, info = ctx.lml_grad(X, y, gp.Hyper(...))  # X: n x d, y: n (FP64, host or CUDA)
    theta.requires_grad_(); gp.GP2SLML.apply(theta, X, y, hyper, opts).backward()
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgp2s.so")

# ---------------------------------------------------------------------------------------------
# C structs (mirror include/gp2s.h)
# ---------------------------------------------------------------------------------------------
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ETIMEOUT, EOVERFLOW, ENOTPD, ENOTREADY = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOCONV", "EBREAKDOWN", "ETIMEOUT", "EOVERFLOW",
                "ENOTPD", "ENOTREADY"]
WENDLAND_C2, WENDLAND_C6_PAPER = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
LOGDET_AUTO, LOGDET_EXACT, LOGDET_SLQ = 0, 1, 2
SOLVER_CG, SOLVER_MINRES = 0, 1
KERNEL_PRODUCT, KERNEL_WENDCONV, KERNEL_FARFIELD = 0, 1, 2


class _Hyper(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("r", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("beta", ctypes.c_double), ("w0", ctypes.c_double), ("centers", ctypes.c_void_p),
                ("radii", ctypes.c_void_p), ("amps", ctypes.c_void_p), ("family", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("ell", ctypes.c_void_p), ("G", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("logdet", ctypes.c_int32), ("n_exact", ctypes.c_int32),
                ("probes", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("tol_inner", ctypes.c_double), ("tol_refine", ctypes.c_double), ("tol_probe", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("precond", ctypes.c_int32), ("exact_support", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("profile", ctypes.c_int32), ("bj_block", ctypes.c_int32),
                ("pattern_cache", ctypes.c_int32), ("solver", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class AssembleInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("band_pairs", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nnz_row_min", ctypes.c_int32),
                ("nnz_row_max", ctypes.c_int32), ("guard_delta", ctypes.c_double), ("cell_h", ctypes.c_double),
                ("ms_geometry", ctypes.c_float), ("ms_count", ctypes.c_float), ("ms_fill", ctypes.c_float),
                ("ms_values64", ctypes.c_float), ("pattern_reused", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("relres", ctypes.c_double),
                ("ms", ctypes.c_float)]


class LogdetInfo(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("probes", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("logdet_diag", ctypes.c_double), ("logdet_hat", ctypes.c_double),
                ("stderr_hat", ctypes.c_double), ("ms", ctypes.c_float)]


class LmlInfo(ctypes.Structure):
    _fields_ = [("lml", ctypes.c_double), ("quad", ctypes.c_double), ("logdet", ctypes.c_double),
                ("logdet_stderr", ctypes.c_double), ("relres", ctypes.c_double), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("iters_y", ctypes.c_int32), ("iters_probes", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("logdet_method", ctypes.c_int32), ("ms_assemble", ctypes.c_float),
                ("ms_solve", ctypes.c_float), ("ms_logdet", ctypes.c_float), ("ms_grad", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("launches", ctypes.c_int64), ("spmm_launches", ctypes.c_int64),
                ("spmm_bytes", ctypes.c_double), ("ms_spmm", ctypes.c_float), ("reserved_f", ctypes.c_float),
                ("bj_block", ctypes.c_int32), ("spmm_seg_tiles", ctypes.c_int32),
                ("pattern_reused", ctypes.c_int32), ("batch_config", ctypes.c_int32)]


class PosteriorInfo(ctypes.Structure):
    _fields_ = [("n_test", ctypes.c_int64), ("cross_entries", ctypes.c_int64), ("batches", ctypes.c_int32),
                ("iters_max", ctypes.c_int32), ("ms_mean", ctypes.c_float), ("ms_var", ctypes.c_float)]


class McmcOpts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("block", ctypes.c_void_p),
                ("step", ctypes.c_void_p), ("lower", ctypes.c_void_p), ("upper", ctypes.c_void_p),
                ("normals", ctypes.c_void_p), ("uniforms", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("checkpoint", ctypes.c_char_p), ("checkpoint_every", ctypes.c_int32), ("resume", ctypes.c_int32)]


class McmcInfo(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int32), ("done", ctypes.c_int32), ("evals", ctypes.c_int32),
                ("pattern_reused", ctypes.c_int32), ("accepted", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lml", ctypes.c_double), ("ms", ctypes.c_float), ("reserved_f", ctypes.c_float)]


class CsrView(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("val32", ctypes.c_void_p),
                ("val64", ctypes.c_void_p), ("dscale", ctypes.c_void_p)]


EXPORTED = ["gp2s_opts_default", "gp2s_num_params", "gp2s_num_params_family", "gp2s_create", "gp2s_destroy", "gp2s_last_error",
            "gp2s_assemble", "gp2s_csr", "gp2s_solve", "gp2s_logdet", "gp2s_lml", "gp2s_lml_grad",
            "gp2s_lml_batched", "gp2s_posterior", "gp2s_mcmc", "gp2s_lml_exact_noalloc"]

_lib = None


class GP2SError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


def library_path() -> str:
    return LIB_PATH


def load(path: str | None = None):
    """Load libgp2s.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2512_06143_gb300.build.build() "
                           "(nvcc, sm_103a); gp2s has no CPU fallback")
    L = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sigs = {
        "gp2s_opts_default": (None, [vp]),
        "gp2s_num_params": (i32, [i32, i32]),
        "gp2s_num_params_family": (i32, [i32, i32, i32]),
        "gp2s_create": (i32, [ctypes.POINTER(vp), ctypes.c_int, vp]),
        "gp2s_destroy": (None, [vp]),
        "gp2s_last_error": (ctypes.c_char_p, [vp]),
        "gp2s_assemble": (i32, [vp, i64, vp, vp, vp, vp]),
        "gp2s_csr": (i32, [vp, vp]),
        "gp2s_solve": (i32, [vp, vp, vp, vp]),
        "gp2s_logdet": (i32, [vp, vp, vp, vp]),
        "gp2s_lml": (i32, [vp, i64, vp, vp, vp, vp, vp, vp]),
        "gp2s_lml_grad": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, vp]),
        "gp2s_lml_batched": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "gp2s_lml_exact_noalloc": (i32, [i64, vp, vp, vp, vp, vp]),
        "gp2s_posterior": (i32, [vp, i64, vp, vp, vp, vp]),
        "gp2s_mcmc": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------------------------------------
# Python-side parameter objects
# ---------------------------------------------------------------------------------------------
@dataclass
class Hyper:
    """Kernel + noise hyperparameters: Wendland radius r, noise sigma2, L bumps (centers L x d,
    radii, amplitudes), bump shape beta, constant w0, Wendland kind."""
    d: int
    r: float
    sigma2: float
    centers: np.ndarray
    radii: np.ndarray
    amps: np.ndarray
    beta: float = 1.0
    w0: float = 0.0
    kind: int = WENDLAND_C2
    family: int = KERNEL_PRODUCT
    ell: np.ndarray | None = None     # KERNEL_WENDCONV: d base length-scale factors
    G: np.ndarray | None = None       # KERNEL_WENDCONV: L x d weights of the length-scale field
    _keep: list = field(default_factory=list, repr=False)

    @property
    def L(self) -> int:
        return int(np.asarray(self.radii).shape[0])

    @property
    def nparams(self) -> int:
        if self.family == KERNEL_WENDCONV:
            return self.L * (2 * self.d + 2) + self.d + 3
        if self.family == KERNEL_FARFIELD:
            return self.L * (self.d + 2) + 4
        return self.L * (self.d + 2) + 2

    def theta(self) -> np.ndarray:
        """[centers (L x d), radii (L), amps (L), r, sigma2] (product kernel), or
        [centers, radii, amps, G (L x d), ell (d), w0, r, sigma2] (Wendland convolution)."""
        head = [np.asarray(self.centers, np.float64).ravel(), np.asarray(self.radii, np.float64),
                np.asarray(self.amps, np.float64)]
        if self.family == KERNEL_WENDCONV:
            head += [np.asarray(self.G, np.float64).ravel(), np.asarray(self.ell, np.float64), [self.w0]]
        if self.family == KERNEL_FARFIELD:
            head += [[float(np.asarray(self.ell, np.float64).ravel()[0]), self.w0]]
        return np.concatenate(head + [[self.r, self.sigma2]])

    def with_theta(self, th) -> "Hyper":
        th = np.asarray(th, np.float64)
        L, d = self.L, self.d
        kw = dict(d=d, centers=th[:L * d].reshape(L, d).copy(), radii=th[L * d:L * d + L].copy(),
                  amps=th[L * d + L:L * d + 2 * L].copy(), r=float(th[-2]), sigma2=float(th[-1]),
                  beta=self.beta, w0=self.w0, kind=self.kind, family=self.family)
        if self.family == KERNEL_WENDCONV:
            o = L * d + 2 * L
            kw.update(G=th[o:o + L * d].reshape(L, d).copy(), ell=th[o + L * d:o + L * d + d].copy(),
                      w0=float(th[o + L * d + d]))
        if self.family == KERNEL_FARFIELD:
            o = L * d + 2 * L
            kw.update(ell=np.array([th[o]]), w0=float(th[o + 1]))
        return Hyper(**kw)

    def c(self) -> _Hyper:
        c = np.ascontiguousarray(np.asarray(self.centers, np.float64).reshape(self.L, self.d))
        r = np.ascontiguousarray(np.asarray(self.radii, np.float64))
        a = np.ascontiguousarray(np.asarray(self.amps, np.float64))
        e = np.ascontiguousarray(np.asarray(self.ell if self.ell is not None else np.ones(self.d), np.float64).ravel())
        g = np.ascontiguousarray(np.asarray(self.G if self.G is not None else np.zeros((self.L, self.d)),
                                            np.float64).reshape(self.L, self.d))
        self._keep = [c, r, a, e, g]
        return _Hyper(self.d, self.L, int(self.kind), 0, float(self.r), float(self.sigma2), float(self.beta),
                      float(self.w0), c.ctypes.data, r.ctypes.data, a.ctypes.data, int(self.family), 0,
                      e.ctypes.data, g.ctypes.data)


def default_opts(**kw) -> Opts:
    o = Opts()
    load().gp2s_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _struct_dict(s) -> dict:
    return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved"}


def _ptr(x):
    """(pointer, keepalive) for a numpy array or a torch tensor (host or CUDA), FP64 contiguous."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            t = x.detach()
            if t.dtype != torch.float64:
                t = t.to(torch.float64)
            t = t.contiguous()
            return t.data_ptr(), t
    except ImportError:
        pass
    a = np.ascontiguousarray(np.asarray(x, np.float64))
    return a.ctypes.data, a


def _stream_handle(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class Context:
    """One engine context on one CUDA device; all work goes on `stream` (default: torch's current
    stream at construction)."""

    def __init__(self, device: int = 0, stream=None):
        L = load()
        h = ctypes.c_void_p()
        st = L.gp2s_create(ctypes.byref(h), int(device), _stream_handle(stream))
        if st != OK:
            raise GP2SError(st, "gp2s_create failed (no CUDA device?)")
        self._h = h
        self._lib = L

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gp2s_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != OK and st not in allow:
            raise GP2SError(st, self._lib.gp2s_last_error(self._h).decode())
        return st

    # -- entry points ---------------------------------------------------------------------------
    def assemble(self, X, hyper: Hyper, opts: Opts | None = None) -> dict:
        px, kx = _ptr(X)
        n = int(kx.shape[0])
        hc = hyper.c()
        info = AssembleInfo()
        o = opts or default_opts()
        self._check(self._lib.gp2s_assemble(self._h, n, px, ctypes.byref(hc), ctypes.byref(o), ctypes.byref(info)))
        return _struct_dict(info)

    def csr_view(self) -> CsrView:
        v = CsrView()
        self._check(self._lib.gp2s_csr(self._h, ctypes.byref(v)))
        return v

    def csr(self) -> dict:
        """Copies of the assembled CSR (sorted numbering) as torch CUDA tensors."""
        import torch
        v = self.csr_view()
        n, nnz = int(v.n), int(v.nnz)

        typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.float64: "<f8"}

        def wrap(ptr, count, dtype):
            if not ptr or count == 0:
                return None
            view = _CudaArray(ptr, count, typestr[dtype])
            return torch.as_tensor(view, device="cuda").clone()

        return dict(n=n, nnz=nnz, rowptr=wrap(v.rowptr, n + 1, torch.int32), col=wrap(v.col, nnz, torch.int32),
                    perm=wrap(v.perm, n, torch.int32), val32=wrap(v.val32, nnz, torch.float32),
                    val64=wrap(v.val64, nnz, torch.float64), dscale=wrap(v.dscale, n, torch.float64))

    def solve(self, y, out=None) -> tuple:
        py, ky = _ptr(y)
        n = int(ky.shape[0])
        if out is None:
            import torch
            out = torch.empty(n, dtype=torch.float64, device=ky.device) if isinstance(ky, torch.Tensor) else np.empty(n)
        pa, ka = _ptr(out)
        info = SolveInfo()
        self._check(self._lib.gp2s_solve(self._h, py, pa, ctypes.byref(info)), allow=(ENOCONV,))
        return ka, _struct_dict(info)

    def logdet(self) -> tuple:
        ld = ctypes.c_double()
        se = ctypes.c_double()
        info = LogdetInfo()
        self._check(self._lib.gp2s_logdet(self._h, ctypes.byref(ld), ctypes.byref(se), ctypes.byref(info)))
        return ld.value, se.value, _struct_dict(info)

    def lml(self, X, y, hyper: Hyper, opts: Opts | None = None) -> tuple:
        px, kx = _ptr(X)
        py, ky = _ptr(y)
        hc = hyper.c()
        o = opts or default_opts()
        out = ctypes.c_double()
        info = LmlInfo()
        self._check(self._lib.gp2s_lml(self._h, int(kx.shape[0]), px, py, ctypes.byref(hc), ctypes.byref(o),
                                       ctypes.byref(out), ctypes.byref(info)))
        return out.value, _struct_dict(info)

    def lml_grad(self, X, y, hyper: Hyper, opts: Opts | None = None) -> tuple:
        px, kx = _ptr(X)
        py, ky = _ptr(y)
        hc = hyper.c()
        o = opts or default_opts()
        out = ctypes.c_double()
        g = np.empty(hyper.nparams)
        info = LmlInfo()
        self._check(self._lib.gp2s_lml_grad(self._h, int(kx.shape[0]), px, py, ctypes.byref(hc), ctypes.byref(o),
                                            ctypes.byref(out), g.ctypes.data, ctypes.byref(info)))
        return out.value, g, _struct_dict(info)

    def posterior(self, Xtest, variance: bool = True) -> tuple:
        """Posterior mean (and latent variance) of Eq. 2 at Xtest (n* x d) on the last solved
        problem.  Outputs are CUDA tensors when Xtest is one, else numpy arrays."""
        px, kx = _ptr(Xtest)
        ns = int(kx.shape[0])
        try:
            import torch
            on_dev = isinstance(kx, torch.Tensor) and kx.is_cuda
        except ImportError:
            on_dev = False
        if on_dev:
            mean = torch.empty(ns, dtype=torch.float64, device=kx.device)
            var = torch.empty(ns, dtype=torch.float64, device=kx.device) if variance else None
        else:
            mean = np.empty(ns)
            var = np.empty(ns) if variance else None
        pm, km = _ptr(mean)
        pv = _ptr(var)[0] if variance else None
        info = PosteriorInfo()
        self._check(self._lib.gp2s_posterior(self._h, ns, px, pm, pv, ctypes.byref(info)))
        return mean, var, _struct_dict(info)

    def mcmc(self, X, y, hyper0: Hyper, block, step, iters: int, opts: Opts | None = None, lower=None,
             upper=None, normals=None, uniforms=None, seed: int = 0, checkpoint: str | None = None,
             checkpoint_every: int = 0, resume: bool = False) -> tuple:
        """Block Metropolis-Hastings over theta (App. D).  block / step / lower / upper: one entry per
        theta component.  Returns (chain iters x (P + 1), accept iters x nblocks, info)."""
        px, kx = _ptr(X)
        py, ky = _ptr(y)
        P = hyper0.nparams
        blk = np.ascontiguousarray(np.asarray(block, np.int32))
        stp = np.ascontiguousarray(np.asarray(step, np.float64))
        if blk.shape != (P,) or stp.shape != (P,):
            raise ValueError("block and step need one entry per theta component")
        nb = int(blk.max()) + 1 if blk.size else 1
        keep = [blk, stp]

        def arr(a, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, np.float64))
            if a.shape != shape:
                raise ValueError(f"expected shape {shape}, got {a.shape}")
            keep.append(a)
            return a.ctypes.data

        mo = McmcOpts(int(iters), nb, blk.ctypes.data, stp.ctypes.data, arr(lower, (P,)), arr(upper, (P,)),
                      arr(normals, (int(iters), P)), arr(uniforms, (int(iters), nb)), int(seed) & (2**64 - 1),
                      checkpoint.encode() if checkpoint else None, int(checkpoint_every), 1 if resume else 0)
        hc = hyper0.c()
        o = opts or default_opts()
        chain = np.full((int(iters), P + 1), np.nan)
        acc = np.zeros((int(iters), nb), np.int32)
        info = McmcInfo()
        self._check(self._lib.gp2s_mcmc(self._h, int(kx.shape[0]), px, py, ctypes.byref(hc), ctypes.byref(o),
                                        ctypes.byref(mo), chain.ctypes.data, acc.ctypes.data, ctypes.byref(info)))
        return chain, acc, _struct_dict(info)

    def lml_batched(self, problems: list, opts: Opts | None = None) -> tuple:
        """problems: list of (X, y, Hyper).  Returns (lml array, list of info dicts)."""
        B = len(problems)
        keep = []
        ns = np.array([int(np.asarray(p[0].shape[0])) for p in problems], np.int64)
        Xp = (ctypes.c_void_p * B)()
        Yp = (ctypes.c_void_p * B)()
        H = (_Hyper * B)()
        for b, (X, y, h) in enumerate(problems):
            px, kx = _ptr(X)
            py, ky = _ptr(y)
            keep += [kx, ky, h]
            Xp[b], Yp[b] = px, py
            H[b] = h.c()
            keep.append(list(h._keep))
        o = opts or default_opts()
        out = np.empty(B)
        infos = (LmlInfo * B)()
        self._check(self._lib.gp2s_lml_batched(self._h, B, ns.ctypes.data, ctypes.cast(Xp, ctypes.c_void_p),
                                               ctypes.cast(Yp, ctypes.c_void_p), ctypes.cast(H, ctypes.c_void_p),
                                               ctypes.byref(o), out.ctypes.data, ctypes.cast(infos, ctypes.c_void_p)))
        return out, [_struct_dict(infos[b]) for b in range(B)]


class _CudaArray:
    """A borrowed 1-D device buffer exposed through __cuda_array_interface__ (so torch can view it)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


# ---------------------------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------------------------
_default_ctx = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


def _autograd_function():
    import torch

    class GP2SLML(torch.autograd.Function):
        """LML(theta) with theta = [centers (L x d), radii (L), amps (L), r, sigma2] (FP64 tensor);
        forward calls gp2s_lml_grad once and keeps the gradient for backward."""

        @staticmethod
        def forward(ctx, theta, X, y, hyper: Hyper, opts: Opts | None = None):
            h = hyper.with_theta(theta.detach().cpu().numpy())
            dev = X.device.index if isinstance(X, torch.Tensor) and X.is_cuda else 0
            val, g, _ = default_context(dev or 0).lml_grad(X, y, h, opts)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return torch.tensor(val, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None, None

    return GP2SLML


def __getattr__(name):
    if name == "GP2SLML":
        fn = _autograd_function()
        globals()["GP2SLML"] = fn
        return fn
    raise AttributeError(name)
