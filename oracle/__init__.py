"""FP64 CPU oracle for the sparse-kernel GP log marginal likelihood (gp2Scale, arXiv 2512.06143).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  Nothing here imports, loads or calls the CUDA package, and
the CUDA package never imports this one.  The per-pair and sparse loops live in
``gp2s_oracle.c`` (plain C, FP64, no fused multiply-add); this module strings them together in
the order the paper states the method, using numpy / scipy library routines (Cholesky, a
symmetric eigensolver, a k-d tree candidate search) as single steps.

What each function follows:
  * ``assemble``        -- Sec. 4.6: every pair is evaluated; A = K + sigma^2 I (Sec. 3), with the
                           product kernel of Sec. 4.1 / 4.3 (family 0), the Wendland
                           convolution kernel of Eq. 6, Sec. 4.2 (family 1), or the far-field
                           form of Sec. 4.5 with a global core (family 2).
  * ``lml_exact``       -- the LML of Sec. 3 (Background) with m = 0, V = sigma^2 I, by a dense
                           Cholesky factorisation (solve and log-determinant exactly).
  * ``grad_exact``      -- the standard LML derivative 1/2 a^T dA a - 1/2 tr(A^{-1} dA) with the
                           dense inverse (exact trace).
  * ``posterior``       -- Eq. 2 (Sec. 3): posterior mean k(X,x*)^T A^{-1} y and latent variance
                           k(x*,x*) - k(X,x*)^T A^{-1} k(X,x*), A = K + sigma^2 I, by a dense
                           Cholesky factorisation of the brute-force A and cross-covariance.
  * ``minres``          -- the solver the paper uses for K^{-1} y (App. B.6): MINRES (Paige &
                           Saunders 1975), the Lanczos process with Givens rotations.
  * ``mcmc``            -- App. D's block Metropolis-Hastings training: normal random-walk
                           proposals per parameter block, a flat prior inside bounds, one LML
                           evaluation per block per iteration.
  * ``lml_slq``         -- where the paper leaves the log-determinant method open (Sec. 4.6,
                           App. B.7): Jacobi-scaled conjugate gradients for a = A^{-1} y,
                           stochastic Lanczos quadrature (Ubaru, Chen & Saad 2017) with
                           Rademacher probes for log|A|, Hutchinson's estimator for the trace.

Every function here is pinned by the ``-m "not gpu"`` tests against closed forms, library
routines, brute force on tiny inputs and finite differences; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp2s_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gp2s.so")
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
          "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FMA contraction) next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Hyper(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("L", ctypes.c_int), ("kind", ctypes.c_int),
                ("pad_", ctypes.c_int), ("r", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("beta", ctypes.c_double), ("w0", ctypes.c_double),
                ("centers", ctypes.c_void_p), ("radii", ctypes.c_void_p),
                ("amps", ctypes.c_void_p), ("family", ctypes.c_int), ("pad2_", ctypes.c_int),
                ("ell", ctypes.c_void_p), ("G", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, i32, dbl, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_uint64)
        hp = ctypes.POINTER(_Hyper)
        sig = {
            "orc_splitmix64": (u64, [u64]),
            "orc_rademacher": (None, [i64, i32, u64, vp]),
            "orc_phi": (dbl, [i32, i32, dbl]),
            "orc_dphi": (dbl, [i32, i32, dbl]),
            "orc_bumps": (None, [hp, vp, vp, vp]),
            "orc_sqdist": (dbl, [i32, vp, vp]),
            "orc_in_pattern": (i32, [i32, vp, vp, dbl]),
            "orc_kernel": (dbl, [hp, vp, vp]),
            "orc_assemble_brute": (i64, [i64, vp, hp, vp, vp, vp]),
            "orc_row_brute": (i64, [i64, vp, hp, i64, vp, vp]),
            "orc_rows_brute": (None, [i64, vp, hp, i64, vp, vp, vp, vp]),
            "orc_assemble_candidates": (i64, [i64, vp, hp, i64, vp, vp, vp, vp, vp]),
            "orc_dense_A": (None, [i64, vp, hp, vp]),
            "orc_cross_K": (None, [i64, vp, i64, vp, hp, vp]),
            "orc_point_values": (None, [hp, i64, vp, vp]),
            "orc_wc_q": (dbl, [i32, vp, vp, vp, vp]),
            "orc_dphi_over_t": (dbl, [i32, i32, dbl]),
            "orc_spmm": (None, [i64, vp, vp, vp, i32, vp, vp]),
            "orc_cg": (i32, [i64, vp, vp, vp, i32, vp, vp, dbl, i32, i32, vp, vp, vp]),
            "orc_lanczos": (None, [i64, vp, vp, vp, i32, vp, i32, vp, vp, vp]),
            "orc_grad_contract": (i32, [i64, vp, vp, vp, hp, vp, i32, vp, vp, vp, vp]),
            "orc_num_threads": (i32, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------------------
# Hyperparameters
# ----------------------------------------------------------------------------------------
@dataclass
class Hyper:
    """Kernel + noise hyperparameters (Eq. 3, Eq. 7, Sec. 3 noise)."""
    d: int
    r: float
    sigma2: float
    centers: np.ndarray          # L x d
    radii: np.ndarray            # L
    amps: np.ndarray             # L
    beta: float = 1.0
    w0: float = 0.0
    kind: int = 0                # 0 = Wendland C2 reading, 1 = Eq. 3 C6
    family: int = 0              # 0 = product kernel (Sec. 4.1 / 4.3), 1 = Wendland convolution (Eq. 6)
    ell: np.ndarray | None = None   # family 1: d base length-scale factors
    G: np.ndarray | None = None     # family 1: L x d weights of the length-scale field
    _keep: list = field(default_factory=list, repr=False)

    @property
    def L(self) -> int:
        return int(np.asarray(self.radii).shape[0])

    @property
    def nparams(self) -> int:
        if self.family == 1:
            return self.L * (2 * self.d + 2) + self.d + 3
        if self.family == 2:
            return self.L * (self.d + 2) + 4
        return self.L * (self.d + 2) + 2

    def theta(self) -> np.ndarray:
        """theta = [centers (L x d row-major), radii (L), amps (L), r, sigma2] (family 0), or
        [centers, radii, amps, G (L x d), ell (d), w0, r, sigma2] (family 1)."""
        head = [np.asarray(self.centers, np.float64).ravel(), np.asarray(self.radii, np.float64),
                np.asarray(self.amps, np.float64)]
        if self.family == 1:
            head += [np.asarray(self.G, np.float64).ravel(), np.asarray(self.ell, np.float64), [self.w0]]
        if self.family == 2:
            head += [[float(np.asarray(self.ell, np.float64).ravel()[0]), self.w0]]
        return np.concatenate(head + [[self.r, self.sigma2]])

    def with_theta(self, th) -> "Hyper":
        th = np.asarray(th, np.float64)
        L, d = self.L, self.d
        kw = dict(d=d, centers=th[:L * d].reshape(L, d).copy(), radii=th[L * d:L * d + L].copy(),
                  amps=th[L * d + L:L * d + 2 * L].copy(), r=float(th[-2]), sigma2=float(th[-1]),
                  beta=self.beta, w0=self.w0, kind=self.kind, family=self.family)
        if self.family == 1:
            o = L * d + 2 * L
            kw.update(G=th[o:o + L * d].reshape(L, d).copy(), ell=th[o + L * d:o + L * d + d].copy(),
                      w0=float(th[o + L * d + d]))
        if self.family == 2:
            o = L * d + 2 * L
            kw.update(ell=np.array([th[o]]), w0=float(th[o + 1]))
        return Hyper(**kw)

    def c(self):
        c = np.ascontiguousarray(np.asarray(self.centers, np.float64).reshape(self.L, self.d))
        rr = np.ascontiguousarray(np.asarray(self.radii, np.float64))
        aa = np.ascontiguousarray(np.asarray(self.amps, np.float64))
        ee = np.ascontiguousarray(np.asarray(self.ell if self.ell is not None else np.ones(self.d), np.float64).ravel())
        gg = np.ascontiguousarray(np.asarray(self.G if self.G is not None else np.zeros((self.L, self.d)),
                                             np.float64).reshape(self.L, self.d))
        self._keep = [c, rr, aa, ee, gg]
        h = _Hyper(self.d, self.L, self.kind, 0, float(self.r), float(self.sigma2),
                   float(self.beta), float(self.w0), _p(c), _p(rr), _p(aa), int(self.family), 0, _p(ee), _p(gg))
        return ctypes.byref(h), h


# ----------------------------------------------------------------------------------------
# Scalar pieces (exposed for the pins)
# ----------------------------------------------------------------------------------------
def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def probes(n: int, m: int, seed: int) -> np.ndarray:
    """Rademacher probes z (n x m), z[i, s-1] for probe s = 1..m at original index i."""
    z = np.empty((n, m), np.float64)
    if n and m:
        lib().orc_rademacher(n, m, ctypes.c_uint64(seed & (2**64 - 1)), _p(z))
    return z


def phi(kind: int, d: int, t) -> np.ndarray:
    f = lib().orc_phi
    return np.vectorize(lambda v: f(kind, d, float(v)))(np.asarray(t, np.float64))


def dphi(kind: int, d: int, t) -> np.ndarray:
    f = lib().orc_dphi
    return np.vectorize(lambda v: f(kind, d, float(v)))(np.asarray(t, np.float64))


def bumps(h: Hyper, x, with_grad: bool = False):
    """b_l(x) for every bump (and d b_l / d (c_l, rho_l, a_l) when with_grad)."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(h.d))
    b = np.empty(h.L)
    db = np.empty(h.L * (h.d + 2)) if with_grad else None
    hr, _keep = h.c()
    lib().orc_bumps(hr, _p(x), _p(b), _p(db))
    return (b, db.reshape(h.L, h.d + 2)) if with_grad else b


def kernel(h: Hyper, xi, xj) -> float:
    xi = np.ascontiguousarray(np.asarray(xi, np.float64).reshape(h.d))
    xj = np.ascontiguousarray(np.asarray(xj, np.float64).reshape(h.d))
    hr, _keep = h.c()
    return float(lib().orc_kernel(hr, _p(xi), _p(xj)))


# ----------------------------------------------------------------------------------------
# Assembly (Sec. 4.6) -> CSR of A = K + sigma^2 I in original index order, columns ascending
# ----------------------------------------------------------------------------------------
@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int64 n+1
    col: np.ndarray      # int32 nnz
    val: np.ndarray      # float64 nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def diag(self) -> np.ndarray:
        out = np.zeros(self.n)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        m = rows == self.col
        out[rows[m]] = self.val[m]
        return out

    def matmat(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float64)
        one = X.ndim == 1
        Xm = X.reshape(self.n, -1)
        Y = np.empty_like(Xm)
        lib().orc_spmm(self.n, _p(self.rowptr), _p(self.col), _p(self.val), Xm.shape[1], _p(Xm), _p(Y))
        return Y.ravel() if one else Y

    def scaled(self, s: np.ndarray) -> "CSR":
        """diag(s) M diag(s) (Jacobi scaling with s = D^{-1/2})."""
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        return CSR(self.n, self.rowptr, self.col, self.val * s[rows] * s[self.col])


def assemble(X, h: Hyper, method: str = "auto") -> CSR:
    """A = K + sigma^2 I as CSR.  method: 'brute' (all n^2 pairs, Sec. 4.6), 'tree'
    (k-d-tree candidates, each decided by the same exact FP64 test), or 'auto'."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    n = X.shape[0]
    if method == "auto":
        method = "brute" if n <= 20000 or h.family == 2 else "tree"
    hr, _keep = h.c()
    rowptr = np.zeros(n + 1, np.int64)
    L = lib()
    if method == "brute":
        nnz = L.orc_assemble_brute(n, _p(X), hr, _p(rowptr), None, None)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        L.orc_assemble_brute(n, _p(X), hr, _p(rowptr), _p(col), _p(val))
        return CSR(n, rowptr, col, val)
    if method == "tree":
        from scipy.spatial import cKDTree
        # enlarged search radius: a superset of every pair in the pattern (d2 < r*r; for the
        # Wendland convolution Q < r*r needs |D| < r sqrt(max lambda))
        if h.family == 2:
            raise ValueError("the far-field kernel's pattern is not a Euclidean ball: use method='brute'")
        rs = float(h.r) * (1.0 + 1e-9) + 1e-300
        if h.family == 1:
            pv = point_values(X, h)
            rs = float(h.r) * math.sqrt(float(pv[:, 1:].max())) * (1.0 + 1e-9) + 1e-300
        pairs = cKDTree(X).query_pairs(rs, output_type="ndarray").astype(np.int64)
        ci = np.ascontiguousarray(pairs[:, 0])
        cj = np.ascontiguousarray(pairs[:, 1])
        del pairs
        nnz = L.orc_assemble_candidates(n, _p(X), hr, ci.shape[0], _p(ci), _p(cj), _p(rowptr), None, None)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        L.orc_assemble_candidates(n, _p(X), hr, ci.shape[0], _p(ci), _p(cj), _p(rowptr), _p(col), _p(val))
        return CSR(n, rowptr, col, val)
    raise ValueError(method)


def point_values(X, h: Hyper) -> np.ndarray:
    """Per-point kernel quantities: the bump values (family 0, n x L) or [s, lambda_1..d]
    (family 1, n x (d + 1))."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    w = h.d + 1 if h.family == 1 else (2 * h.L if h.family == 2 else h.L)
    out = np.empty((X.shape[0], max(w, 1)))
    hr, _keep = h.c()
    lib().orc_point_values(hr, X.shape[0], _p(X), _p(out))
    return out


def rows_brute(X, h: Hyper, rows) -> list:
    """[(cols, vals)] for the given rows of A by brute force over all n points."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    n = X.shape[0]
    rows = np.ascontiguousarray(np.asarray(rows, np.int64))
    out = []
    hr, _keep = h.c()
    step = max(1, min(len(rows), (1 << 27) // max(n, 1)))
    for a in range(0, len(rows), step):
        rr = rows[a:a + step]
        cols = np.empty((len(rr), n), np.int32)
        vals = np.empty((len(rr), n), np.float64)
        cnt = np.empty(len(rr), np.int64)
        lib().orc_rows_brute(n, _p(X), hr, len(rr), _p(rr), _p(cols), _p(vals), _p(cnt))
        for k in range(len(rr)):
            out.append((cols[k, :cnt[k]].copy(), vals[k, :cnt[k]].copy()))
    return out


def dense_A(X, h: Hyper) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    n = X.shape[0]
    A = np.empty((n, n))
    hr, _keep = h.c()
    lib().orc_dense_A(n, _p(X), hr, _p(A))
    return A


# ----------------------------------------------------------------------------------------
# LML (Sec. 3): exact dense path
# ----------------------------------------------------------------------------------------
LOG2PI = math.log(2.0 * math.pi)


def lml_exact(X, y, h: Hyper) -> dict:
    """log p(y) = -1/2 y^T A^{-1} y - 1/2 log|A| - n/2 log(2 pi), A = K + sigma^2 I, by a dense
    Cholesky factorisation (library routine) of the brute-force A."""
    y = np.asarray(y, np.float64)
    A = dense_A(X, h)
    Lc = np.linalg.cholesky(A)
    logdet = 2.0 * float(np.sum(np.log(np.diag(Lc))))
    import scipy.linalg as sl
    a = sl.cho_solve((Lc, True), y)
    quad = float(y @ a)
    n = y.shape[0]
    return dict(lml=-0.5 * quad - 0.5 * logdet - 0.5 * n * LOG2PI, quad=quad, logdet=logdet, a=a,
                A=A, chol=Lc)


def cross_K(Xs, X, h: Hyper) -> np.ndarray:
    """K(X*, X) (n* x n) by brute force over every (test, training) pair."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    Xs = np.ascontiguousarray(np.asarray(Xs, np.float64).reshape(-1, h.d))
    Ks = np.empty((Xs.shape[0], X.shape[0]))
    hr, _keep = h.c()
    lib().orc_cross_K(Xs.shape[0], _p(Xs), X.shape[0], _p(X), hr, _p(Ks))
    return Ks


def prior_var(Xs, h: Hyper) -> np.ndarray:
    """k(x*, x*) for every test point (the kernel definition at zero distance)."""
    Xs = np.asarray(Xs, np.float64).reshape(-1, h.d)
    return np.array([kernel(h, x, x) for x in Xs])


def posterior(X, y, h: Hyper, Xs) -> dict:
    """Eq. 2 with zero prior mean and A = K + sigma^2 I in place of the paper's K (the same
    matrix whose inverse the LML of Sec. 3 uses):
        mean_i = k(X, x*_i)^T A^{-1} y,   var_i = k(x*_i, x*_i) - k(X, x*_i)^T A^{-1} k(X, x*_i)
    (the latent f* variance; the noisy y* adds sigma^2), by a dense Cholesky factorisation
    (library routine) of the brute-force A."""
    import scipy.linalg as sl
    y = np.asarray(y, np.float64)
    A = dense_A(X, h)
    Lc = np.linalg.cholesky(A)
    Ks = cross_K(Xs, X, h)
    a = sl.cho_solve((Lc, True), y)
    W = sl.solve_triangular(Lc, Ks.T, lower=True)          # L^{-1} k(X, x*)
    return dict(mean=Ks @ a, var=prior_var(Xs, h) - np.sum(W * W, axis=0), a=a, Ks=Ks, A=A)


def grad_contract(X, h: Hyper, csr: CSR, a, U=None, V=None, Wd=None) -> np.ndarray:
    """g_p = 1/2 sum_{(i,j) stored} W_ij dA_ij/dtheta_p (see gp2s_oracle.c)."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    a = np.ascontiguousarray(a, np.float64)
    m = 0 if U is None else U.shape[1]
    U = None if U is None else np.ascontiguousarray(U, np.float64)
    V = None if V is None else np.ascontiguousarray(V, np.float64)
    Wd = None if Wd is None else np.ascontiguousarray(Wd, np.float64)
    g = np.empty(h.nparams)
    hr, _keep = h.c()
    rc = lib().orc_grad_contract(csr.n, _p(csr.rowptr), _p(csr.col), _p(X), hr, _p(a), m, _p(U), _p(V),
                                 _p(Wd), _p(g))
    if rc != 0:
        raise MemoryError("oracle gradient contraction")
    return g


def grad_exact(X, y, h: Hyper) -> np.ndarray:
    """d LML / d theta = 1/2 a^T dA a - 1/2 tr(A^{-1} dA) with the exact dense inverse."""
    e = lml_exact(X, y, h)
    import scipy.linalg as sl
    n = e["A"].shape[0]
    Ainv = sl.cho_solve((e["chol"], True), np.eye(n))
    csr = assemble(X, h, "brute")
    return grad_contract(X, h, csr, e["a"], Wd=Ainv)


def lml_fd_grad(X, y, h: Hyper, step: float = 1e-5, richardson: bool = True) -> np.ndarray:
    """Central finite differences of the exact LML over theta (the pattern is rebuilt for
    every shifted theta).  With richardson=True the central differences at step and step/2 are
    combined as (4 D(step/2) - D(step)) / 3, which cancels their O(step^2) error term."""
    th = h.theta()

    def central(p, hs):
        tp, tm = th.copy(), th.copy()
        tp[p] += hs
        tm[p] -= hs
        return (lml_exact(X, y, h.with_theta(tp))["lml"] - lml_exact(X, y, h.with_theta(tm))["lml"]) / (2 * hs)

    g = np.empty_like(th)
    for p in range(th.size):
        g[p] = (4.0 * central(p, step / 2) - central(p, step)) / 3.0 if richardson else central(p, step)
    return g


# ----------------------------------------------------------------------------------------
# Krylov path: Jacobi-scaled CG, SLQ log-determinant, Hutchinson gradient
# ----------------------------------------------------------------------------------------
def cg(M: CSR, B, tol: float = 1e-10, maxit: int = 100000, kmax: int = 0):
    """CG on SPD M for the columns of B (x0 = 0).  Returns X, steps, alpha, beta
    (alpha/beta: k x kmax records of the first kmax iterations)."""
    B = np.ascontiguousarray(B, np.float64)
    one = B.ndim == 1
    Bm = B.reshape(M.n, -1)
    k = Bm.shape[1]
    Xm = np.empty_like(Bm)
    steps = np.zeros(k, np.int32)
    al = np.zeros((k, max(kmax, 1)))
    be = np.zeros((k, max(kmax, 1)))
    st = lib().orc_cg(M.n, _p(M.rowptr), _p(M.col), _p(M.val), k, _p(Bm), _p(Xm), tol, maxit, kmax,
                      _p(al) if kmax else None, _p(be) if kmax else None, _p(steps))
    if st < 0:
        raise MemoryError("oracle cg")
    return (Xm.ravel() if one else Xm), steps, al[:, :kmax], be[:, :kmax], st


def minres(M, b, tol: float = 1e-10, maxit: int = 100000):
    """MINRES (Paige & Saunders 1975) for a symmetric M x = b, x0 = 0 (the paper's solver for
    K^{-1} y, App. B.6).  M is a CSR or a callable v -> M v.  Lanczos with beta_1 v_1 = b:
        u = M v_k - beta_k v_{k-1},  alpha_k = v_k^T u,  u -= alpha_k v_k,  beta_{k+1} v_{k+1} = u,
    and the tridiagonal's QR factorisation by Givens rotations G_k = [[c_k, s_k], [-s_k, c_k]]:
        eps_k = s_{k-2} beta_k,  dbar_k = c_{k-2} beta_k,
        delta_k = c_{k-1} dbar_k + s_{k-1} alpha_k,  gbar_k = -s_{k-1} dbar_k + c_{k-1} alpha_k,
        gamma_k = |(gbar_k, beta_{k+1})|,  c_k = gbar_k / gamma_k,  s_k = beta_{k+1} / gamma_k,
        tau_k = c_k phibar_{k-1},  phibar_k = -s_k phibar_{k-1}   (phibar_0 = beta_1),
        w_k = (v_k - delta_k w_{k-1} - eps_k w_{k-2}) / gamma_k,  x_k = x_{k-1} + tau_k w_k,
    with |b - M x_k| = |phibar_k|.  Stops when |phibar_k| <= tol |b|.
    Returns x, iterations, and the residual norms |phibar_k| (k = 0, 1, ...)."""
    op = M.matmat if isinstance(M, CSR) else M
    b = np.asarray(b, np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    beta1 = float(np.linalg.norm(b))
    hist = [beta1]
    if beta1 == 0.0:
        return x, 0, hist
    v_prev = np.zeros(n)
    v = b / beta1
    beta = beta1
    c_km2, s_km2, c_km1, s_km1 = 1.0, 0.0, 1.0, 0.0
    w_km2 = np.zeros(n)
    w_km1 = np.zeros(n)
    phibar = beta1
    k = 0
    while k < maxit:
        k += 1
        u = op(v) - beta * v_prev
        alpha = float(v @ u)
        u = u - alpha * v
        beta_next = float(np.linalg.norm(u))
        eps = s_km2 * beta
        dbar = c_km2 * beta
        delta = c_km1 * dbar + s_km1 * alpha
        gbar = -s_km1 * dbar + c_km1 * alpha
        gamma = math.hypot(gbar, beta_next)
        c_k, s_k = gbar / gamma, beta_next / gamma
        tau = c_k * phibar
        phibar = -s_k * phibar
        w = (v - delta * w_km1 - eps * w_km2) / gamma
        x = x + tau * w
        hist.append(abs(phibar))
        if abs(phibar) <= tol * beta1 or beta_next == 0.0:
            break
        v_prev, v = v, u / beta_next
        beta = beta_next
        c_km2, s_km2, c_km1, s_km1 = c_km1, s_km1, c_k, s_k
        w_km2, w_km1 = w_km1, w
    return x, k, hist


def lanczos(M: CSR, Q1, steps: int):
    """Lanczos tridiagonals T_c (diag, off, order) for the unit columns of Q1."""
    Q1 = np.ascontiguousarray(Q1, np.float64).reshape(M.n, -1)
    k = Q1.shape[1]
    dg = np.zeros((k, steps))
    of = np.zeros((k, steps))
    ns = np.zeros(k, np.int32)
    lib().orc_lanczos(M.n, _p(M.rowptr), _p(M.col), _p(M.val), k, _p(Q1), steps, _p(dg), _p(of), _p(ns))
    return [(dg[c, :ns[c]].copy(), of[c, :max(ns[c] - 1, 0)].copy()) for c in range(k)]


def tridiag_from_cg(alpha, beta):
    """Lanczos tridiagonal from CG coefficients (the CG-Lanczos relation, Saad Sec. 6.7.3):
    T_00 = 1/alpha_0, T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j."""
    alpha = np.asarray(alpha, np.float64)
    beta = np.asarray(beta, np.float64)
    k = alpha.shape[0]
    dg = np.empty(k)
    dg[0] = 1.0 / alpha[0]
    for j in range(1, k):
        dg[j] = 1.0 / alpha[j] + beta[j - 1] / alpha[j - 1]
    off = np.sqrt(beta[:k - 1]) / alpha[:k - 1]
    return dg, off


def gauss_quadrature_log(dg, off) -> float:
    """sum_j tau_j^2 log(theta_j) over the eigenpairs of the tridiagonal T (a symmetric
    eigensolver from the library; tau_j = first component of the j-th unit eigenvector)."""
    k = len(dg)
    T = np.diag(np.asarray(dg, np.float64))
    if k > 1:
        T += np.diag(off, 1) + np.diag(off, -1)
    w, Z = np.linalg.eigh(T)
    return float(np.sum(Z[0, :] ** 2 * np.log(w)))


def lml_slq(X, y, h: Hyper, m: int = 64, k: int = 100, seed: int = 0, tol: float = 1e-10,
            maxit: int = 20000, csr: CSR | None = None, tridiag: str = "lanczos",
            grad: bool = True, lanczos_probes: int | None = None) -> dict:
    """LML with a = A^{-1} y by Jacobi-scaled CG and log|A| by stochastic Lanczos quadrature.

    With D = diag(A) and Ah = D^{-1/2} A D^{-1/2}:
      log|A| = sum_i log D_ii + log|Ah|,
      log|Ah| ~= (n/m) sum_s sum_j tau_sj^2 log theta_sj   (q1 = z_s / sqrt(n), k Lanczos steps),
      tr(A^{-1} dA) ~= (1/m) sum_s u_s^T dA v_s,  v_s = D^{-1/2} z_s,  u_s = D^{-1/2} Ah^{-1} z_s.
    The probes z_s are the SplitMix64 Rademacher vectors of ``probes``.
    tridiag: 'lanczos' (explicit three-term Lanczos) or 'cg' (the CG-Lanczos relation applied
    to the recorded CG coefficients of the probe columns).
    """
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, h.d))
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    if csr is None:
        csr = assemble(X, h)
    D = csr.diag()
    s = 1.0 / np.sqrt(D)
    Ah = csr.scaled(s)
    Z = probes(n, m, seed)
    B = np.concatenate([(s * y)[:, None], Z], axis=1)
    Xs, steps, al, be, st = cg(Ah, B, tol=tol, maxit=maxit, kmax=k)
    a = s * Xs[:, 0]
    quad = float(y @ a)
    mp = m if lanczos_probes is None else min(m, lanczos_probes)
    gam = np.empty(mp)
    if tridiag == "lanczos":
        Ts = lanczos(Ah, Z[:, :mp] / math.sqrt(n), k)
        for c in range(mp):
            gam[c] = gauss_quadrature_log(*Ts[c])
    else:
        for c in range(mp):
            kk = min(k, int(steps[1 + c]))
            gam[c] = gauss_quadrature_log(*tridiag_from_cg(al[1 + c, :kk], be[1 + c, :kk]))
    logdet_hat = n * float(np.mean(gam))
    logdet = float(np.sum(np.log(D))) + logdet_hat
    res = y - csr.matmat(a)
    out = dict(lml=-0.5 * quad - 0.5 * logdet - 0.5 * n * LOG2PI, quad=quad, logdet=logdet,
               logdet_diag=float(np.sum(np.log(D))), probe_quadrature=n * gam, a=a, steps=steps,
               relres=float(np.linalg.norm(res) / np.linalg.norm(y)), cg_status=st, csr=csr, D=D)
    if grad:
        U = s[:, None] * Xs[:, 1:]
        V = s[:, None] * Z
        out["grad"] = grad_contract(X, h, csr, a, U=U, V=V)
        out["U"], out["V"] = U, V
    return out


def mcmc(logpost, theta0, block, step, lower, upper, normals, uniforms):
    """Block Metropolis-Hastings (App. D): for every iteration t and every block b in order,
        theta' = theta + step * normals[t]   on the components p with block[p] == b,
    rejected outright if any component leaves [lower, upper] (the flat prior's support), else
    accepted when log(uniforms[t, b]) < logpost(theta') - logpost(theta).  Components with
    block -1 never move.  logpost(theta) is the log-density (the LML for a flat prior).
    Returns the chain (iters x (P + 1): theta after the sweep, then its log-density) and the
    acceptance flags (iters x nblocks)."""
    theta = np.array(theta0, np.float64)
    block = np.asarray(block)
    step = np.asarray(step, np.float64)
    normals = np.asarray(normals, np.float64)
    uniforms = np.asarray(uniforms, np.float64)
    iters, nblocks = uniforms.shape
    cur = float(logpost(theta))
    chain = np.empty((iters, theta.size + 1))
    acc = np.zeros((iters, nblocks), np.int32)
    for t in range(iters):
        for b in range(nblocks):
            sel = block == b
            if not np.any(sel):
                continue                      # a block without members proposes nothing
            prop = theta.copy()
            prop[sel] = theta[sel] + step[sel] * normals[t, sel]
            if np.any(prop < lower) or np.any(prop > upper):
                continue
            new = float(logpost(prop))
            logu = math.log(uniforms[t, b]) if uniforms[t, b] > 0.0 else -math.inf
            if logu < new - cur:
                theta, cur = prop, new
                acc[t, b] = 1
        chain[t, :-1] = theta
        chain[t, -1] = cur
    return chain, acc


def num_threads() -> int:
    return int(lib().orc_num_threads())
