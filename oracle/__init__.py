"""Plain FP64 CPU oracle for the improved seed method (ctypes over seed_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product path (the CUDA
library and its binding) never imports this package, and this package never
imports the product path; the two share only the seeded input generators.

Every function here is a thin marshalling layer; the arithmetic is in
``seed_oracle.c`` (see its header for the passage each routine follows),
except ``adjoint_reference``, which assembles a loss and its gradients from
the oracle's CG solves and operator applies with numpy inner products.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seed_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None          # the library the functions below call
_libs = {}           # loaded builds by path

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 4: "ENOTSPD", 5: "ENOTCONV"}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile seed_oracle.c into liboracle.so (gcc, -O2, no FMA contraction),
    or with omp=True into liboracle_omp.so: the same source with OpenMP on its
    independent loops (bit-identical results; for timing on all host cores)."""
    lib = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + ".%d.tmp" % os.getpid()
        extra = ["-fopenmp", "-DORC_OMP"] if omp else []
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + extra +
                       ["-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, lib)
    return lib


def _open(path):
    if path not in _libs:
        lib = C.CDLL(path)
        _declare(lib)
        _libs[path] = lib
    return _libs[path]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _open(_LIB)
    return _lib


def set_threads(k: int) -> int:
    """Run the oracle on k host threads from now on (k <= 1: the one-thread
    build, k > 1: the OpenMP build, same results bit for bit).  Returns the
    number of threads the active build uses."""
    global _lib
    with _lock:
        if k <= 1:
            build()
            _lib = _open(_LIB)
        else:
            build(omp=True)
            _lib = _open(_LIB_OMP)
        return int(_lib.orc_threads(int(k)))


class _Op(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("n", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p),
                ("dims", C.c_int32 * 4), ("kappa", C.c_double), ("bc_t", C.c_int32),
                ("pad2_", C.c_int32), ("links", C.c_void_p), ("dense", C.c_void_p)]


class _SeedParams(C.Structure):
    _fields_ = [("m_max", C.c_int32), ("reorth_freq", C.c_int32), ("reorth_passes", C.c_int32),
                ("extra_iters", C.c_int32), ("x0_zero", C.c_int32), ("pad_", C.c_int32),
                ("tol", C.c_double), ("breakdown_rel", C.c_double)]


class _SeedOut(C.Structure):
    _fields_ = [("iters", C.c_int32), ("mvps", C.c_int32), ("converged_at", C.c_int32),
                ("breakdown", C.c_int32), ("rho", C.c_double), ("bnorm1", C.c_double)]


class _CgOut(C.Structure):
    _fields_ = [("iters", C.c_int32), ("mvps", C.c_int32), ("restarts", C.c_int32),
                ("converged", C.c_int32), ("true_relres", C.c_double)]


def _declare(lib):
    P = C.c_void_p
    lib.orc_threads.argtypes = [C.c_int]
    lib.orc_threads.restype = C.c_int
    lib.orc_csr_apply.argtypes = [C.c_int64, P, P, P, P, P]
    lib.orc_wilson_neighbors.argtypes = [P, P]
    lib.orc_wilson_dslash.argtypes = [P, C.c_double, C.c_int32, C.c_int32, P, P, P]
    lib.orc_seed_multiple.argtypes = [C.POINTER(_Op), C.c_int32, P, P, C.c_double, C.c_int32, P, P, P, P]
    lib.orc_seed_multiple.restype = C.c_int
    lib.orc_wilson_dA_dkappa.argtypes = [P, C.c_double, C.c_int32, P, P, P]
    lib.orc_wilson_dA_dkappa.restype = C.c_int
    lib.orc_op_apply.argtypes = [C.POINTER(_Op), P, P]
    lib.orc_op_apply.restype = C.c_int
    lib.orc_seed_first.argtypes = [C.POINTER(_Op), C.c_int32, P, P, C.POINTER(_SeedParams),
                                   C.POINTER(_SeedOut), P, P, P, P]
    lib.orc_seed_first.restype = C.c_int
    lib.orc_cg.argtypes = [C.POINTER(_Op), P, P, C.c_double, C.c_int32, C.c_int32, C.POINTER(_CgOut)]
    lib.orc_cg.restype = C.c_int
    lib.orc_related_project.argtypes = [C.c_int64, P, P, P, P]
    lib.orc_cholesky_solve.argtypes = [C.c_int64, P, P, P]
    lib.orc_cholesky_solve.restype = C.c_int
    lib.orc_tridiag_eigs.argtypes = [C.c_int32, P, P, P]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _zvec(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.complex128)


class Operator:
    """An SPD/HPD operator the oracle can apply: CSR (real), Wilson normal
    operator A = D^H D, or a dense Hermitian matrix."""

    def __init__(self, kind: int, n: int, keep: tuple, **fields):
        self._keep = keep
        self.kind = kind
        self.n = int(n)
        self.s = _Op()
        self.s.kind = kind
        self.s.n = self.n
        for k, v in fields.items():
            setattr(self.s, k, v)

    @classmethod
    def csr(cls, row_ptr, col_idx, vals):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        va = np.ascontiguousarray(vals, dtype=np.float64)
        return cls(0, rp.shape[0] - 1, (rp, ci, va), row_ptr=_p(rp).value, col_idx=_p(ci).value,
                   vals=_p(va).value)

    @classmethod
    def wilson(cls, dims, kappa: float, links, bc_t: int = 0):
        lk = np.ascontiguousarray(links, dtype=np.complex128)
        vol = int(np.prod(dims))
        assert lk.size == 4 * vol * 9
        op = cls(1, 12 * vol, (lk,), kappa=float(kappa), bc_t=int(bc_t), links=_p(lk).value)
        for k in range(4):
            op.s.dims[k] = int(dims[k])
        op.dims = tuple(int(d) for d in dims)
        op.kappa = float(kappa)
        op.bc_t = int(bc_t)
        op.links = lk
        return op

    @classmethod
    def dense(cls, A):
        a = np.ascontiguousarray(A, dtype=np.complex128)
        return cls(2, a.shape[0], (a,), dense=_p(a).value)

    def apply(self, x) -> np.ndarray:
        x = _zvec(x)
        y = np.empty(self.n, dtype=np.complex128)
        rc = _load().orc_op_apply(C.byref(self.s), _p(x), _p(y))
        assert rc == 0
        return y

    def to_dense(self) -> np.ndarray:
        """Dense matrix by applying the operator to unit vectors (small n only)."""
        n = self.n
        M = np.empty((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for c in range(n):
            e[c] = 1.0
            M[:, c] = self.apply(e)
            e[c] = 0.0
        return M


def wilson_dslash(dims, kappa, bc_t, sign, links, x) -> np.ndarray:
    """D x (sign=+1) or D^H x (sign=-1) for the Wilson-Dirac operator."""
    d = np.asarray(dims, dtype=np.int32)
    lk = np.ascontiguousarray(links, dtype=np.complex128)
    x = _zvec(x)
    y = np.empty_like(x)
    _load().orc_wilson_dslash(_p(d), float(kappa), int(bc_t), int(sign), _p(lk), _p(x), _p(y))
    return y


def wilson_dA_dkappa(dims, kappa, bc_t, links, x) -> np.ndarray:
    """(dA/dkappa) x for the Wilson normal operator A = D^H D."""
    d = np.asarray(dims, dtype=np.int32)
    lk = np.ascontiguousarray(links, dtype=np.complex128)
    x = _zvec(x)
    y = np.empty_like(x)
    rc = _load().orc_wilson_dA_dkappa(_p(d), float(kappa), int(bc_t), _p(lk), _p(x), _p(y))
    if rc != 0:
        raise MemoryError("orc_wilson_dA_dkappa")
    return y


def adjoint_reference(dims, kappa, links, B, T, bc_t: int = 0, tol: float = 1e-12) -> dict:
    """Loss L = sum_j ||x_j - t_j||^2 with x_j = A^{-1} b_j (A = D^H D) and its
    gradients by the chain rule, from CG solves to ``tol``:
      dL/db_j = lambda_j = A^{-1} g_j,  g_j = 2 (x_j - t_j)   (A Hermitian; the
        conjugate-Wirtinger convention, dL = Re <dL/db, db>),
      dL/dkappa = -sum_j Re <lambda_j, (dA/dkappa) x_j>.
    Returns L, X, Lambda (= dL/dB) and dL/dkappa."""
    op = Operator.wilson(dims, kappa, links, bc_t=bc_t)
    B = np.asfortranarray(B, dtype=np.complex128)
    T = np.asfortranarray(T, dtype=np.complex128)
    n, p = B.shape
    X = np.zeros((n, p), dtype=np.complex128, order="F")
    Lam = np.zeros((n, p), dtype=np.complex128, order="F")
    loss, gk = 0.0, 0.0
    for j in range(p):
        X[:, j] = cg(op, B[:, j], np.zeros(n, dtype=np.complex128), tol=tol)["x"]
        d = X[:, j] - T[:, j]
        loss += float(np.vdot(d, d).real)
        Lam[:, j] = cg(op, 2.0 * d, np.zeros(n, dtype=np.complex128), tol=tol)["x"]
        gk -= float(np.vdot(Lam[:, j], wilson_dA_dkappa(dims, kappa, bc_t, links, X[:, j])).real)
    return dict(loss=loss, X=X, grad_B=Lam, grad_kappa=gk)


def wilson_neighbors(dims) -> np.ndarray:
    d = np.asarray(dims, dtype=np.int32)
    vol = int(np.prod(d))
    out = np.empty(8 * vol, dtype=np.int32)
    _load().orc_wilson_neighbors(_p(d), _p(out))
    return out.reshape(vol, 8)


def seed_first(op: Operator, B, X0=None, *, m_max: int, reorth_freq: int = 0, reorth_passes: int = 2,
               tol: float = 1e-8, extra_iters: int = 0, breakdown_rel: float = 1e-14,
               keep_V: bool = False) -> dict:
    """The Sec. 3 seed solve (Lanczos form of CG, periodic reorthogonalization,
    seeding of the other columns) on all columns of B (n x nrhs)."""
    B = np.asfortranarray(B, dtype=np.complex128)
    n, nrhs = B.shape
    assert n == op.n
    X = np.zeros((n, nrhs), dtype=np.complex128, order="F") if X0 is None else \
        np.array(X0, dtype=np.complex128, order="F", copy=True)
    prm = _SeedParams(m_max=m_max, reorth_freq=reorth_freq, reorth_passes=reorth_passes,
                      extra_iters=extra_iters, x0_zero=1 if X0 is None else 0, tol=tol,
                      breakdown_rel=breakdown_rel)
    out = _SeedOut()
    alpha = np.zeros(m_max, dtype=np.float64)
    beta = np.zeros(m_max + 1, dtype=np.float64)
    rho = np.zeros(m_max, dtype=np.float64)
    V = np.zeros((n, m_max + 1), dtype=np.complex128, order="F") if keep_V else None
    rc = _load().orc_seed_first(C.byref(op.s), nrhs, _p(B), _p(X), C.byref(prm), C.byref(out),
                                _p(alpha), _p(beta), _p(rho), _p(V) if keep_V else None)
    it = out.iters
    res = dict(status=STATUS.get(rc, rc), X=X, iters=it, mvps=out.mvps, converged_at=out.converged_at,
               breakdown=bool(out.breakdown), rho=out.rho, bnorm1=out.bnorm1,
               alpha=alpha[:it].copy(), beta=beta[:it + 1].copy(), rho_hist=rho[:it].copy())
    if keep_V:
        res["V"] = V[:, :it].copy()
    return res


def cg(op: Operator, b, x0, *, tol: float = 1e-8, maxit: int = 100000, max_restarts: int = 3) -> dict:
    """Plain CG from x0 (see seed_oracle.c orc_cg)."""
    b = _zvec(b)
    x = np.array(x0, dtype=np.complex128, copy=True)
    out = _CgOut()
    rc = _load().orc_cg(C.byref(op.s), _p(b), _p(x), float(tol), int(maxit), int(max_restarts),
                        C.byref(out))
    return dict(status=STATUS.get(rc, rc), x=x, iters=out.iters, mvps=out.mvps,
                restarts=out.restarts, converged=bool(out.converged), true_relres=out.true_relres)


def seed_solve_all(op: Operator, B, *, m_max: int, reorth_freq: int, reorth_passes: int = 2,
                   tol_seed: float = 1e-12, tol_rest: float = 1e-8, extra_iters: int = 0,
                   breakdown_rel: float = 1e-14, maxit_rest: int = 100000, rest_cols=None) -> dict:
    """Single seeding (Sec. 2.2) with the Sec. 3 seed solve, then plain CG on
    the seeded systems 2..nrhs (or the subset ``rest_cols``)."""
    s = seed_first(op, B, m_max=m_max, reorth_freq=reorth_freq, reorth_passes=reorth_passes,
                   tol=tol_seed, extra_iters=extra_iters, breakdown_rel=breakdown_rel)
    X = s["X"]
    B = np.asfortranarray(B, dtype=np.complex128)
    rest = []
    cols = range(1, B.shape[1]) if rest_cols is None else rest_cols
    X_seeded = X.copy()
    for j in cols:
        r = cg(op, B[:, j], X[:, j], tol=tol_rest, maxit=maxit_rest)
        X[:, j] = r["x"]
        rest.append(r)
    return dict(seed=s, rest=rest, X=X, X_seeded=X_seeded)


def seed_multiple(op: Operator, B, *, tol: float = 1e-8, maxit: int = 100000) -> dict:
    """Multiple seeding, the seed CG that Sec. 2.1 compares against (see orc_seed_multiple)."""
    B = np.asfortranarray(B, dtype=np.complex128)
    n, p = B.shape
    X = np.zeros((n, p), dtype=np.complex128, order="F")
    Xs = np.zeros((n, p), dtype=np.complex128, order="F")
    iters = np.zeros(p, dtype=np.int32)
    mvps = np.zeros(p, dtype=np.int32)
    relres = np.zeros(p, dtype=np.float64)
    rc = _load().orc_seed_multiple(C.byref(op.s), p, _p(B), _p(X), float(tol), int(maxit), _p(iters), _p(mvps),
                                   _p(relres), _p(Xs))
    return dict(status=STATUS.get(rc, rc), X=X, X_seeded=Xs, iters=iters.tolist(), mvps=mvps.tolist(),
                relres=relres.tolist())


def seed_solve_related(op: Operator, B, *, m_max: int, reorth_freq: int, reorth_passes: int = 2,
                       tol_seed: float = 1e-12, tol_rest: float = 1e-8, maxit_rest: int = 100000) -> dict:
    """Sec. 2.3 (single seeding for related right-hand sides): system 1 by the
    Sec. 3 seed solve (no initial guesses), then: project the
    remaining systems over x^1 (x^1_bcg = 0, r^1_bcg = b^1); for j = 2..nrhs run
    CG on system j from its current approximation and project the later
    systems over that CG's correction x^j - x^j_bcg (orc_related_project)."""
    s = seed_first(op, B, m_max=m_max, reorth_freq=reorth_freq, reorth_passes=reorth_passes, tol=tol_seed)
    B = np.asfortranarray(B, dtype=np.complex128)
    X = s["X"]
    n, p = B.shape
    R = np.zeros((n, p), dtype=np.complex128, order="F")
    for i in range(1, p):
        R[:, i] = B[:, i] - op.apply(X[:, i])
    for i in range(1, p):
        X[:, i], R[:, i] = related_project(X[:, 0], B[:, 0], X[:, i], R[:, i])
    rest = []
    for j in range(1, p):
        xb, rb = X[:, j].copy(), R[:, j].copy()
        r = cg(op, B[:, j], X[:, j], tol=tol_rest, maxit=maxit_rest)
        X[:, j] = r["x"]
        rest.append(r)
        xcg = X[:, j] - xb
        for i in range(j + 1, p):
            X[:, i], R[:, i] = related_project(xcg, rb, X[:, i], R[:, i])
    return dict(seed=s, rest=rest, X=X)


def related_project(x_cg, r_bcg, x_bpr, r_bpr):
    """The Sec. 2.3 projection over one CG correction, on copies; returns (x_new, r_new)."""
    x_cg = _zvec(x_cg)
    r_bcg = _zvec(r_bcg)
    x = np.array(x_bpr, dtype=np.complex128, copy=True)
    r = np.array(r_bpr, dtype=np.complex128, copy=True)
    _load().orc_related_project(x.shape[0], _p(x_cg), _p(r_bcg), _p(x), _p(r))
    return x, r


def cholesky_solve(A, b) -> np.ndarray:
    a = np.ascontiguousarray(A, dtype=np.complex128)
    b = _zvec(b)
    x = np.empty_like(b)
    rc = _load().orc_cholesky_solve(a.shape[0], _p(a), _p(b), _p(x))
    if rc != 0:
        raise ValueError("matrix not positive definite (%s)" % STATUS.get(rc, rc))
    return x


def tridiag_eigs(alpha, beta_off) -> np.ndarray:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta_off, dtype=np.float64)
    m = a.shape[0]
    assert b.shape[0] == m - 1
    e = np.empty(m, dtype=np.float64)
    _load().orc_tridiag_eigs(m, _p(a), _p(b) if m > 1 else None, _p(e))
    return e
