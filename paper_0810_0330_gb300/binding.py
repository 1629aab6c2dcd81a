"""Thin Python binding of the C ABI in include/seed.h (ctypes).

Argument marshalling only: every step of the solve runs in the CUDA library
libseed.so.  PyTorch supplies device memory and the current stream.  If the
library has not been built, loading fails with an error; there is no other
implementation to fall back on.

Blocks of vectors are torch tensors viewed as column-major n x ncols: either
a 1-d tensor of length n, or a 2-d tensor of shape (n, ncols) with stride
(1, ld), e.g. ``Bt.t()`` for a contiguous (ncols, n) tensor ``Bt``.  CSR
operators use float64, the Wilson operator complex128.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libseed.so")
_lib = None
_lock = threading.Lock()

SEED_OK, SEED_EINVAL, SEED_ENOMEM, SEED_ECUDA, SEED_ENOTSPD, SEED_ENOTCONV, SEED_ESTATE, SEED_ETIMEOUT = range(8)
SEED_F64, SEED_C128, SEED_F32, SEED_C64 = range(4)
STATUS_NAMES = ["SEED_OK", "SEED_EINVAL", "SEED_ENOMEM", "SEED_ECUDA", "SEED_ENOTSPD", "SEED_ENOTCONV",
                "SEED_ESTATE", "SEED_ETIMEOUT"]

# symbols declared in include/seed.h
EXPORTS = ["seed_abi_version", "seed_params_default", "seed_create_csr", "seed_create_wilson",
           "seed_solve_first", "seed_project", "seed_solve_rest", "seed_apply", "seed_wilson_neighbors",
           "seed_get_tridiag", "seed_get_basis", "seed_get_stats", "seed_time_operator", "seed_last_error",
           "seed_destroy", "seed_wilson_apply_noalloc", "seed_solve_cg", "seed_grad_kappa", "seed_solve_related",
           "seed_batch_solve", "seed_solve_multiple", "seed_inject_alloc_failure", "seed_check_barrier_timeout",
           "seed_time_fma", "seed_block_products", "seed_time_fp64_paths"]


class SeedError(RuntimeError):
    """A status other than SEED_OK; `info` holds the per-system seed_info of a
    failed solve call (None for other calls)."""

    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        self.info = None
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s (%s)" % (where, name, msg))


class seed_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("vals", C.c_void_p)]


class seed_wilson(C.Structure):
    _fields_ = [("dims", C.c_int32 * 4), ("kappa", C.c_double), ("bc_t", C.c_int32), ("reserved", C.c_int32),
                ("links", C.c_void_p)]


class seed_params(C.Structure):
    _fields_ = [("m_max", C.c_int32), ("reorth_freq", C.c_int32), ("reorth_passes", C.c_int32),
                ("extra_iters", C.c_int32), ("keep_basis", C.c_int32), ("x0_zero", C.c_int32),
                ("maxit_rest", C.c_int32), ("max_restarts", C.c_int32), ("tol_seed", C.c_double),
                ("tol_rest", C.c_double), ("breakdown_rel", C.c_double), ("kernel_path", C.c_int32),
                ("precision", C.c_int32), ("autotune", C.c_int32), ("reliable_delta", C.c_double)]


class seed_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("mvps", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("est_relres", C.c_double), ("true_relres", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class seed_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("graph_launches", C.c_int64), ("mvps", C.c_int64),
                ("reorth_events", C.c_int64), ("ms_seed", C.c_double), ("ms_project", C.c_double),
                ("ms_rest", C.c_double), ("csr_tpr", C.c_int32), ("csr_block", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load libseed.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libseed.so is not built (run __graft_entry__.build() or "
                                   "python -m paper_0810_0330_gb300.build)")
            L = C.CDLL(LIB_PATH)
            P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
            L.seed_abi_version.restype = I32
            L.seed_params_default.argtypes = [C.POINTER(seed_params)]
            L.seed_create_csr.argtypes = [C.POINTER(P), C.POINTER(seed_csr), C.POINTER(seed_params), P]
            L.seed_create_wilson.argtypes = [C.POINTER(P), C.POINTER(seed_wilson), C.POINTER(seed_params), P]
            L.seed_solve_first.argtypes = [P, P, I64, P, I64, I32, P]
            L.seed_solve_rest.argtypes = [P, P, I64, P, I64, I32, P]
            L.seed_project.argtypes = [P, P, I64, P, I64, I32]
            L.seed_apply.argtypes = [P, I32, P, I64, P, I64, I32]
            L.seed_wilson_neighbors.argtypes = [P, P, P]
            L.seed_get_tridiag.argtypes = [P, P, P, I32, C.POINTER(I32)]
            L.seed_get_basis.argtypes = [P, P, I32]
            L.seed_get_stats.argtypes = [P, C.POINTER(seed_stats)]
            L.seed_time_operator.argtypes = [P, I32, I32, I32, C.POINTER(C.c_double)]
            L.seed_wilson_apply_noalloc.argtypes = [C.POINTER(seed_wilson), P, I64, P, I64, I32, P]
            L.seed_solve_cg.argtypes = [P, P, I64, P, I64, I32, P]
            L.seed_solve_related.argtypes = [P, P, I64, P, I64, I32, P]
            L.seed_solve_multiple.argtypes = [P, P, I64, P, I64, I32, P]
            L.seed_batch_solve.argtypes = [P, P, P, P, P, P, I32, I32, P]
            L.seed_grad_kappa.argtypes = [P, P, I64, P, I64, I32, C.POINTER(C.c_double)]
            L.seed_inject_alloc_failure.argtypes = [I32]
            L.seed_inject_alloc_failure.restype = I32
            L.seed_check_barrier_timeout.argtypes = [P, C.POINTER(I32), C.POINTER(C.c_double)]
            L.seed_time_fma.argtypes = [I32, P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.seed_block_products.argtypes = [P, I64, I32, P, I64, I32, I64, P, I32, C.POINTER(C.c_double), P]
            L.seed_time_fp64_paths.argtypes = [P, C.POINTER(C.c_double)]
            L.seed_last_error.argtypes = [P]
            L.seed_last_error.restype = C.c_char_p
            L.seed_destroy.argtypes = [P]
            L.seed_destroy.restype = None
            for name in EXPORTS:
                if name not in ("seed_last_error", "seed_destroy", "seed_abi_version", "seed_inject_alloc_failure"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status: int, where: str, ctx=None):
    if status != SEED_OK:
        msg = lib().seed_last_error(ctx)
        raise SeedError(status, where, msg.decode() if msg else "")


def _check_info(status: int, where: str, ctx, info):
    try:
        _check(status, where, ctx)
    except SeedError as e:
        e.info = [i.as_dict() for i in info]
        raise


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _block(t: torch.Tensor, n: int, name: str):
    """(pointer, ld, ncols) of a column-major block."""
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dim() == 1:
        if t.shape[0] != n or t.stride(0) != 1:
            raise ValueError("%s: expected a contiguous vector of length %d" % (name, n))
        return t.data_ptr(), n, 1
    if t.dim() != 2 or t.shape[0] != n or (t.shape[1] > 1 and t.stride(0) != 1) or (t.shape[1] == 1 and t.stride(0) != 1):
        raise ValueError("%s: expected shape (n, ncols) with stride (1, ld)" % name)
    ld = t.stride(1) if t.shape[1] > 1 else n
    return t.data_ptr(), ld, t.shape[1]


class Context:
    """An opaque seed_ctx* plus references that keep the operator arrays alive."""

    def __init__(self, handle: int, n: int, dtype: torch.dtype, keep: tuple):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.dtype = dtype
        self._keep = keep

    def __del__(self):
        try:
            seed_destroy(self)
        except Exception:
            pass


def seed_params_default(**overrides) -> seed_params:
    p = seed_params()
    _check(lib().seed_params_default(C.byref(p)), "seed_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def seed_create_csr(row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor, params: seed_params,
                    stream=None) -> Context:
    assert row_ptr.dtype == torch.int32 and col_idx.dtype == torch.int32 and vals.dtype == torch.float64
    rp, ci, va = row_ptr.contiguous(), col_idx.contiguous(), vals.contiguous()
    a = seed_csr(n=rp.shape[0] - 1, nnz=ci.shape[0], row_ptr=rp.data_ptr(), col_idx=ci.data_ptr(),
                 vals=va.data_ptr())
    h = C.c_void_p()
    _check(lib().seed_create_csr(C.byref(h), C.byref(a), C.byref(params), _stream(stream)), "seed_create_csr")
    return Context(h.value, a.n, torch.float64, (rp, ci, va))


def seed_create_wilson(dims, kappa: float, links: torch.Tensor, params: seed_params, bc_t: int = 0,
                       stream=None) -> Context:
    assert links.dtype == torch.complex128
    lk = links.contiguous()
    a = seed_wilson(kappa=float(kappa), bc_t=int(bc_t), reserved=0, links=lk.data_ptr())
    for k in range(4):
        a.dims[k] = int(dims[k])
    h = C.c_void_p()
    _check(lib().seed_create_wilson(C.byref(h), C.byref(a), C.byref(params), _stream(stream)),
           "seed_create_wilson")
    vol = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    return Context(h.value, 12 * vol, torch.complex128, (lk,))


def _infos(nrhs):
    return (seed_info * nrhs)()


def seed_solve_first(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    info = _infos(nb)
    _check_info(lib().seed_solve_first(ctx.handle, pb, ldb, px, ldx, nb, info), "seed_solve_first", ctx.handle, info)
    return [i.as_dict() for i in info]


def seed_solve_rest(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    info = _infos(nb)
    _check_info(lib().seed_solve_rest(ctx.handle, pb, ldb, px, ldx, nb, info), "seed_solve_rest", ctx.handle, info)
    return [i.as_dict() for i in info]


def seed_batch_solve(ctxs, Bs, Xs, workers: int = 0):
    """seed_solve_first + seed_solve_rest for every (ctx, B, X), all problems
    concurrently; returns one info list per problem."""
    k = len(ctxs)
    if not (len(Bs) == len(Xs) == k):
        raise ValueError("ctxs, Bs and Xs must have the same length")
    hs = (C.c_void_p * k)(*[c.handle.value for c in ctxs])
    pb, ldb, px, ldx, nr = (C.c_void_p * k)(), (C.c_int64 * k)(), (C.c_void_p * k)(), (C.c_int64 * k)(), \
        (C.c_int32 * k)()
    infos = []
    for i, (c, B, X) in enumerate(zip(ctxs, Bs, Xs)):
        b, lb, nb = _block(B, c.n, "B")
        x, lx, nx = _block(X, c.n, "X")
        if nb != nx:
            raise ValueError("B and X must have the same number of columns (problem %d)" % i)
        pb[i], ldb[i], px[i], ldx[i], nr[i] = b, lb, x, lx, nb
        infos.append(_infos(nb))
    ip = (C.c_void_p * k)(*[C.cast(inf, C.c_void_p).value for inf in infos])
    _check(lib().seed_batch_solve(hs, pb, ldb, px, ldx, nr, int(k), int(workers), ip), "seed_batch_solve")
    return [[i.as_dict() for i in inf] for inf in infos]


def seed_solve_multiple(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    """Multiple seeding (the Sec. 2.1 comparison method): all systems, in order."""
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    info = _infos(nb)
    _check(lib().seed_solve_multiple(ctx.handle, pb, ldb, px, ldx, nb, info), "seed_solve_multiple", ctx.handle)
    return [i.as_dict() for i in info]


def seed_solve_related(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    """Sec. 2.3 (related right-hand sides) after seed_solve_first: systems 2.. solved one after another,
    each later system projected over every CG correction."""
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    info = _infos(nb)
    _check(lib().seed_solve_related(ctx.handle, pb, ldb, px, ldx, nb, info), "seed_solve_related", ctx.handle)
    return [i.as_dict() for i in info]


def seed_solve_cg(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    """CG on every column of B from the guesses in X (X is overwritten with the solutions)."""
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    info = _infos(nb)
    _check(lib().seed_solve_cg(ctx.handle, pb, ldb, px, ldx, nb, info), "seed_solve_cg", ctx.handle)
    return [i.as_dict() for i in info]


def seed_grad_kappa(ctx: Context, Lam: torch.Tensor, X: torch.Tensor) -> float:
    """sum_j Re <Lam_j, (dA/dkappa) X_j> for a Wilson context."""
    pl, ldl, nl = _block(Lam, ctx.n, "Lambda")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nl != nx:
        raise ValueError("Lambda and X must have the same number of columns")
    out = C.c_double()
    _check(lib().seed_grad_kappa(ctx.handle, pl, ldl, px, ldx, nl, C.byref(out)), "seed_grad_kappa", ctx.handle)
    return out.value


def seed_project(ctx: Context, B: torch.Tensor, X: torch.Tensor):
    pb, ldb, nb = _block(B, ctx.n, "B")
    px, ldx, nx = _block(X, ctx.n, "X")
    if nb != nx:
        raise ValueError("B and X must have the same number of columns")
    _check(lib().seed_project(ctx.handle, pb, ldb, px, ldx, nb), "seed_project", ctx.handle)


def wilson_tiled_length(n: int) -> int:
    """Column length of the tiled FP32 layout (seed_apply ops 6, 7) for n = 12 * sites."""
    return 384 * ((n // 12 + 31) // 32)


def seed_apply(ctx: Context, op: int, X: torch.Tensor, Y: torch.Tensor):
    length = wilson_tiled_length(ctx.n) if op in (6, 7) else ctx.n
    px, ldx, nx = _block(X, length, "X")
    py, ldy, ny = _block(Y, length, "Y")
    if nx != ny:
        raise ValueError("X and Y must have the same number of columns")
    _check(lib().seed_apply(ctx.handle, int(op), px, ldx, py, ldy, nx), "seed_apply", ctx.handle)


def seed_inject_alloc_failure(k: int) -> int:
    """Fail the k-th device allocation from now (k = 1: the next); k <= 0 disarms.
    Returns the previous countdown."""
    return int(lib().seed_inject_alloc_failure(int(k)))


def seed_check_barrier_timeout(stream=None):
    """(timed_out, ms): the persistent kernels' barrier wait run against a
    barrier that cannot complete (about 2 s)."""
    t, ms = C.c_int32(), C.c_double()
    _check(lib().seed_check_barrier_timeout(_stream(stream), C.byref(t), C.byref(ms)), "seed_check_barrier_timeout")
    return bool(t.value), ms.value


def seed_wilson_neighbors(dims, out: torch.Tensor, stream=None):
    assert out.dtype == torch.int32 and out.is_cuda and out.is_contiguous()
    d = (C.c_int32 * 4)(*[int(x) for x in dims])
    _check(lib().seed_wilson_neighbors(d, out.data_ptr(), _stream(stream)), "seed_wilson_neighbors")


def seed_get_tridiag(ctx: Context):
    """(alpha_1..alpha_m, beta_0..beta_m) of the last seed solve, as numpy arrays."""
    import numpy as np
    m = C.c_int32()
    _check(lib().seed_get_tridiag(ctx.handle, None, None, 0, C.byref(m)), "seed_get_tridiag", ctx.handle)
    a = np.zeros(max(m.value, 1), dtype=np.float64)
    b = np.zeros(m.value + 1, dtype=np.float64)
    _check(lib().seed_get_tridiag(ctx.handle, a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
                                  m.value + 1, C.byref(m)), "seed_get_tridiag", ctx.handle)
    return a[:m.value], b


def seed_get_basis(ctx: Context, ncols: int):
    import numpy as np
    dt = np.float64 if ctx.dtype == torch.float64 else np.complex128
    V = np.zeros((ncols, ctx.n), dtype=dt)
    _check(lib().seed_get_basis(ctx.handle, V.ctypes.data_as(C.c_void_p), int(ncols)), "seed_get_basis",
           ctx.handle)
    return V.T


def seed_get_stats(ctx: Context) -> dict:
    s = seed_stats()
    _check(lib().seed_get_stats(ctx.handle, C.byref(s)), "seed_get_stats", ctx.handle)
    return s.as_dict()


def seed_time_operator(ctx: Context, op: int, ncols: int, reps: int) -> float:
    """Mean device time (ms) of one application of op over ncols columns."""
    ms = C.c_double()
    _check(lib().seed_time_operator(ctx.handle, int(op), int(ncols), int(reps), C.byref(ms)), "seed_time_operator",
           ctx.handle)
    return ms.value


def seed_wilson_apply_noalloc(dims, kappa: float, links: torch.Tensor, X: torch.Tensor, Y: torch.Tensor,
                              bc_t: int = 0, stream=None):
    """Y = D^H D X without any device allocation, for callers that cannot
    allocate while they run (scratch: a fixed 8 MiB device array shared by all
    calls; see include/seed.h)."""
    assert links.dtype == torch.complex128 and links.is_contiguous()
    vol = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    px, ldx, nx = _block(X, 12 * vol, "X")
    py, ldy, ny = _block(Y, 12 * vol, "Y")
    if nx != ny:
        raise ValueError("X and Y must have the same number of columns")
    a = seed_wilson(kappa=float(kappa), bc_t=int(bc_t), reserved=0, links=links.data_ptr())
    for k in range(4):
        a.dims[k] = int(dims[k])
    _check(lib().seed_wilson_apply_noalloc(C.byref(a), px, ldx, py, ldy, nx, _stream(stream)),
           "seed_wilson_apply_noalloc")


def seed_time_fma(dtype: int = 0, stream=None) -> dict:
    """Measured FMA rate of the FP64 (dtype SEED_F64) or FP32 (SEED_F32) pipe:
    {"tflops": ..., "ms": ...} (see include/seed.h)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().seed_time_fma(int(dtype), _stream(stream), C.byref(tf), C.byref(ms)), "seed_time_fma")
    return {"tflops": tf.value, "ms": ms.value}


def seed_time_fp64_paths(stream=None) -> dict:
    """FP64 FMA chains against the FP64 matrix instructions (see include/seed.h):
    rates in TFLOP/s, and the mixed launch's time over the two halves' sum
    (~0.5: separate units, ~1: one shared unit)."""
    out = (C.c_double * 7)()
    _check(lib().seed_time_fp64_paths(_stream(stream), out), "seed_time_fp64_paths")
    return {"fma_tflops": out[0], "dmma_m8n8k4_tflops": out[1], "dmma_m16n8k16_tflops": out[2],
            "mix_over_sum": out[3], "ms_fma_half": out[4], "ms_dmma_half": out[5], "ms_mix": out[6]}


def seed_block_products(V: torch.Tensor, R: torch.Tensor, reps: int = 1, stream=None):
    """G = V^H R (k x nr complex128, numpy) from FP32 complex blocks V (n x k) and
    R (n x nr) on the tensor cores, and the mean device time of one launch in ms
    (see include/seed.h)."""
    import numpy as np
    assert V.dtype == torch.complex64 and R.dtype == torch.complex64
    n = V.shape[0]
    pv, ldv, k = _block(V, n, "V")
    pr, ldr, nr = _block(R, n, "R")
    G = np.zeros((k, nr), dtype=np.complex128)
    ms = C.c_double()
    _check(lib().seed_block_products(pv, ldv, k, pr, ldr, nr, n, G.ctypes.data_as(C.c_void_p), int(reps),
                                     C.byref(ms), _stream(stream)), "seed_block_products")
    return G, ms.value


def seed_last_error(ctx: Context = None) -> str:
    r = lib().seed_last_error(ctx.handle if ctx is not None else None)
    return r.decode() if r else ""


def seed_destroy(ctx: Context):
    if ctx is not None and ctx.handle:
        lib().seed_destroy(ctx.handle)
        ctx.handle = C.c_void_p()
