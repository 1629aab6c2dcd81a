"""The C-ABI library loads and exports every entry point include/seed.h
declares; argument errors come back as status codes (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "seed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(seed_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("seed_create_csr", "seed_create_wilson", "seed_solve_first", "seed_project", "seed_solve_rest",
              "seed_destroy", "seed_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(seedlib):
    L = C.CDLL(seedlib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(seedlib.EXPORTS) == _declared()


def test_abi_version_and_defaults(seedlib):
    L = seedlib.lib()
    assert L.seed_abi_version() == 2
    p = seedlib.seed_params_default()
    assert p.m_max == 1000 and p.reorth_passes == 2 and p.x0_zero == 1
    assert p.tol_seed == 1e-12 and p.tol_rest == 1e-8
    assert p.precision == 0 and p.reliable_delta == 0.0 and p.kernel_path == 0
    # the ctypes mirror has the C struct's size (4 + 8 int32, 3 doubles, 4 int32, 1 double)
    assert C.sizeof(seedlib.seed_params) == 4 * 8 + 8 * 3 + 4 * 4 + 8


def test_argument_errors_are_status_codes(seedlib):
    L = seedlib.lib()
    P = seedlib
    assert L.seed_params_default(None) == P.SEED_EINVAL
    h = C.c_void_p()
    prm = P.seed_params_default()
    # NULL operator / out pointer
    assert L.seed_create_csr(None, None, C.byref(prm), None) == P.SEED_EINVAL
    assert L.seed_create_csr(C.byref(h), None, C.byref(prm), None) == P.SEED_EINVAL
    assert h.value is None
    # bad sizes are rejected before any device call
    a = P.seed_csr(n=0, nnz=0)
    assert L.seed_create_csr(C.byref(h), C.byref(a), C.byref(prm), None) == P.SEED_EINVAL
    w = P.seed_wilson(kappa=0.1, bc_t=0)
    for k in range(4):
        w.dims[k] = 1
    assert L.seed_create_wilson(C.byref(h), C.byref(w), C.byref(prm), None) == P.SEED_EINVAL
    w.dims[0] = w.dims[1] = w.dims[2] = w.dims[3] = 4
    w.bc_t = 3
    assert L.seed_create_wilson(C.byref(h), C.byref(w), C.byref(prm), None) == P.SEED_EINVAL
    assert b"bc_t" in L.seed_last_error(None)
    # bad parameters
    bad = P.seed_params_default(reorth_passes=3)
    w.bc_t = 0
    assert L.seed_create_wilson(C.byref(h), C.byref(w), C.byref(bad), None) == P.SEED_EINVAL
    for kw in (dict(precision=2), dict(precision=-1), dict(reliable_delta=1.0), dict(reliable_delta=-0.5),
               dict(kernel_path=3)):
        bad = P.seed_params_default(**kw)
        assert L.seed_create_wilson(C.byref(h), C.byref(w), C.byref(bad), None) == P.SEED_EINVAL, kw
    # NULL context
    assert L.seed_solve_first(None, None, 0, None, 0, 1, None) == P.SEED_EINVAL
    assert L.seed_solve_rest(None, None, 0, None, 0, 1, None) == P.SEED_EINVAL
    assert L.seed_project(None, None, 0, None, 0, 1) == P.SEED_EINVAL
    L.seed_destroy(None)


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No fallback: without libseed.so every entry point raises instead of
    computing anything another way."""
    from paper_0810_0330_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", "/nonexistent/libseed.so")
    with pytest.raises(RuntimeError, match="not built"):
        B.seed_params_default()
    with pytest.raises(RuntimeError, match="not built"):
        B.seed_inject_alloc_failure(0)


def _doc_before(src, name):
    """The comment block right before the declaration of `name` in the header."""
    m = re.search(r"/\*((?:(?!\*/).)*?)\*/\s*(?:seed_status|void|const char \*|int32_t)\s*" + name + r"\s*\(",
                  src, flags=re.S)
    assert m, name
    return " ".join(m.group(1).replace("*", " ").split())


def test_boundary_calls_cite_their_passage():
    """Every call of the boundary cites the passage of the paper that defines
    its operation (Sec. 1 problem, Sec. 3 algorithm and its basis storage,
    Sec. 4 normal equations); the error-reporting call says it has none."""
    src = open(os.path.join(ROOT, "include", "seed.h")).read()
    for name in ("seed_create_csr", "seed_create_wilson", "seed_solve_first", "seed_project", "seed_solve_rest",
                 "seed_destroy", "seed_solve_related", "seed_solve_multiple", "seed_get_tridiag"):
        assert "Sec." in _doc_before(src, name), name
    assert "Sec. 4" in _doc_before(src, "seed_create_wilson")
    assert "Sec. 1" in _doc_before(src, "seed_create_csr")
    assert "no counterpart" in _doc_before(src, "seed_last_error")
    assert "no counterpart" in _doc_before(src, "seed_wilson_apply_noalloc")
