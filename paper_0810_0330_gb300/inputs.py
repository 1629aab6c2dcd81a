"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds none of the seed method's arithmetic: it only builds
operators and right-hand sides (a CSR Laplacian, a random diagonal, SU(3)
gauge links, Gaussian / point-source / Z4 right-hand sides) from a numpy
``default_rng`` seed.  The oracle and the CUDA path both consume the exact
bytes produced here.

Workloads (the paper's problems, restated as synthetic stand-ins):

* Sec. 2, Example 1: a diagonal matrix, n = 5000, entries U[0,1] sorted,
  right-hand sides N(0,1).
* Sec. 4: A = D^H D for a Wilson-Dirac D on a 4-d lattice (the paper's
  quenched 20^3x32 configuration is not available, so links are random SU(3)
  matrices exp(i*eps*H) with H Hermitian traceless).
* A 2-d 5-point Dirichlet Laplacian as a real SPD test operator.
"""
from __future__ import annotations

import numpy as np


def laplacian_2d_csr(n1: int, n2: int):
    """2-d 5-point Dirichlet Laplacian on an n1 x n2 grid, unscaled (4 on the
    diagonal, -1 per neighbour).  Row r = i + n1*j (i fastest); columns are
    ascending within each row.  Returns (row_ptr i32, col_idx i32, vals f64)."""
    n = n1 * n2
    r = np.arange(n, dtype=np.int64)
    i, j = r % n1, r // n1
    # candidate entries of each row in ascending column order: r-n1, r-1, r, r+1, r+n1
    cand = np.stack([r - n1, r - 1, r, r + 1, r + n1], axis=1)
    ok = np.stack([j > 0, i > 0, np.ones(n, dtype=bool), i < n1 - 1, j < n2 - 1], axis=1)
    v = np.broadcast_to(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (n, 5))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(ok.sum(axis=1), out=row_ptr[1:])
    return row_ptr.astype(np.int32), cand[ok].astype(np.int32), np.ascontiguousarray(v[ok], dtype=np.float64)


def laplacian_3d_csr(n1: int, n2: int, n3: int, shift: float = 0.0):
    """3-d 7-point Dirichlet Laplacian (6 on the diagonal, -1 per neighbour)
    plus ``shift`` on the diagonal; row r = i + n1*(j + n2*k)."""
    n = n1 * n2 * n3
    idx = np.arange(n, dtype=np.int64)
    i = idx % n1
    j = (idx // n1) % n2
    k = idx // (n1 * n2)
    offs = [(-n1 * n2, k > 0), (-n1, j > 0), (-1, i > 0), (0, np.ones(n, bool)),
            (1, i < n1 - 1), (n1, j < n2 - 1), (n1 * n2, k < n3 - 1)]
    counts = sum(m.astype(np.int64) for _, m in offs)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col_idx = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    pos = row_ptr[:-1].copy()
    for off, m in offs:
        rows = idx[m]
        col_idx[pos[m]] = (rows + off).astype(np.int32)
        vals[pos[m]] = (6.0 + shift) if off == 0 else -1.0
        pos[m] += 1
    return row_ptr.astype(np.int32), col_idx, vals


def shifted_laplacian_2d_csr(n1: int, n2: int, shift: float):
    """laplacian_2d_csr plus ``shift`` on the diagonal."""
    row_ptr, col_idx, vals = laplacian_2d_csr(n1, n2)
    rows = np.repeat(np.arange(n1 * n2, dtype=np.int64), np.diff(row_ptr))
    vals = vals.copy()
    vals[col_idx == rows] += shift
    return row_ptr, col_idx, vals


def batch_problems(count: int = 32, n_min: float = 1e4, n_max: float = 1e6, seed: int = 0):
    """Uneven batch of SPD problems: each a 2-d (side round(sqrt n)) or 3-d
    (side round(cbrt n)) Dirichlet Laplacian plus a diagonal shift U(0.01, 1),
    n log-uniform in [n_min, n_max], 4..16 right-hand sides.  Returns a list of
    dicts (kind, sides, shift, nrhs, rhs_seed); ``batch_problem_arrays`` builds
    the CSR arrays and right-hand sides of one entry."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        kind = "2d" if rng.uniform() < 0.5 else "3d"
        side = max(2, int(round(n ** 0.5 if kind == "2d" else n ** (1.0 / 3.0))))
        shift = float(rng.uniform(0.01, 1.0))
        nrhs = int(rng.integers(4, 17))
        out.append(dict(kind=kind, sides=(side,) * (2 if kind == "2d" else 3), shift=shift, nrhs=nrhs,
                        rhs_seed=seed * 1000 + i))
    return out


def batch_problem_arrays(p):
    """(row_ptr, col_idx, vals, B) of one batch_problems entry; B Gaussian N(0,1), column-major."""
    if p["kind"] == "2d":
        rp, ci, v = shifted_laplacian_2d_csr(p["sides"][0], p["sides"][1], p["shift"])
    else:
        rp, ci, v = laplacian_3d_csr(*p["sides"], shift=p["shift"])
    return rp, ci, v, gaussian_rhs(rp.shape[0] - 1, p["nrhs"], seed=p["rhs_seed"])


def diagonal_csr(d: np.ndarray):
    """CSR of diag(d)."""
    n = d.shape[0]
    return (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
            np.ascontiguousarray(d, dtype=np.float64))


def paper_diagonal(n: int = 5000, seed: int = 0) -> np.ndarray:
    """Sec. 2, Example 1: diagonal entries uniform on [0, 1], sorted."""
    return np.sort(np.random.default_rng(seed).uniform(0.0, 1.0, n))


def gaussian_rhs(n: int, nrhs: int, seed: int = 0, complex_: bool = False) -> np.ndarray:
    """Column-major (Fortran-ordered) n x nrhs block of N(0,1) right-hand sides.
    Real case: ``default_rng(seed).standard_normal((nrhs, n))`` transposed, so
    column j is the j-th row drawn.  Complex case: re and im each N(0,1)."""
    rng = np.random.default_rng(seed)
    if complex_:
        re = rng.standard_normal((nrhs, n))
        im = rng.standard_normal((nrhs, n))
        return np.asfortranarray((re + 1j * im).T)
    return np.asfortranarray(rng.standard_normal((nrhs, n)).T)


def related_rhs(n: int, nrhs: int, seed: int = 0, ratio: float = 0.2) -> np.ndarray:
    """Sec. 2.3, Example 3: b^j = b^{j-1} + ratio^{j-1} u^j, b^1 and u^j N(0,1)."""
    rng = np.random.default_rng(seed)
    b = np.empty((n, nrhs), order="F")
    b[:, 0] = rng.standard_normal(n)
    for j in range(1, nrhs):
        b[:, j] = b[:, j - 1] + ratio ** j * rng.standard_normal(n)
    return b


# ----------------------------------------------------------------------------
# Lattice inputs.  Canonical layouts (shared by the oracle and the CUDA path):
#   site s = x + X*(y + Y*(z + Z*t))            (x fastest)
#   spinor  [site][spin 0..3][colour 0..2]      complex128 (n = 12 * sites)
#   links   [mu 0..3][site][row a][col b]       complex128, U_mu(s)[a][b]
# ----------------------------------------------------------------------------

def lattice_sites(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def _random_hermitian_traceless(rng, count: int) -> np.ndarray:
    m = rng.standard_normal((count, 3, 3)) + 1j * rng.standard_normal((count, 3, 3))
    h = 0.5 * (m + np.conj(np.swapaxes(m, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h -= tr[:, None, None] * np.eye(3)[None]
    return h


def su3_from_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for a stack of Hermitian 3x3 H, via H = Q diag(l) Q^H."""
    lam, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return np.einsum("kab,kb,kcb->kac", q, ph, np.conj(q))


def random_su3_links(dims, eps: float = 0.3, seed: int = 0) -> np.ndarray:
    """Links U_mu(s) = exp(i*eps*H) with H = (M+M^H)/2 - tr(.)/3, M complex
    Gaussian (re, im each N(0,1)).  Shape (4, sites, 3, 3), complex128."""
    vol = lattice_sites(dims)
    rng = np.random.default_rng(seed)
    h = _random_hermitian_traceless(rng, 4 * vol)
    u = su3_from_hermitian(h, eps)
    return np.ascontiguousarray(u.reshape(4, vol, 3, 3))


def unit_links(dims) -> np.ndarray:
    vol = lattice_sites(dims)
    u = np.zeros((4, vol, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def random_gauge_transform(dims, seed: int = 1) -> np.ndarray:
    """One SU(3) matrix g(s) per site, shape (sites, 3, 3)."""
    vol = lattice_sites(dims)
    rng = np.random.default_rng(seed)
    return su3_from_hermitian(_random_hermitian_traceless(rng, vol), 1.0)


def point_sources(dims, nrhs: int = 12, site: int = 0) -> np.ndarray:
    """Unit point sources at one site: column j is 1 at (site, spin j//3,
    colour j%3).  Column-major n x nrhs complex128."""
    n = 12 * lattice_sites(dims)
    b = np.zeros((n, nrhs), dtype=np.complex128, order="F")
    for j in range(nrhs):
        b[12 * site + j % 12, j] = 1.0
    return b


def z4_noise(n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """Entries uniform in {1, i, -1, -i}; column-major n x nrhs complex128."""
    k = np.random.default_rng(seed).integers(0, 4, size=(nrhs, n))
    return np.asfortranarray((1j ** k).T.astype(np.complex128))
