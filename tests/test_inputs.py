"""The seeded input generators (no GPU, no method arithmetic) produce what
the workload recipes say: SU(3) links, point and Z4 sources, and the uneven
batch of shifted Laplacians."""
import numpy as np

from paper_0810_0330_gb300 import inputs as I


def test_links_are_special_unitary_and_seeded():
    dims = (3, 2, 2, 4)
    U = I.random_su3_links(dims, 0.3, seed=5)
    assert U.shape == (4, I.lattice_sites(dims), 3, 3) and U.dtype == np.complex128
    M = U.reshape(-1, 3, 3)
    eye = np.broadcast_to(np.eye(3), M.shape)
    assert np.abs(M @ np.conj(np.swapaxes(M, 1, 2)) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(M) - 1.0).max() < 1e-13
    # exp(i eps H): eps -> 0 gives the identity; the same seed gives the same links
    assert np.abs(I.random_su3_links(dims, 1e-9, seed=5).reshape(-1, 3, 3) - eye).max() < 1e-7
    assert np.array_equal(U, I.random_su3_links(dims, 0.3, seed=5))
    assert not np.array_equal(U, I.random_su3_links(dims, 0.3, seed=6))


def test_point_sources_and_z4_noise():
    dims = (2, 2, 2, 2)
    n = 12 * I.lattice_sites(dims)
    P = I.point_sources(dims, 12, site=3)
    assert P.shape == (n, 12) and P.flags.f_contiguous
    for j in range(12):
        nz = np.flatnonzero(P[:, j])
        assert list(nz) == [12 * 3 + j] and P[nz[0], j] == 1.0
    Z = I.z4_noise(n, 5, seed=0)
    assert Z.shape == (n, 5) and Z.flags.f_contiguous
    vals = np.unique(np.round(Z, 12))
    assert set(vals.tolist()) == {1 + 0j, -1 + 0j, 1j, -1j}
    assert np.array_equal(Z, I.z4_noise(n, 5, seed=0))


def test_batch_problems_recipe():
    ps = I.batch_problems(32, seed=0)
    assert len(ps) == 32
    for p in ps:
        side = p["sides"][0]
        n = side ** len(p["sides"])
        assert p["kind"] in ("2d", "3d") and len(set(p["sides"])) == 1
        assert 0.01 <= p["shift"] <= 1.0 and 4 <= p["nrhs"] <= 16
        assert 0.5e4 <= n <= 1.2e6, (p, n)
    rp, ci, v, B = I.batch_problem_arrays(ps[0])
    n = rp.shape[0] - 1
    assert B.shape == (n, ps[0]["nrhs"]) and rp[-1] == ci.shape[0] == v.shape[0]
    # diagonally dominant with a positive shift: symmetric positive definite
    diag = np.zeros(n)
    off = np.zeros(n)
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            if ci[k] == r:
                diag[r] += v[k]
            else:
                off[r] += abs(v[k])
    assert np.all(diag - off >= ps[0]["shift"] - 1e-12)
