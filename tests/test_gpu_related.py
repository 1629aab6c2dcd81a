"""Sec. 2.3 single seeding of related right-hand sides (seed_solve_related)
against the oracle's seed_solve_related, same seeded inputs.

Each system's CG iteration count within 5 % of the oracle's; every true
residual (recomputed here with the oracle's operator) <= 1.5 tol_rest; each
solution within 2 cond(A) 1.5 tol_rest of the oracle's (both have relative
residual <= 1.5 tol_rest; for the diagonal matrix cond(A) is max/min of its
entries, for the lattice it comes from the oracle's extreme Ritz values).
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().t()


def host(t):
    return t.t().cpu().numpy().T


def check(orc, op, B, X, ref, info, cond, tol, label):
    for j in range(1, B.shape[1]):
        r = ref["rest"][j - 1]
        g = info[j]
        assert g["converged"] == 1, (label, j)
        assert abs(g["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"]), (label, j, g["iters"], r["iters"])
        rr = np.linalg.norm(B[:, j] - op.apply(X[:, j])) / np.linalg.norm(B[:, j])
        assert rr <= 1.5 * tol, (label, j, rr)
        e = np.linalg.norm(X[:, j] - ref["X"][:, j]) / np.linalg.norm(ref["X"][:, j])
        assert e <= 2 * cond * 1.5 * tol, (label, j, e)


def test_related_example3_diagonal(seedlib, orc):
    """Sec. 2.3, Example 3: the Example 1 diagonal matrix (n = 5000), 8 related
    right-hand sides b^j = b^{j-1} + 0.2^{j-1} u^j."""
    n = 5000
    d = I.paper_diagonal(n, seed=0)
    rp, ci, v = I.diagonal_csr(d)
    B = I.related_rhs(n, 8, seed=1)
    p = seedlib.seed_params_default(m_max=5000, reorth_freq=1, tol_seed=1e-8, tol_rest=1e-8)
    ctx = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                  torch.from_numpy(v).cuda(), p)
    Bd = dev(B)
    Xd = torch.zeros_like(Bd.t()).t()
    seedlib.seed_solve_first(ctx, Bd, Xd)
    info = seedlib.seed_solve_related(ctx, Bd, Xd)
    torch.cuda.synchronize()
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_related(op, B, m_max=5000, reorth_freq=1, tol_seed=1e-8, tol_rest=1e-8)
    check(orc, op, B, host(Xd).real, ref, info, d.max() / d.min(), 1e-8, "example3")
    # the later systems start close: the last takes far fewer iterations than the first CG system
    assert info[-1]["iters"] < 0.5 * info[1]["iters"], [i["iters"] for i in info]


def test_related_wilson_small(seedlib, orc):
    """3x4x5x6 lattice, kappa 0.14, antiperiodic t; b^j = D^H eta^j with
    related complex sources eta^j = eta^{j-1} + 0.2^{j-1} u^j."""
    dims, kappa = (3, 4, 5, 6), 0.14
    U = I.random_su3_links(dims, 0.3, seed=7)
    n = 12 * I.lattice_sites(dims)
    re = I.related_rhs(n, 5, seed=3)
    im = I.related_rhs(n, 5, seed=4)
    eta = re + 1j * im
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(5)], axis=1)
    p = seedlib.seed_params_default(m_max=600, reorth_freq=10, tol_seed=1e-12, tol_rest=1e-8)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=1)
    Bd = dev(B)
    Xd = torch.zeros_like(Bd.t()).t()
    seedlib.seed_solve_first(ctx, Bd, Xd)
    info = seedlib.seed_solve_related(ctx, Bd, Xd)
    torch.cuda.synchronize()
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_related(op, B, m_max=600, reorth_freq=10, tol_seed=1e-12, tol_rest=1e-8)
    ev = orc.tridiag_eigs(ref["seed"]["alpha"], ref["seed"]["beta"][1:len(ref["seed"]["alpha"])])
    check(orc, op, B, host(Xd), ref, info, ev.max() / ev.min(), 1e-8, "wilson-related")


def test_related_rejects_mixed_and_guesses(seedlib):
    dims = (4, 4, 4, 4)
    U = torch.from_numpy(I.random_su3_links(dims, 0.3, seed=2)).cuda()
    B = dev(I.gaussian_rhs(12 * 256, 3, seed=1, complex_=True))
    X = torch.zeros_like(B.t()).t()
    for kw in (dict(precision=1), dict(x0_zero=0)):
        ctx = seedlib.seed_create_wilson(dims, 0.12, U, seedlib.seed_params_default(m_max=100, **kw))
        with pytest.raises(seedlib.SeedError):
            seedlib.seed_solve_related(ctx, B, X)
