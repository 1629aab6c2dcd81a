"""Adjoint of the seed solve (NEXT: differentiation) against the FP64 oracle.

 * seed_grad_kappa against the oracle's sum_j Re <lambda_j, (dA/dkappa) x_j>
   (the oracle's dA/dkappa is pinned by central differences of A), 1e-12
   relative: the same FP64 sums in another order.
 * seed_solve_cg against the oracle's CG: the same iteration counts (within
   5 %) and solutions within 1e-9.
 * wilson_seed_solve (torch.autograd): loss sum_j ||x_j - t_j||^2, gradients
   for B and kappa against the oracle's adjoint_reference (pinned by finite
   differences of the loss).  Forward and backward solves run to 1e-12, so
   both gradients are accurate to ~kappa(A) 1e-12; the bound is 1e-8 relative.
   The backward pass seeded from the forward basis gives the same gradients
   as an unseeded one with fewer CG iterations.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().t()


def host(t):
    return t.detach().t().cpu().numpy().T


@pytest.mark.parametrize("dims,bc_t", [((3, 4, 5, 6), 1), ((4, 4, 4, 4), 0)])
def test_grad_kappa_inner_matches_oracle(seedlib, orc, dims, bc_t):
    kappa = 0.13
    U = I.random_su3_links(dims, 0.3, seed=11)
    n = 12 * I.lattice_sites(dims)
    L = I.gaussian_rhs(n, 3, seed=12, complex_=True)
    X = I.gaussian_rhs(n, 3, seed=13, complex_=True)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), seedlib.seed_params_default(m_max=4),
                                     bc_t=bc_t)
    got = seedlib.seed_grad_kappa(ctx, dev(L), dev(X))
    ref = sum(float(np.vdot(L[:, j], orc.wilson_dA_dkappa(dims, kappa, bc_t, U, X[:, j])).real) for j in range(3))
    scale = sum(np.linalg.norm(L[:, j]) * np.linalg.norm(orc.wilson_dA_dkappa(dims, kappa, bc_t, U, X[:, j]))
                for j in range(3))
    assert abs(got - ref) <= 1e-12 * scale, (got, ref)


def test_solve_cg_all_columns_matches_oracle(seedlib, orc):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = I.random_su3_links(dims, 0.3, seed=3)
    n = 12 * I.lattice_sites(dims)
    B = I.gaussian_rhs(n, 3, seed=4, complex_=True)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(),
                                     seedlib.seed_params_default(m_max=4, tol_rest=1e-10))
    X = torch.zeros((3, n), dtype=torch.complex128, device="cuda").t()
    info = seedlib.seed_solve_cg(ctx, dev(B), X)
    Xh = host(X)
    op = orc.Operator.wilson(dims, kappa, U)
    for j in range(3):
        r = orc.cg(op, B[:, j], np.zeros(n, dtype=np.complex128), tol=1e-10)
        assert abs(info[j]["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"])
        assert np.linalg.norm(Xh[:, j] - r["x"]) <= 1e-9 * np.linalg.norm(r["x"])
        assert info[j]["converged"] == 1 and info[j]["true_relres"] <= 1.5e-10


def _loss_and_grads(seedlib, dims, kappa, U, B, T, seeded):
    from paper_0810_0330_gb300.adjoint import WilsonSeedSolve
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    Bd = dev(B).requires_grad_(True)
    Td = dev(T)
    prm = dict(m_max=2000, reorth_freq=10, tol_seed=1e-12, tol_rest=1e-12)
    Xd = WilsonSeedSolve.apply(k, Bd, torch.from_numpy(U).cuda(), dims, 0, prm, seeded)
    loss = ((Xd - Td).abs() ** 2).sum()
    loss.backward()
    return loss.item(), float(k.grad), host(Bd.grad)


def test_autograd_gradients_match_oracle(seedlib, orc):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = I.random_su3_links(dims, 0.3, seed=21)
    n = 12 * I.lattice_sites(dims)
    B = I.gaussian_rhs(n, 3, seed=22, complex_=True)
    T = I.gaussian_rhs(n, 3, seed=23, complex_=True)
    ref = orc.adjoint_reference(dims, kappa, U, B, T, tol=1e-13)
    loss, gk, gB = _loss_and_grads(seedlib, dims, kappa, U, B, T, True)
    assert abs(loss - ref["loss"]) <= 1e-9 * ref["loss"]
    assert abs(gk - ref["grad_kappa"]) <= 1e-8 * abs(ref["grad_kappa"]), (gk, ref["grad_kappa"])
    assert np.linalg.norm(gB - ref["grad_B"]) <= 1e-8 * np.linalg.norm(ref["grad_B"])
    # unseeded backward: same gradients
    loss2, gk2, gB2 = _loss_and_grads(seedlib, dims, kappa, U, B, T, False)
    assert abs(gk2 - gk) <= 1e-8 * abs(gk)
    assert np.linalg.norm(gB2 - gB) <= 1e-8 * np.linalg.norm(gB)


def test_autograd_backward_seeded_saves_iterations(seedlib):
    from paper_0810_0330_gb300.adjoint import WilsonSeedSolve
    dims, kappa = (4, 4, 4, 4), 0.12
    U = torch.from_numpy(I.random_su3_links(dims, 0.3, seed=21)).cuda()
    n = 12 * I.lattice_sites(dims)
    B = dev(I.gaussian_rhs(n, 4, seed=22, complex_=True))
    T = dev(I.gaussian_rhs(n, 4, seed=23, complex_=True))
    its = {}
    for seeded in (True, False):
        k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
        prm = dict(m_max=2000, reorth_freq=10, tol_seed=1e-10, tol_rest=1e-8)
        X = WilsonSeedSolve.apply(k, B, U, dims, 0, prm, seeded)
        ((X - T).abs() ** 2).sum().backward()
        its[seeded] = sum(i["iters"] for i in X.grad_fn.info_backward)
    assert its[True] < its[False], its


def test_autograd_kappa_central_difference_on_gpu(seedlib):
    """dL/dkappa from the backward pass against (L(k+h) - L(k-h)) / 2h of the
    GPU loss, at kappa = 0.10 where A is well conditioned (free-field bound
    cond(A) <= ((1 + 8k) / (1 - 8k))^2 = 81; near kappa = 1/8 it is not): the
    solves' error (<= 81 x 1e-13 relative in x) moves each L by ~1e-11 L, so
    the quotient's rounding part is ~1e-6 L, below 1e-6 of the derivative,
    whose scale is L / (1/8 - kappa); the truncation (h^2 / 6 times the third derivative) is smaller."""
    from paper_0810_0330_gb300.adjoint import WilsonSeedSolve
    dims, kappa, h = (4, 4, 4, 4), 0.10, 1e-5
    U = torch.from_numpy(I.random_su3_links(dims, 0.3, seed=31)).cuda()
    n = 12 * I.lattice_sites(dims)
    B = dev(I.gaussian_rhs(n, 2, seed=32, complex_=True))
    T = dev(I.gaussian_rhs(n, 2, seed=33, complex_=True))
    prm = dict(m_max=2000, reorth_freq=10, tol_seed=1e-13, tol_rest=1e-13)

    def loss(kv, grad=False):
        k = torch.tensor(kv, dtype=torch.float64, requires_grad=grad)
        X = WilsonSeedSolve.apply(k, B, U, dims, 0, prm, True)
        L = ((X - T).abs() ** 2).sum()
        if grad:
            L.backward()
            return L.item(), float(k.grad)
        return L.item()

    _, g = loss(kappa, grad=True)
    fd = (loss(kappa + h) - loss(kappa - h)) / (2 * h)
    assert abs(fd - g) <= 1e-6 * abs(g), (fd, g)


def test_autograd_mixed_precision_gradients_match_oracle(seedlib, orc):
    """Forward and adjoint solves in mixed precision (FP32 iterations, FP64
    reliable updates to the same 1e-12 tolerances): the same 1e-8 bound."""
    from paper_0810_0330_gb300.adjoint import WilsonSeedSolve
    dims, kappa = (4, 4, 4, 4), 0.12
    U = I.random_su3_links(dims, 0.3, seed=21)
    n = 12 * I.lattice_sites(dims)
    B = I.gaussian_rhs(n, 3, seed=22, complex_=True)
    T = I.gaussian_rhs(n, 3, seed=23, complex_=True)
    ref = orc.adjoint_reference(dims, kappa, U, B, T, tol=1e-13)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    Bd = dev(B).requires_grad_(True)
    prm = dict(m_max=2000, reorth_freq=10, tol_seed=1e-12, tol_rest=1e-12, precision=1)
    X = WilsonSeedSolve.apply(k, Bd, torch.from_numpy(U).cuda(), dims, 0, prm, True)
    loss = ((X - dev(T)).abs() ** 2).sum()
    loss.backward()
    assert abs(loss.item() - ref["loss"]) <= 1e-9 * ref["loss"]
    assert abs(float(k.grad) - ref["grad_kappa"]) <= 1e-8 * abs(ref["grad_kappa"])
    assert np.linalg.norm(host(Bd.grad) - ref["grad_B"]) <= 1e-8 * np.linalg.norm(ref["grad_B"])
