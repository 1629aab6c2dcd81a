"""Failure detection, tested without a GPU fault.

 * Malformed operators are rejected on the host before any launch.
 * Non-finite right-hand sides end as status codes: in the seed system the
   initial residual norm beta_0 of the Sec. 3 start is not finite and no step
   runs (SEED_EINVAL); in a seeded system CG stops that system at its first
   non-finite residual while the others converge (SEED_ENOTCONV).
 * Injected allocation failures (host side: the k-th device allocation
   fails without calling cudaMalloc) give SEED_ENOMEM, leak nothing, and
   leave a context that completes the same solve bit for bit on retry.
 * The persistent kernels' grid-barrier wait gives up after its time limit
   (a barrier that can never complete) and the device stays usable.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, KAPPA = (4, 4, 4, 4), 0.12


def dev_cols(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().t()


def wilson_ctx(seedlib, U, **kw):
    prm = dict(m_max=200, reorth_freq=10, tol_seed=1e-10, tol_rest=1e-8, maxit_rest=2000)
    prm.update(kw)
    return seedlib.seed_create_wilson(DIMS, KAPPA, torch.from_numpy(U).cuda(), seedlib.seed_params_default(**prm))


def solve(seedlib, ctx, B):
    Bd = dev_cols(B)
    X = torch.zeros_like(Bd.t()).t()
    seedlib.seed_solve_first(ctx, Bd, X)
    seedlib.seed_solve_rest(ctx, Bd, X)
    torch.cuda.synchronize()
    return X


def test_malformed_csr_rejected_on_host(seedlib):
    rp, ci, v = I.laplacian_2d_csr(8, 8)
    n = 64
    p = seedlib.seed_params_default(m_max=10)
    cases = []
    bad = rp.copy()
    bad[5], bad[6] = bad[6], bad[5]
    cases.append((bad, ci, "nondecreasing"))
    bad = ci.copy()
    bad[7] = n
    cases.append((rp, bad, "col_idx"))
    bad = ci.copy()
    bad[3] = -1
    cases.append((rp, bad, "col_idx"))
    bad = rp.copy()
    bad[0] = 1
    cases.append((bad, ci, "row_ptr"))
    for r, c, word in cases:
        with pytest.raises(seedlib.SeedError) as e:
            seedlib.seed_create_csr(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(),
                                    torch.from_numpy(v).cuda(), p)
        assert e.value.status == seedlib.SEED_EINVAL and word in str(e.value), (word, str(e.value))


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_right_hand_sides_end_as_status(seedlib, precision):
    U = I.random_su3_links(DIMS, 0.3, seed=4)
    n = 12 * I.lattice_sites(DIMS)
    B = I.gaussian_rhs(n, 3, seed=2, complex_=True)
    ctx = wilson_ctx(seedlib, U, precision=precision)
    # NaN in the seed system
    Bn = B.copy()
    Bn[5, 0] = np.nan
    Bd = dev_cols(Bn)
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_solve_first(ctx, Bd, torch.zeros_like(Bd.t()).t())
    assert e.value.status == seedlib.SEED_EINVAL and "not finite" in str(e.value)
    # NaN in a seeded system: the seed solve is unaffected; CG ends that
    # system at once and converges the other
    Bn = B.copy()
    Bn[7, 1] = np.nan
    Bd = dev_cols(Bn)
    X = torch.zeros_like(Bd.t()).t()
    i1 = seedlib.seed_solve_first(ctx, Bd, X)
    assert i1[0]["converged"] == 1
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_solve_rest(ctx, Bd, X)
    assert e.value.status == seedlib.SEED_ENOTCONV
    info = e.value.info
    assert info[1]["converged"] == 0 and info[1]["iters"] <= 2, info[1]
    assert info[2]["converged"] == 1 and info[2]["true_relres"] <= 1.01e-8, info[2]
    # the context is still usable: a clean solve equals a fresh context's, bit for bit
    X1 = solve(seedlib, ctx, B)
    X2 = solve(seedlib, wilson_ctx(seedlib, U, precision=precision), B)
    assert torch.equal(X1, X2)


@pytest.mark.parametrize("precision", [0, 1])
def test_injected_allocation_failures(seedlib, precision):
    U = I.random_su3_links(DIMS, 0.3, seed=5)
    n = 12 * I.lattice_sites(DIMS)
    B = I.gaussian_rhs(n, 3, seed=3, complex_=True)
    far = 1 << 30
    # how many device allocations a create and a first solve make
    seedlib.seed_inject_alloc_failure(far)
    ctx = wilson_ctx(seedlib, U, precision=precision)
    n_create = far - seedlib.seed_inject_alloc_failure(far)
    Xref = solve(seedlib, ctx, B)
    n_solve = far - seedlib.seed_inject_alloc_failure(0)
    seedlib.seed_destroy(ctx)
    assert n_create >= 20 and n_solve >= 1, (n_create, n_solve)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # each allocation of seed_create_wilson fails in turn: SEED_ENOMEM, nothing leaked
    for k in range(1, n_create + 1):
        assert seedlib.seed_inject_alloc_failure(k) == 0
        with pytest.raises(seedlib.SeedError) as e:
            wilson_ctx(seedlib, U, precision=precision)
        assert e.value.status == seedlib.SEED_ENOMEM and "injected" in str(e.value), k
    seedlib.seed_inject_alloc_failure(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
    # each allocation of the first solve fails in turn: the context stays
    # valid and the retry completes the same solve
    for k in range(1, n_solve + 1):
        ctx = wilson_ctx(seedlib, U, precision=precision)
        seedlib.seed_inject_alloc_failure(k)
        with pytest.raises(seedlib.SeedError) as e:
            solve(seedlib, ctx, B)
        assert e.value.status == seedlib.SEED_ENOMEM, k
        seedlib.seed_inject_alloc_failure(0)
        assert torch.equal(solve(seedlib, ctx, B), Xref), k
        seedlib.seed_destroy(ctx)


def test_barrier_wait_times_out_and_device_stays_usable(seedlib):
    timed_out, ms = seedlib.seed_check_barrier_timeout()
    assert timed_out and 1900.0 <= ms <= 5000.0, (timed_out, ms)
    # persistent kernels still run afterwards (kernel_path 0 uses them here)
    U = I.random_su3_links(DIMS, 0.3, seed=6)
    n = 12 * I.lattice_sites(DIMS)
    B = I.gaussian_rhs(n, 2, seed=1, complex_=True)
    ctx = wilson_ctx(seedlib, U, kernel_path=0, reorth_freq=0)
    Bd = dev_cols(B)
    X = torch.zeros_like(Bd.t()).t()
    i1 = seedlib.seed_solve_first(ctx, Bd, X)
    i2 = seedlib.seed_solve_rest(ctx, Bd, X)
    assert i1[0]["converged"] == 1 and i2[1]["converged"] == 1
