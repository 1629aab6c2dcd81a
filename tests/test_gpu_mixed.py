"""Mixed-precision path (precision = 1: FP32 operator and Krylov vectors, FP64
scalars, reductions and reliable updates) against the FP64 oracle.

Bounds, and where they come from:
 * FP32 operator applies are compared with the oracle applied in FP64 to the
   same inputs rounded to FP32 (links, matrix values and vectors), so that
   only the kernel's FP32 arithmetic differs.  An output element of D is
   psi - kappa * (sum of 8 hops), each hop a projected two-spinor (1 add)
   times a 3x3 complex matrix (3 complex FMAs) and a reconstruction (1 add),
   then 8 accumulations: a chain of at most ~20 roundings of unit
   u = 2^-24 on terms bounded by 2 |U| |psi|, so |err| <= 20 u * 16 * 2 *
   max|psi| * (1 + kappa) < 1e-5 max|psi|.  The test uses 1e-5 max|psi|;
   for A = D^H D the first product's error is carried through D^H
   (|D^H| <= 1 + 16 kappa < 3.5) and the second adds its own, so 1e-4 max|psi|;
   for the Laplacian's rows (5 terms bounded by 4 |x|, 5 roundings) 5e-6 max|x|.
 * Solves: every system's FP64 true residual, recomputed here with the
   oracle's operator, meets its tolerance (tol_seed for system 1, tol_rest for
   the others; factor 1.01 for the different summation order); the error
   against the oracle's FP64 solution is at most 2 kappa(A) tol relative,
   since both solutions have relative residual <= tol:
   ||x - x_o|| <= ||A^-1|| (||r|| + ||r_o||) and ||b|| <= ||A|| ||x_o||.
   kappa(A) comes from the extreme Ritz values of the oracle's seed run.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I
from tiled_layout import from_tiled, to_tiled

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev_cols(a, dtype=None):
    a = np.ascontiguousarray(np.asarray(a).T)
    t = torch.from_numpy(a).cuda()
    if dtype is not None:
        t = t.to(dtype)
    return t.t()


def host_cols(t):
    return t.t().cpu().numpy().T


def ritz_kappa(orc, seed):
    ev = orc.tridiag_eigs(seed["alpha"], seed["beta"][1:len(seed["alpha"])])
    return ev.max() / ev.min()


def true_relres(op, B, X):
    return np.array([np.linalg.norm(B[:, j] - op.apply(X[:, j])) / np.linalg.norm(B[:, j])
                     for j in range(B.shape[1])])


def mixed_solve(seedlib, ctx, B, X0=None):
    Bd = dev_cols(B)
    Xd = dev_cols(np.zeros_like(B) if X0 is None else X0)
    i1 = seedlib.seed_solve_first(ctx, Bd, Xd)
    i2 = seedlib.seed_solve_rest(ctx, Bd, Xd)
    torch.cuda.synchronize()
    return i1, i2, host_cols(Xd)


def check_solution(orc, op, B, X, ref, info1, info2, tol_seed, tol_rest, label):
    k = ritz_kappa(orc, ref["seed"])
    rr = true_relres(op, B, X)
    assert rr[0] <= 1.01 * tol_seed, (label, rr[0])
    assert np.all(rr[1:] <= 1.01 * tol_rest), (label, rr)
    assert info1[0]["converged"] == 1 and all(i["converged"] for i in info2[1:]), label
    # the library's own FP64 true residuals agree with the oracle's recomputation
    assert abs(info1[0]["true_relres"] - rr[0]) <= 1e-3 * rr[0] + 1e-16, (label, info1[0]["true_relres"], rr[0])
    for j in range(1, B.shape[1]):
        assert abs(info2[j]["true_relres"] - rr[j]) <= 1e-3 * rr[j] + 1e-16, (label, j)
    err0 = np.linalg.norm(X[:, 0] - ref["X"][:, 0]) / np.linalg.norm(ref["X"][:, 0])
    assert err0 <= 2 * k * tol_seed, (label, err0, k)
    for j in range(1, B.shape[1]):
        e = np.linalg.norm(X[:, j] - ref["X"][:, j]) / np.linalg.norm(ref["X"][:, j])
        assert e <= 2 * k * tol_rest, (label, j, e, k)
    # at least one FP64 reliable update per system (the last one certifies convergence)
    assert info1[0]["restarts"] >= 1 and all(i["restarts"] >= 1 for i in info2[1:])


# --------------------------------------------------------------------------
# FP32 operator applies
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 0), ((3, 4, 5, 6), 1), ((16, 16, 16, 16), 1)])
def test_fp32_wilson_apply(seedlib, orc, dims, bc_t):
    """From 16^4 = 65536 sites on, the FP32 operator runs one thread per site
    over column pairs (3 columns: one pair and one single column)."""
    kappa = 0.155
    U = I.random_su3_links(dims, 0.3, seed=2)
    n = 12 * I.lattice_sites(dims)
    p = seedlib.seed_params_default(m_max=4, precision=1)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=bc_t)
    X = I.gaussian_rhs(n, 3, seed=5, complex_=True)
    X32 = X.astype(np.complex64)
    U32 = U.astype(np.complex64).astype(np.complex128)
    Xd = dev_cols(X32)
    Yd = dev_cols(np.zeros_like(X32))
    oop = orc.Operator.wilson(dims, kappa, U32, bc_t=bc_t)
    for op, sign in ((4, +1), (5, -1), (3, None)):
        seedlib.seed_apply(ctx, op, Xd, Yd)
        torch.cuda.synchronize()
        Y = host_cols(Yd)
        for j in range(3):
            x = X32[:, j].astype(np.complex128)
            ref = oop.apply(x) if sign is None else orc.wilson_dslash(dims, kappa, bc_t, sign, U32, x)
            bound = (1e-4 if sign is None else 1e-5) * np.abs(x).max()
            assert np.abs(Y[:, j] - ref).max() <= bound, (op, j)


@pytest.mark.parametrize("dims,bc_t,ncols", [((16, 16, 16, 32), 0, 11), ((17, 17, 15, 16), 1, 3)])
def test_fp32_wilson_apply_tiled(seedlib, orc, dims, bc_t, ncols):
    """The FP32 operator in the mixed solver's own tiled layout and launch
    (seed_apply ops 6 and 7: the kernel, layout and column count that the
    benchmark times): the 16^3 x 32 workload lattice with the 11 columns of a
    lockstep CG launch, and a ragged 17x17x15x16 lattice whose last tile holds
    padding sites.  Every output against the oracle (the bound above), the
    padding written as zeros, and the result bitwise equal to the site-major
    launch of the same arithmetic (ops 4 and 5)."""
    kappa = 0.155
    U = I.random_su3_links(dims, 0.3, seed=3)
    sites = I.lattice_sites(dims)
    n = 12 * sites
    p = seedlib.seed_params_default(m_max=4, precision=1)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=bc_t)
    X32 = I.gaussian_rhs(n, ncols, seed=6, complex_=True).astype(np.complex64)
    Xt = dev_cols(to_tiled(X32, sites))
    Yt = dev_cols(np.full((384 * ((sites + 31) // 32), ncols), 7.0, dtype=np.complex64))
    Xs, Ys = dev_cols(X32), dev_cols(np.zeros_like(X32))
    U32 = U.astype(np.complex64).astype(np.complex128)
    for op_t, op_s, sign in ((6, 4, +1), (7, 5, -1)):
        seedlib.seed_apply(ctx, op_t, Xt, Yt)
        seedlib.seed_apply(ctx, op_s, Xs, Ys)
        torch.cuda.synchronize()
        Y, pad = from_tiled(host_cols(Yt), sites)
        assert np.all(pad == 0), op_t
        assert np.array_equal(Y, host_cols(Ys)), op_t
        for j in range(ncols):
            x = X32[:, j].astype(np.complex128)
            ref = orc.wilson_dslash(dims, kappa, bc_t, sign, U32, x)
            assert np.abs(Y[:, j] - ref).max() <= 1e-5 * np.abs(x).max(), (op_t, j)
    # the tiled ops need a mixed-precision Wilson context
    ctx64 = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), seedlib.seed_params_default(m_max=4))
    with pytest.raises(seedlib.SeedError):
        seedlib.seed_apply(ctx64, 6, Xt, Yt)


def test_fp32_csr_apply(seedlib, orc):
    rp, ci, v = I.laplacian_2d_csr(37, 29)
    n = 37 * 29
    p = seedlib.seed_params_default(m_max=4, precision=1)
    ctx = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                  torch.from_numpy(v).cuda(), p)
    X32 = I.gaussian_rhs(n, 2, seed=1).astype(np.float32)
    Xd, Yd = dev_cols(X32), dev_cols(np.zeros_like(X32))
    seedlib.seed_apply(ctx, 3, Xd, Yd)
    torch.cuda.synchronize()
    Y = host_cols(Yd)
    oop = orc.Operator.csr(rp, ci, v)
    for j in range(2):
        ref = oop.apply(X32[:, j].astype(np.float64)).real
        assert np.abs(Y[:, j] - ref).max() <= 5e-6 * np.abs(X32[:, j]).max()


# --------------------------------------------------------------------------
# solves
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nrhs", [2, 4])
@pytest.mark.parametrize("delta", [0.0, 0.1])   # 0: the default, 0.001
def test_mixed_laplacian_64(seedlib, orc, nrhs, delta):
    """64x64 Laplacian, Gaussian RHS (seed 0), seed to 1e-12 with full
    reorthogonalization; nrhs = 2 makes system 1's refinement and the rest
    phase run on one column each."""
    rp, ci, v = I.laplacian_2d_csr(64, 64)
    B = I.gaussian_rhs(4096, nrhs, seed=0)
    p = seedlib.seed_params_default(m_max=4096, reorth_freq=1, tol_seed=1e-12, tol_rest=1e-8, precision=1,
                                    reliable_delta=delta)
    ctx = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                  torch.from_numpy(v).cuda(), p)
    i1, i2, X = mixed_solve(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, m_max=4096, reorth_freq=1, tol_seed=1e-12, tol_rest=1e-8)
    check_solution(orc, op, B, X.real, ref, i1, i2, 1e-12, 1e-8, "lap64-mixed")


@pytest.mark.parametrize("kernel_path", [0, 1])
def test_mixed_csr_persistent_seed(seedlib, orc, kernel_path):
    """Shifted 96x80 Laplacian (shift 0.05), 4 Gaussian RHS, reorthogonalization
    every 10 steps: on path 0 the FP32 seed run is the persistent CSR kernel,
    on path 1 the step kernels; both certified against the oracle as the
    other solves are."""
    rp, ci, v = I.shifted_laplacian_2d_csr(96, 80, 0.05)
    n = 96 * 80
    B = I.gaussian_rhs(n, 4, seed=6)
    p = seedlib.seed_params_default(m_max=2000, reorth_freq=10, tol_seed=1e-10, tol_rest=1e-8, precision=1,
                                    kernel_path=kernel_path)
    ctx = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                  torch.from_numpy(v).cuda(), p)
    i1, i2, X = mixed_solve(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, m_max=2000, reorth_freq=10, tol_seed=1e-10, tol_rest=1e-8)
    check_solution(orc, op, B, X.real, ref, i1, i2, 1e-10, 1e-8, "csr-mixed-persistent-%d" % kernel_path)


@pytest.mark.parametrize("freq", [0, 10])
def test_mixed_wilson_small(seedlib, orc, freq):
    """3x4x5x6 lattice, kappa 0.14, antiperiodic t, 5 RHS b = D^H eta; an
    initial guess for every system (x0_zero = 0)."""
    dims, kappa = (3, 4, 5, 6), 0.14
    U = I.random_su3_links(dims, 0.3, seed=7)
    eta = I.point_sources(dims, 5, site=17)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(5)], axis=1)
    X0 = 0.01 * I.gaussian_rhs(B.shape[0], 5, seed=3, complex_=True)
    p = seedlib.seed_params_default(m_max=600, reorth_freq=freq, tol_seed=1e-12, tol_rest=1e-8, precision=1,
                                    x0_zero=0)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=1)
    i1, i2, X = mixed_solve(seedlib, ctx, B, X0)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_all(op, B, m_max=600, reorth_freq=freq, tol_seed=1e-12, tol_rest=1e-8)
    check_solution(orc, op, B, X, ref, i1, i2, 1e-12, 1e-8, "wilson-small-mixed")


def test_mixed_wilson_more_tiles_than_sms(seedlib, orc):
    """5x6x7x24 lattice (5040 sites, 158 tiles of 32: more than the GB300's 152
    SMs), kappa 0.12, antiperiodic t, 3 RHS, reorthogonalization every 25
    steps: the persistent FP32 seed run takes its site form (one thread per
    site, 448 sites per block: the last blocks of the grid hold no site and
    only join the barriers; one partial sum per block); smaller lattices take
    the resident form.  The 17x17x15x17 and 16^3 x 32 cases below run it with
    up to two sites per thread."""
    dims, kappa = (5, 6, 7, 24), 0.12
    U = I.random_su3_links(dims, 0.3, seed=11)
    eta = I.point_sources(dims, 3, site=101)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(3)], axis=1)
    p = seedlib.seed_params_default(m_max=800, reorth_freq=25, tol_seed=1e-12, tol_rest=1e-8, precision=1)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=1)
    i1, i2, X = mixed_solve(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_all(op, B, m_max=800, reorth_freq=25, tol_seed=1e-12, tol_rest=1e-8)
    check_solution(orc, op, B, X, ref, i1, i2, 1e-12, 1e-8, "wilson-158-tiles-mixed")


def test_mixed_wilson_large_lattice(seedlib, orc):
    """17x17x15x17 = 73695 sites (one thread per site in the FP32 operator,
    a site count that is not a multiple of 32, so the solver's tiled FP32
    vectors carry padding, and 2303 tiles, so the last 128-thread block of
    the operator's launches has threads past the last tile), kappa 0.10,
    antiperiodic t, 3 Gaussian RHS.
    Every system's FP64 true residual, recomputed by the oracle's operator,
    meets its tolerance, and the mixed solve needs at most 30 % more CG
    iterations than the FP64 solve of the same systems (a wrong FP32 operator
    would show up as slower or stalled convergence between reliable updates)."""
    dims, kappa = (17, 17, 15, 17), 0.10
    U = I.random_su3_links(dims, 0.3, seed=11)
    n = 12 * I.lattice_sites(dims)
    B = I.gaussian_rhs(n, 3, seed=4, complex_=True)
    prm = dict(m_max=400, reorth_freq=10, tol_seed=1e-9, tol_rest=1e-8)
    out = {}
    for prec in (0, 1):
        ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(),
                                         seedlib.seed_params_default(precision=prec, **prm), bc_t=1)
        out[prec] = mixed_solve(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    i1, i2, X = out[1]
    rr = true_relres(op, B, X)
    assert rr[0] <= 1.01 * 1e-9 and np.all(rr[1:] <= 1.01 * 1e-8), rr
    assert i1[0]["converged"] == 1 and all(i["converged"] for i in i2[1:])
    for j in (1, 2):
        it64 = out[0][1][j]["iters"]
        assert i2[j]["iters"] <= 1.3 * it64 + 2, (j, i2[j]["iters"], it64)


@pytest.mark.slow
def test_mixed_wilson_8_4_workload(seedlib, orc):
    """The 8^4 benchmark workload (12 point sources, seed to 1e-12 with
    reorthogonalization every 100 steps, CG to 1e-8) in mixed precision."""
    from test_gpu_parity import _workload_reference
    w = _workload_reference(orc)
    dims, kappa, U, B, ref = w["dims"], w["kappa"], w["U"], w["B"], w["ref"]
    p = seedlib.seed_params_default(m_max=3000, reorth_freq=100, reorth_passes=2, tol_seed=1e-12, tol_rest=1e-8,
                                    precision=1)
    ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p)
    i1, i2, X = mixed_solve(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U)
    check_solution(orc, op, B, X, ref, i1, i2, 1e-12, 1e-8, "wilson-8^4-mixed")


@pytest.mark.slow
def test_mixed_16x3x32_workload_certified_by_oracle(seedlib, orc):
    """The benchmark's 16^3 x 32 workload at full size, in the launch
    configuration the benchmark times: kappa 0.155, links of spread 0.3 (seed
    0), 12 Z4 noise sources (seed 0) with b = D^H eta formed by the oracle,
    seed to 1e-12 with reorthogonalization every 100 steps, CG to 1e-8, mixed
    precision.  The oracle cannot run this solve in seconds, so it certifies
    the result instead: every system's FP64 true residual, recomputed with the
    oracle's operator, meets its tolerance and agrees with the library's own;
    and the mixed CG needs at most 30 % more iterations per system than the
    FP64 solve of the same systems."""
    dims, kappa, nrhs = (16, 16, 16, 32), 0.155, 12
    U = I.random_su3_links(dims, 0.3, seed=0)
    n = 12 * I.lattice_sites(dims)
    eta = I.z4_noise(n, nrhs, seed=0)
    B = np.stack([orc.wilson_dslash(dims, kappa, 0, -1, U, eta[:, j]) for j in range(nrhs)], axis=1)
    prm = dict(m_max=3000, reorth_freq=100, reorth_passes=2, tol_seed=1e-12, tol_rest=1e-8)
    out = {}
    for prec in (1, 0):
        ctx = seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(),
                                         seedlib.seed_params_default(precision=prec, **prm))
        out[prec] = mixed_solve(seedlib, ctx, B)
        seedlib.seed_destroy(ctx)
    i1, i2, X = out[1]
    assert i1[0]["converged"] == 1 and all(i["converged"] for i in i2[1:])
    op = orc.Operator.wilson(dims, kappa, U)
    rr = true_relres(op, B, X)
    assert rr[0] <= 1.01e-12 and np.all(rr[1:] <= 1.01e-8), rr
    assert abs(i1[0]["true_relres"] - rr[0]) <= 1e-3 * rr[0] + 1e-16
    for j in range(1, nrhs):
        assert abs(i2[j]["true_relres"] - rr[j]) <= 1e-3 * rr[j] + 1e-16, j
        assert i2[j]["iters"] <= 1.3 * out[0][1][j]["iters"] + 2, (j, i2[j]["iters"], out[0][1][j]["iters"])


def test_mixed_rejects_fp64_basis_calls(seedlib):
    dims = (4, 4, 4, 4)
    U = I.random_su3_links(dims, 0.3, seed=2)
    p = seedlib.seed_params_default(m_max=50, precision=1, keep_basis=1, tol_seed=1e-8)
    ctx = seedlib.seed_create_wilson(dims, 0.12, torch.from_numpy(U).cuda(), p)
    B = dev_cols(I.gaussian_rhs(12 * 256, 2, seed=1, complex_=True))
    X = torch.zeros_like(B.t()).t()
    seedlib.seed_solve_first(ctx, B, X)
    with pytest.raises(seedlib.SeedError):
        seedlib.seed_project(ctx, B, X)
    with pytest.raises(seedlib.SeedError):
        seedlib.seed_get_basis(ctx, 2)
