"""GPU path (C ABI, sm_103a kernels) against the FP64 oracle, same seeded inputs.

Tolerances (FP64): operator applies 1e-13 relative per element; index tables
bit-exact; the seed system's x^1 to 1e-9 relative and the same number of
Lanczos steps; seeded-system CG iteration counts within 5 percent; true
residuals within 1.5 x 1e-8.  The seeded vectors x^2.., the final solutions of
systems 2.. and the late Lanczos coefficients are compared against
max(1e-9, 10 x the oracle's own change under random one-ulp noise on B),
measured in the test: loss of orthogonality between reorthogonalizations and
exactly degenerate eigenvalues make those quantities depend on rounding in any
implementation (the oracle included), see self_sensitivity below.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_X = 1e-9


def dev_cols(a: np.ndarray, ld: int = None):
    """numpy (n, k) -> CUDA tensor viewed (n, k) column-major, leading dimension ld."""
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    n, k = a.shape
    ld = ld or n
    buf = np.zeros((k, ld), dtype=a.dtype)
    buf[:, :n] = a.T
    t = torch.from_numpy(buf).cuda()
    return t[:, :n].t() if ld != n else t.t()


def host_cols(t) -> np.ndarray:
    return t.t().cpu().numpy().T if t.dim() == 2 else t.cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def wilson_ctx(seedlib, dims, kappa, U, bc_t=0, **prm):
    p = seedlib.seed_params_default(**prm)
    return seedlib.seed_create_wilson(dims, kappa, torch.from_numpy(U).cuda(), p, bc_t=bc_t)


def csr_ctx(seedlib, rp, ci, v, **prm):
    p = seedlib.seed_params_default(**prm)
    return seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                   torch.from_numpy(v).cuda(), p)


# --------------------------------------------------------------------------
# index tables and operators
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 4, 5, 6), (2, 2, 2, 2), (8, 8, 8, 8), (16, 2, 3, 5)])
def test_neighbor_table_bit_exact(seedlib, orc, dims):
    vol = int(np.prod(dims))
    out = torch.full((8 * vol,), -7, dtype=torch.int32, device="cuda")
    seedlib.seed_wilson_neighbors(dims, out)
    assert np.array_equal(out.cpu().numpy().reshape(vol, 8), orc.wilson_neighbors(dims))


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 0), ((3, 4, 5, 6), 1), ((2, 3, 2, 5), 0), ((8, 8, 8, 8), 1)])
def test_wilson_apply_matches_oracle(seedlib, orc, dims, bc_t):
    kappa = 0.155
    U = I.random_su3_links(dims, 0.3, seed=2)
    vol = I.lattice_sites(dims)
    n = 12 * vol
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=bc_t, m_max=4)
    X = I.gaussian_rhs(n, 3, seed=5, complex_=True)
    Xd = dev_cols(X, ld=n + 5)
    Yd = dev_cols(np.zeros_like(X), ld=n + 3)
    oop = orc.Operator.wilson(dims, kappa, U, bc_t=bc_t)
    for op, sign in ((1, +1), (2, -1), (0, None)):
        seedlib.seed_apply(ctx, op, Xd, Yd)
        torch.cuda.synchronize()
        Y = host_cols(Yd)
        for j in range(3):
            ref = oop.apply(X[:, j]) if sign is None else orc.wilson_dslash(dims, kappa, bc_t, sign, U, X[:, j])
            err = np.abs(Y[:, j] - ref).max() / np.abs(ref).max()
            assert err < 1e-13, (op, j, err)


def test_wilson_apply_past_grid_y_limit(seedlib, orc):
    """8x8x8x4096 = 2^21 sites = 65536 tiles of 32, one more than a grid's y
    extent: the hopping kernel runs its (tile, column) grid with the tile on x
    (the other order); D and D^H on two columns against the oracle.  The links
    are 64 random t-slices repeated (the kernel's indexing does not care)."""
    dims, kappa = (8, 8, 8, 4096), 0.155
    U = np.ascontiguousarray(np.tile(I.random_su3_links((8, 8, 8, 64), 0.3, seed=2), (1, 64, 1, 1)))
    n = 12 * I.lattice_sites(dims)
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=4)
    X = I.gaussian_rhs(n, 2, seed=6, complex_=True)
    Xd = dev_cols(X)
    Yd = dev_cols(np.zeros_like(X))
    for op, sign, cols in ((1, +1, (0, 1)), (2, -1, (1,))):
        seedlib.seed_apply(ctx, op, Xd, Yd)
        torch.cuda.synchronize()
        Y = host_cols(Yd)
        for j in cols:
            ref = orc.wilson_dslash(dims, kappa, 1, sign, U, X[:, j])
            err = np.abs(Y[:, j] - ref).max() / np.abs(ref).max()
            assert err < 1e-13, (op, j, err)
    seedlib.seed_destroy(ctx)


def test_csr_apply_matches_oracle(seedlib, orc):
    rp, ci, v = I.laplacian_2d_csr(37, 29)
    n = 37 * 29
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=4)
    X = I.gaussian_rhs(n, 2, seed=1)
    Xd, Yd = dev_cols(X), dev_cols(np.zeros_like(X))
    seedlib.seed_apply(ctx, 0, Xd, Yd)
    torch.cuda.synchronize()
    Y = host_cols(Yd)
    oop = orc.Operator.csr(rp, ci, v)
    for j in range(2):
        assert np.abs(Y[:, j] - oop.apply(X[:, j]).real).max() < 1e-13


# --------------------------------------------------------------------------
# Sec. 3 seed solve and the full single-seeding solve
# --------------------------------------------------------------------------

def run_gpu(seedlib, ctx, B, rest=True, ld=None):
    n, k = B.shape
    Bd = dev_cols(B, ld=ld)
    Xd = dev_cols(np.zeros_like(B), ld=ld)
    info1 = seedlib.seed_solve_first(ctx, Bd, Xd)
    torch.cuda.synchronize()
    Xs = host_cols(Xd)
    info2 = seedlib.seed_solve_rest(ctx, Bd, Xd) if rest else None
    torch.cuda.synchronize()
    return info1, info2, Xs, host_cols(Xd)


def self_sensitivity(orc, op, B, ref, cols=(1,), tol_rest=1e-8, **seed_kw):
    """How far the oracle's own seeded x^j and final CG solutions move when B
    is perturbed elementwise by random one-ulp noise.  Between
    reorthogonalizations the Lanczos basis loses orthogonality and the seeding
    projection amplifies rounding (Sec. 3): on the 8^4 Wilson workload with a
    reorthogonalization every 100 steps the oracle's seeded vectors move by
    about 4e-2 and its final solutions by about 7e-9, against 1e-13 and 5e-10
    every 10 steps.  Two correct implementations that round differently can
    differ by that much, so the parity bound for systems 2.. is
    max(1e-9, 10 x this sensitivity)."""
    rng = np.random.default_rng(12345)
    Bp = B * (1 + 2.2e-16 * rng.standard_normal(B.shape))
    sp = orc.seed_first(op, Bp, **seed_kw)
    self_sensitivity.perturbed = (Bp, sp["X"])
    seeded = np.linalg.norm(sp["X"][:, 1:] - ref["X_seeded"][:, 1:]) / np.linalg.norm(ref["X_seeded"][:, 1:])
    final = 0.0
    for j in cols:
        x = orc.cg(op, Bp[:, j], sp["X"][:, j], tol=tol_rest)["x"]
        final = max(final, relerr(x, ref["rest"][j - 1]["x"]))
    self_sensitivity.tridiag = tridiag_dev(sp["alpha"], sp["beta"], ref["seed"]["alpha"], ref["seed"]["beta"])
    return seeded, final


def seeded_only_sensitivity(orc, op, B, X0=None, **seed_kw):
    """The oracle's own one-ulp sensitivity of the seeded x^2.. alone.  Besides
    loss of orthogonality, exactly degenerate eigenvalues (the square
    Laplacian's lambda_kl = lambda_lk) make it large even with full
    reorthogonalization: Lanczos finds the second direction of a degenerate
    eigenspace from rounding, so which direction it finds -- and the
    projection of the other right-hand sides onto it -- depends on rounding."""
    rng = np.random.default_rng(12345)
    Bp = B * (1 + 2.2e-16 * rng.standard_normal(B.shape))
    a = orc.seed_first(op, B, X0=X0, **seed_kw)["X"][:, 1:]
    b = orc.seed_first(op, Bp, X0=X0, **seed_kw)["X"][:, 1:]
    return np.linalg.norm(a - b) / np.linalg.norm(a)


def tridiag_dev(a, b, a_ref, b_ref):
    """max relative deviation of alpha_1..alpha_m and beta_0..beta_m (common length)"""
    m = min(len(a), len(a_ref))
    da = np.abs(a[:m] - a_ref[:m]).max() / np.abs(a_ref).max()
    db = np.abs(b[:m + 1] - b_ref[:m + 1]).max() / np.abs(b_ref).max()
    return max(da, db)


def compare_full(orc_res, info1, info2, Xs, X, label, seeded_tol=REL_X, final_tol=REL_X, min_counted=0):
    """min_counted: compare CG iteration counts only where the oracle's is at
    least this (a system whose seeded residual is already near the tolerance
    can need 1 or 6 iterations depending on rounding of the seeding)."""
    s = orc_res["seed"]
    assert info1[0]["iters"] == s["iters"], (label, info1[0]["iters"], s["iters"])
    assert relerr(X[:, 0], s["X"][:, 0]) < REL_X
    assert relerr(Xs[:, 1:], orc_res["X_seeded"][:, 1:]) < seeded_tol, \
        (label, relerr(Xs[:, 1:], orc_res["X_seeded"][:, 1:]), seeded_tol)
    for j, r in enumerate(orc_res["rest"], start=1):
        g = info2[j]
        assert g["converged"] == 1
        if r["iters"] >= min_counted:
            assert abs(g["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"]), (label, j, g["iters"], r["iters"])
        if g["iters"] == r["iters"]:
            assert relerr(X[:, j], r["x"]) < final_tol, (label, j, relerr(X[:, j], r["x"]), final_tol)
        else:
            # counts apart: both meet the tolerance; solutions agree to the CG accuracy
            assert relerr(X[:, j], r["x"]) < max(1e-6, final_tol), (label, j)
        assert g["true_relres"] <= 1.5e-8


@pytest.mark.parametrize("kernel_path", [0, 1, 2])
def test_seed_config_laplacian_64(seedlib, orc, kernel_path):
    """64x64 Laplacian, 4 Gaussian RHS (seed 0), seed to 1e-12 with full
    reorthogonalization, then CG to 1e-8 (persistent CG kernel on path 0,
    step kernels on path 1)."""
    rp, ci, v = I.laplacian_2d_csr(64, 64)
    B = I.gaussian_rhs(4096, 4, seed=0)
    prm = dict(m_max=4096, reorth_freq=1, tol_seed=1e-12, tol_rest=1e-8, keep_basis=1, kernel_path=kernel_path)
    ctx = csr_ctx(seedlib, rp, ci, v, **prm)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, m_max=4096, reorth_freq=1, tol_seed=1e-12, tol_rest=1e-8)
    s_seed, s_final = self_sensitivity(orc, op, B, ref, cols=(1, 2), m_max=4096, reorth_freq=1, tol=1e-12)
    compare_full(ref, info1, info2, Xs.real, X.real, "lap64", seeded_tol=max(REL_X, 10 * s_seed),
                 final_tol=max(REL_X, 10 * s_final))
    a, b = seedlib.seed_get_tridiag(ctx)
    assert np.abs(a - ref["seed"]["alpha"]).max() < 1e-9 * np.abs(ref["seed"]["alpha"]).max()
    assert np.abs(b - ref["seed"]["beta"]).max() < 1e-9 * np.abs(ref["seed"]["beta"]).max()
    m = info1[0]["iters"]
    V = seedlib.seed_get_basis(ctx, m)
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-12
    assert info1[0]["true_relres"] < 1e-11


@pytest.mark.parametrize("kernel_path", [0, 1, 2])
@pytest.mark.parametrize("freq,passes", [(1, 2), (5, 1), (0, 2), (7, 2), (10, 2)])
def test_seed_wilson_small(seedlib, orc, freq, passes, kernel_path):
    """3x4x5x6 lattice (n = 4320, sites not a multiple of the block), kappa
    0.14, antiperiodic t, 5 point-source-derived RHS b = D^H eta.  Frequencies
    0 and 10 run the seed in persistent segments on path 0."""
    dims, kappa = (3, 4, 5, 6), 0.14
    U = I.random_su3_links(dims, 0.3, seed=7)
    eta = I.point_sources(dims, 5, site=17)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(5)], axis=1)
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=600, reorth_freq=freq, reorth_passes=passes,
                     tol_seed=1e-12, tol_rest=1e-8, kernel_path=kernel_path)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_all(op, B, m_max=600, reorth_freq=freq, reorth_passes=passes, tol_seed=1e-12,
                             tol_rest=1e-8)
    s_seed, s_final = self_sensitivity(orc, op, B, ref, cols=(1, 3), m_max=600, reorth_freq=freq,
                                       reorth_passes=passes, tol=1e-12)
    compare_full(ref, info1, info2, Xs, X, "wilson-small-%d" % freq, seeded_tol=max(REL_X, 10 * s_seed),
                 final_tol=max(REL_X, 10 * s_final))


@pytest.mark.parametrize("kernel_path", [0, 1])
def test_seed_wilson_more_tiles_than_sms(seedlib, orc, kernel_path):
    """5x6x7x24 lattice (5040 sites: 158 tiles of 32 sites, the last one
    ragged), kappa 0.12, antiperiodic t, 3 RHS, reorthogonalization every 25
    steps (152 seed steps): more tiles than the GB300's 152 SMs, so the
    persistent FP64 run (path 0) takes its general form, with several tiles
    per block and the links, indices and tile vectors read from global memory;
    smaller lattices (every other Wilson test here) take the resident form."""
    dims, kappa = (5, 6, 7, 24), 0.12
    U = I.random_su3_links(dims, 0.3, seed=11)
    eta = I.point_sources(dims, 3, site=101)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(3)], axis=1)
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=800, reorth_freq=25, reorth_passes=2,
                     tol_seed=1e-12, tol_rest=1e-8, kernel_path=kernel_path)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_all(op, B, m_max=800, reorth_freq=25, reorth_passes=2, tol_seed=1e-12, tol_rest=1e-8)
    s_seed, s_final = self_sensitivity(orc, op, B, ref, cols=(1, 2), m_max=800, reorth_freq=25,
                                       reorth_passes=2, tol=1e-12)
    compare_full(ref, info1, info2, Xs, X, "wilson-158-tiles-%d" % kernel_path, seeded_tol=max(REL_X, 10 * s_seed),
                 final_tol=max(REL_X, 10 * s_final))


@pytest.mark.parametrize("kernel_path", [0, 1])
def test_blocked_seeding_long_run_many_rhs(seedlib, orc, kernel_path):
    """Without reorthogonalization the 3x4x5x6 lattice at kappa 0.15 needs 219
    seed steps: on path 0 the persistent run is cut into segments of at most
    128 steps (one seeding block each), on path 1 into graph runs of 16; 20
    right-hand sides (19 seeded systems: five 4-column tiles of G, five
    4-column chunks of the X update).  Everything against the oracle as in
    test_seed_wilson_small, except that CG counts are compared only where the
    oracle needs 20 or more: without reorthogonalization the seeded vectors
    carry the oracle's own one-ulp sensitivity (checked), and systems seeded
    almost to tolerance finish in anywhere from 1 to a few iterations."""
    dims, kappa = (3, 4, 5, 6), 0.15
    U = I.random_su3_links(dims, 0.3, seed=7)
    eta = I.point_sources(dims, 20, site=17)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(20)], axis=1)
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=3000, reorth_freq=0, tol_seed=1e-12, tol_rest=1e-8,
                     kernel_path=kernel_path)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_solve_all(op, B, m_max=3000, reorth_freq=0, tol_seed=1e-12, tol_rest=1e-8)
    assert ref["seed"]["iters"] > 128
    s_seed, s_final = self_sensitivity(orc, op, B, ref, cols=(1, 19), m_max=3000, reorth_freq=0, tol=1e-12)
    compare_full(ref, info1, info2, Xs, X, "wilson-long-%d" % kernel_path, seeded_tol=max(REL_X, 10 * s_seed),
                 final_tol=max(REL_X, 10 * s_final), min_counted=20)


@pytest.mark.parametrize("kernel_path", [0, 1])
@pytest.mark.parametrize("freq", [1, 0, 10])
def test_lucky_breakdown_diagonal(seedlib, orc, kernel_path, freq):
    """diag(d) with 7 distinct eigenvalues (n = 100), 3 Gaussian RHS: the
    Krylov space of b^1 is exhausted after 7 steps, so the seed run ends at a
    lucky breakdown (beta_i ~ 0) with x^1 exact.  Step count equal to the
    oracle's and x^1 within 1e-9, on the streaming (freq 1) and blocked
    (freq 0, 10) seeding and both kernel paths.  The run's last step works on
    v = f / beta with f at rounding level (beta below the breakdown threshold
    only after it), a direction fixed by rounding; its projection moves the
    seeded x^2, x^3 by O(1e-2), so those are held to max(1e-9, 10 x the
    oracle's own one-ulp sensitivity)."""
    d = np.repeat(np.array([0.5, 1.0, 2.0, 3.0, 5.0, 8.0, 13.0]), [10, 20, 15, 5, 25, 10, 15])
    rp, ci, v = I.diagonal_csr(d)
    B = I.gaussian_rhs(100, 3, seed=1)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=200, reorth_freq=freq, tol_seed=1e-14, kernel_path=kernel_path)
    info1, _, Xs, _ = run_gpu(seedlib, ctx, B, rest=False)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_first(op, B, m_max=200, reorth_freq=freq, tol=1e-14)
    assert info1[0]["iters"] == ref["iters"] <= 8, (info1[0]["iters"], ref["iters"])
    assert info1[0]["converged"] == 1
    assert info1[0]["true_relres"] < 1e-12
    assert relerr(Xs[:, 0].real, ref["X"][:, 0].real) < REL_X
    sens = seeded_only_sensitivity(orc, op, B, m_max=200, reorth_freq=freq, tol=1e-14)
    assert relerr(Xs[:, 1:].real, ref["X"][:, 1:].real) < max(REL_X, 10 * sens), sens


@pytest.mark.parametrize("kernel_path", [0, 1])
@pytest.mark.parametrize("freq", [10, 0])
def test_extra_iters_past_convergence(seedlib, orc, kernel_path, freq):
    """extra_iters = 20 (the seed run continues past convergence to improve
    the seeding): 168 + 20 = 188 steps on the 3x4x5x6 lattice as in the
    oracle; x^1 within 1e-9 and the seeded x^2, x^3 within max(1e-9, 10 x the
    oracle's one-ulp sensitivity)."""
    dims, kappa = (3, 4, 5, 6), 0.14
    U = I.random_su3_links(dims, 0.3, seed=7)
    eta = I.point_sources(dims, 3, site=17)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(3)], axis=1)
    kw = dict(m_max=600, reorth_freq=freq, tol=1e-10, extra_iters=20)
    ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=600, reorth_freq=freq, tol_seed=1e-10, extra_iters=20,
                     kernel_path=kernel_path)
    info1, _, Xs, _ = run_gpu(seedlib, ctx, B, rest=False)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_first(op, B, **kw)
    assert info1[0]["iters"] == ref["iters"], (info1[0]["iters"], ref["iters"])
    assert ref["iters"] == ref["converged_at"] + 20
    assert relerr(Xs[:, 0], ref["X"][:, 0]) < REL_X
    sens = seeded_only_sensitivity(orc, op, B, **kw)
    assert relerr(Xs[:, 1:], ref["X"][:, 1:]) < max(REL_X, 10 * sens), (relerr(Xs[:, 1:], ref["X"][:, 1:]), sens)


def test_fresh_contexts_reuse_freed_memory(seedlib, orc):
    """Contexts created right after others were destroyed get device memory
    that held the old contexts' data; the persistent seed runs of the new ones
    (Wilson and CSR, FP64 and mixed) must not read any of it as state.  Ten
    create / solve / destroy rounds, each compared with the oracle's seed."""
    dims, kappa = (3, 4, 5, 6), 0.14
    U = I.random_su3_links(dims, 0.3, seed=7)
    eta = I.point_sources(dims, 3, site=17)
    B = np.stack([orc.wilson_dslash(dims, kappa, 1, -1, U, eta[:, j]) for j in range(3)], axis=1)
    op = orc.Operator.wilson(dims, kappa, U, bc_t=1)
    ref = orc.seed_first(op, B, m_max=600, reorth_freq=10, tol=1e-10)
    rp, ci, v = I.laplacian_2d_csr(30, 20)
    Bc = I.gaussian_rhs(600, 3, seed=2)
    for r in range(10):
        prec = r % 2
        ctx = wilson_ctx(seedlib, dims, kappa, U, bc_t=1, m_max=600, reorth_freq=10, tol_seed=1e-10,
                         precision=prec)
        info1, _, _, X = run_gpu(seedlib, ctx, B, rest=False)
        assert info1[0]["converged"] == 1, r
        if prec == 0:
            assert info1[0]["iters"] == ref["iters"], (r, info1[0]["iters"], ref["iters"])
        seedlib.seed_destroy(ctx)
        cc = csr_ctx(seedlib, rp, ci, v, m_max=600, reorth_freq=10, tol_seed=1e-10, precision=prec)
        info1, _, _, _ = run_gpu(seedlib, cc, Bc, rest=False)
        assert info1[0]["converged"] == 1, r
        seedlib.seed_destroy(cc)


_WORKLOAD_REF = {}


def _workload_reference(orc):
    """Oracle solution of the benchmark workload and its one-ulp sensitivity (computed once)."""
    if not _WORKLOAD_REF:
        dims, kappa = (8, 8, 8, 8), 0.155
        U = I.random_su3_links(dims, 0.3, seed=0)
        eta = I.point_sources(dims, 12)
        B = np.stack([orc.wilson_dslash(dims, kappa, 0, -1, U, eta[:, j]) for j in range(12)], axis=1)
        op = orc.Operator.wilson(dims, kappa, U)
        ref = orc.seed_solve_all(op, B, m_max=3000, reorth_freq=100, reorth_passes=2, tol_seed=1e-12,
                                 tol_rest=1e-8)
        sens = self_sensitivity(orc, op, B, ref, cols=(1, 6), m_max=3000, reorth_freq=100, reorth_passes=2,
                                tol=1e-12)
        # seeded residual norms and their own one-ulp sensitivity (self_sensitivity's perturbed run)
        res = [np.linalg.norm(B[:, j] - op.apply(ref["X_seeded"][:, j])) / np.linalg.norm(B[:, j])
               for j in range(1, 12)]
        Bp, Xp = self_sensitivity.perturbed
        resp = [np.linalg.norm(Bp[:, j] - op.apply(Xp[:, j])) / np.linalg.norm(Bp[:, j]) for j in range(1, 12)]
        _WORKLOAD_REF.update(dims=dims, kappa=kappa, U=U, B=B, ref=ref, sens=sens, tridiag=self_sensitivity.tridiag,
                             seeded_res=res, seeded_res_sens=max(abs(b / a - 1.0) for a, b in zip(res, resp)))
    return _WORKLOAD_REF


@pytest.mark.slow
@pytest.mark.parametrize("kernel_path", [0, 1, 2])
def test_seed_wilson_8_4_full_workload(seedlib, orc, kernel_path):
    """The benchmark workload: 8^4 lattice, kappa 0.155, links exp(0.3 i H)
    from seed 0, 12 unit point sources, b = D^H eta, seed to 1e-12 with
    reorthogonalization every 100 steps (two CGS passes), then CG to 1e-8.
    All 12 solutions against the oracle, on both kernel paths."""
    w = _workload_reference(orc)
    dims, kappa, U, B, ref = w["dims"], w["kappa"], w["U"], w["B"], w["ref"]
    prm = dict(m_max=3000, reorth_freq=100, reorth_passes=2, tol_seed=1e-12, tol_rest=1e-8, kernel_path=kernel_path)
    ctx = wilson_ctx(seedlib, dims, kappa, U, **prm)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    s_seed, s_final = w["sens"]
    self_sensitivity.tridiag = w["tridiag"]
    compare_full(ref, info1, info2, Xs, X, "wilson-8^4", seeded_tol=max(REL_X, 10 * s_seed),
                 final_tol=max(REL_X, 10 * s_final))
    # the Lanczos coefficients of the late steps inherit the same sensitivity (the
    # oracle's own alpha/beta move by about 7 percent at the last steps under
    # one-ulp noise); the early ones agree to rounding
    a, b = seedlib.seed_get_tridiag(ctx)
    assert len(a) == len(ref["seed"]["alpha"])
    assert tridiag_dev(a, b, ref["seed"]["alpha"], ref["seed"]["beta"]) <= max(1e-9, 10 * self_sensitivity.tridiag)
    assert tridiag_dev(a[:100], b[:101], ref["seed"]["alpha"][:100], ref["seed"]["beta"][:101]) < 1e-9
    # The seeded vectors themselves depend on rounding between reorthogonalizations
    # (Sec. 3), but what seeding achieves -- each system's seeded residual norm
    # ||b^j - A x^j_seed|| / ||b^j||, computed here with the oracle's operator -- does
    # not: the oracle's own values move by < 2e-4 relative under one-ulp noise on B.
    op = orc.Operator.wilson(dims, kappa, U)
    for j in range(1, 12):
        r_gpu = np.linalg.norm(B[:, j] - op.apply(Xs[:, j])) / np.linalg.norm(B[:, j])
        r_orc = w["seeded_res"][j - 1]
        assert abs(r_gpu / r_orc - 1.0) <= max(1e-6, 10 * w["seeded_res_sens"]), (j, r_gpu, r_orc)


_TIGHT_REF = {}


@pytest.mark.slow
@pytest.mark.parametrize("kernel_path", [0, 1])
def test_seed_wilson_8_4_workload_tight_rest(seedlib, orc, kernel_path):
    """The benchmark workload with the remaining systems solved to 1e-12
    instead of 1e-8, on both sides.  Then every final solution is within
    cond(A) x 1.5e-12 of the exact one (cond(A) = 584 from the oracle's Ritz
    values), the oracle's own solutions move by ~4e-12 under one-ulp noise on B,
    and the GPU's are held element-wise (per column, relative to its largest
    entry) and column-norm-wise to the benchmark spec's 1e-9 -- the bound the 1e-8
    run cannot carry because its solutions inherit the seeding's rounding."""
    import os
    w = _workload_reference(orc)
    dims, kappa, U, B = w["dims"], w["kappa"], w["U"], w["B"]
    if not _TIGHT_REF:
        op = orc.Operator.wilson(dims, kappa, U)
        orc.set_threads(os.cpu_count() or 1)      # same bits on any number of threads
        _TIGHT_REF["ref"] = orc.seed_solve_all(op, B, m_max=3000, reorth_freq=100, reorth_passes=2,
                                               tol_seed=1e-12, tol_rest=1e-12)
        orc.set_threads(1)
    ref = _TIGHT_REF["ref"]
    prm = dict(m_max=3000, reorth_freq=100, reorth_passes=2, tol_seed=1e-12, tol_rest=1e-12,
               kernel_path=kernel_path)
    ctx = wilson_ctx(seedlib, dims, kappa, U, **prm)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    seedlib.seed_destroy(ctx)
    assert info1[0]["iters"] == ref["seed"]["iters"]
    assert relerr(X[:, 0], ref["X"][:, 0]) < REL_X
    for j, r in enumerate(ref["rest"], start=1):
        g = info2[j]
        assert g["converged"] == 1 and g["true_relres"] <= 1.5e-12, (j, g)
        assert abs(g["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"]), (j, g["iters"], r["iters"])
        assert relerr(X[:, j], r["x"]) <= REL_X, (j, relerr(X[:, j], r["x"]))
        assert np.abs(X[:, j] - r["x"]).max() <= REL_X * np.abs(r["x"]).max(), j


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_padded_leading_dimension_and_single_rhs(seedlib, orc):
    rp, ci, v = I.laplacian_2d_csr(21, 17)
    n = 21 * 17
    B = I.gaussian_rhs(n, 1, seed=3)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=n, reorth_freq=3, tol_seed=1e-10)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B, ld=n + 13)
    ref = orc.seed_first(orc.Operator.csr(rp, ci, v), B, m_max=n, reorth_freq=3, tol=1e-10)
    assert info1[0]["iters"] == ref["iters"]
    assert relerr(X[:, 0].real, ref["X"][:, 0].real) < REL_X
    assert len(info2) == 1


def test_zero_rhs_and_initial_guess(seedlib, orc):
    """b^1 = 0: the seed system is solved by x = 0 with no Lanczos step; a
    nonzero initial guess (x0_zero = 0) costs one mvp per system and gives
    the oracle's result."""
    rp, ci, v = I.laplacian_2d_csr(16, 16)
    n = 256
    B = I.gaussian_rhs(n, 3, seed=4)
    B0 = B.copy()
    B0[:, 0] = 0.0
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=n, reorth_freq=1, tol_seed=1e-12)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B0)
    assert info1[0]["iters"] == 0 and info1[0]["converged"] == 1
    assert np.abs(X[:, 0]).max() == 0.0
    ref = orc.seed_solve_all(orc.Operator.csr(rp, ci, v), B0, m_max=n, reorth_freq=1)
    for j, r in enumerate(ref["rest"], start=1):
        assert relerr(X[:, j].real, r["x"].real) < 1e-6 and info2[j]["converged"]
    # initial guess
    X0 = I.gaussian_rhs(n, 3, seed=9)
    ctx2 = csr_ctx(seedlib, rp, ci, v, m_max=n, reorth_freq=2, tol_seed=1e-12, x0_zero=0)
    Bd, Xd = dev_cols(B), dev_cols(X0)
    info = seedlib.seed_solve_first(ctx2, Bd, Xd)
    torch.cuda.synchronize()
    op = orc.Operator.csr(rp, ci, v)
    r = orc.seed_first(op, B, X0=X0, m_max=n, reorth_freq=2, tol=1e-12)
    assert info[0]["iters"] == r["iters"]
    Xg = host_cols(Xd).real
    assert relerr(Xg[:, 0], r["X"][:, 0].real) < REL_X
    sens = seeded_only_sensitivity(orc, op, B, X0=X0, m_max=n, reorth_freq=2, tol=1e-12)
    assert relerr(Xg[:, 1:], r["X"][:, 1:].real) < max(REL_X, 10 * sens)


def test_mmax_reached_and_not_spd(seedlib, orc):
    d = np.linspace(0.01, 1.0, 300)
    rp, ci, v = I.diagonal_csr(d)
    B = I.gaussian_rhs(300, 2, seed=1)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=20, reorth_freq=0, tol_seed=1e-12)
    info1, _, _, X = run_gpu(seedlib, ctx, B, rest=False)
    assert info1[0]["iters"] == 20 and info1[0]["converged"] == 0
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_first(op, B, m_max=20, reorth_freq=0, tol=1e-12)
    assert relerr(X[:, 0].real, ref["X"][:, 0].real) < REL_X
    sens = seeded_only_sensitivity(orc, op, B, m_max=20, reorth_freq=0, tol=1e-12)
    assert relerr(X[:, 1:].real, ref["X"][:, 1:].real) < max(REL_X, 10 * sens)
    # an indefinite matrix makes delta_i <= 0: status, not a fault
    dn = d.copy()
    dn[:150] *= -1.0
    ctx2 = csr_ctx(seedlib, *I.diagonal_csr(dn), m_max=300, reorth_freq=0)
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_solve_first(ctx2, dev_cols(B), dev_cols(np.zeros_like(B)))
    assert e.value.status == seedlib.SEED_ENOTSPD


def test_deterministic(seedlib):
    dims, kappa = (4, 4, 4, 4), 0.15
    U = I.random_su3_links(dims, 0.3, seed=1)
    B = I.gaussian_rhs(12 * 256, 3, seed=2, complex_=True)
    ctx = wilson_ctx(seedlib, dims, kappa, U, m_max=500, reorth_freq=10, tol_seed=1e-12)
    out = [run_gpu(seedlib, ctx, B)[3] for _ in range(2)]
    assert np.array_equal(out[0], out[1])


def test_project_matches_dense_formula(seedlib, orc):
    """seed_project: x = V T^{-1} V^H b over the kept basis equals the same
    formula evaluated with the oracle's basis and tridiagonal.  A 20x19 grid
    has distinct eigenvalues (smallest gap 1.5e-4), so the basis itself is
    reproducible to rounding and the strict bound applies."""
    rp, ci, v = I.laplacian_2d_csr(20, 19)
    n = 380
    B = I.gaussian_rhs(n, 2, seed=6)
    Bn = I.gaussian_rhs(n, 3, seed=7)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=n, reorth_freq=1, tol_seed=1e-10, keep_basis=1)
    run_gpu(seedlib, ctx, B, rest=False)
    Xd = dev_cols(np.zeros_like(Bn))
    seedlib.seed_project(ctx, dev_cols(Bn), Xd)
    torch.cuda.synchronize()
    Xp = host_cols(Xd).real
    ref = orc.seed_first(orc.Operator.csr(rp, ci, v), B, m_max=n, reorth_freq=1, tol=1e-10, keep_V=True)
    m = ref["iters"]
    V = ref["V"].real
    T = np.diag(ref["alpha"]) + np.diag(ref["beta"][1:m], 1) + np.diag(ref["beta"][1:m], -1)
    for j in range(3):
        xr = V @ np.linalg.solve(T, V.T @ Bn[:, j])
        assert relerr(Xp[:, j], xr) < REL_X


def test_host_pointer_rejected(seedlib):
    rp, ci, v = I.laplacian_2d_csr(8, 8)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=10)
    L = seedlib.lib()
    host = np.zeros(64)
    st = L.seed_solve_first(ctx.handle, host.ctypes.data, 64, host.ctypes.data, 64, 1, None)
    assert st == seedlib.SEED_EINVAL
    Bd = dev_cols(np.ones((64, 1)))
    st = L.seed_solve_first(ctx.handle, Bd.data_ptr(), 32, Bd.data_ptr(), 64, 1, None)
    assert st == seedlib.SEED_EINVAL   # ld < n


@pytest.mark.parametrize("precision", [0, 1])
def test_long_vectors_two_level_reductions(seedlib, orc, precision):
    """n = 512^2 (shifted 2-d Laplacian, shift 0.5): the single-vector kernels
    run with more than one block per SM and the seed dot products reduce in
    two levels (groups of 32 blocks, then the groups).  FP64: the seed steps
    equal and x^1 within 1e-9 of the oracle's; both precisions: every true
    residual within its tolerance and the seeded CG counts within 5 %."""
    rp, ci, v = I.shifted_laplacian_2d_csr(512, 512, 0.5)
    n = 512 * 512
    B = I.gaussian_rhs(n, 3, seed=9)
    prm = dict(m_max=400, reorth_freq=20, tol_seed=1e-10, tol_rest=1e-8, precision=precision, kernel_path=1)
    ctx = csr_ctx(seedlib, rp, ci, v, **prm)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, m_max=400, reorth_freq=20, tol_seed=1e-10, tol_rest=1e-8)
    if precision == 0:
        assert info1[0]["iters"] == ref["seed"]["iters"]
        assert relerr(X[:, 0].real, ref["seed"]["X"][:, 0].real) < REL_X
    for j in range(3):
        tol = 1e-10 if j == 0 else 1e-8
        rr = np.linalg.norm(B[:, j] - op.apply(X[:, j].real).real) / np.linalg.norm(B[:, j])
        assert rr <= 1.5 * tol, (j, rr)
    for j, r in enumerate(ref["rest"], start=1):
        assert abs(info2[j]["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"]), (j, info2[j]["iters"], r["iters"])


@pytest.mark.parametrize("nrhs,freq", [(17, 1), (64, 1), (64, 10)])
def test_many_rhs_multichunk_dots(seedlib, orc, nrhs, freq):
    """nrhs = 17 (just past the persistent kernels' 16) and 64 (the maximum):
    the seed dot products run in chunks of 15 systems (5 chunks at 64).  20x19
    Laplacian (distinct eigenvalues), Gaussian right-hand sides, full
    reorthogonalization (freq 1: the streaming seeding) or every 10 steps (the
    blocked seeding: 63 seeded systems in sixteen 4-column tiles of G, on the
    persistent CSR run): the seed's steps equal and x^1 within 1e-9; every
    seeded x^j within max(1e-9, 10 x the oracle's one-ulp sensitivity); every
    CG count within 5 % and every true residual within 1.5 tol."""
    rp, ci, v = I.laplacian_2d_csr(20, 19)
    n = 380
    B = I.gaussian_rhs(n, nrhs, seed=11)
    prm = dict(m_max=400, reorth_freq=freq, tol_seed=1e-12, tol_rest=1e-8)
    ctx = csr_ctx(seedlib, rp, ci, v, **prm)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, m_max=400, reorth_freq=freq, tol_seed=1e-12, tol_rest=1e-8)
    assert info1[0]["iters"] == ref["seed"]["iters"]
    assert relerr(X[:, 0].real, ref["seed"]["X"][:, 0].real) < REL_X
    sens = seeded_only_sensitivity(orc, op, B, m_max=400, reorth_freq=freq, tol=1e-12)
    assert relerr(Xs[:, 1:].real, ref["X_seeded"][:, 1:].real) < max(REL_X, 10 * sens)
    for j, r in enumerate(ref["rest"], start=1):
        assert abs(info2[j]["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"]), (j, info2[j]["iters"], r["iters"])
        rr = np.linalg.norm(B[:, j] - op.apply(X[:, j].real).real) / np.linalg.norm(B[:, j])
        assert rr <= 1.5e-8, (j, rr)


def test_too_many_rhs_rejected(seedlib):
    rp, ci, v = I.laplacian_2d_csr(8, 8)
    ctx = csr_ctx(seedlib, rp, ci, v, m_max=10)
    B = dev_cols(I.gaussian_rhs(64, 65, seed=1))
    X = dev_cols(np.zeros((64, 65)))
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_solve_first(ctx, B, X)
    assert e.value.status == seedlib.SEED_EINVAL
