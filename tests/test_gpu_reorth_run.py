"""The one-launch seed run of small real CSR problems that reorthogonalize
every 1 to 7 steps (Sec. 3, the streaming form of the seeding), against the
oracle on its launch shapes: 16 rows per block with a ragged last block and
the most right-hand sides the run takes (16), 32 rows per block (more than
304 blocks of 16 would be needed) with a ragged last block and one
Gram-Schmidt pass, the largest size the run takes, and the first size past it
(the step kernels run instead).  Reorthogonalization every 3 and 7 steps
mixes reorthogonalizing steps (eight grid barriers) with plain ones (two).

Checks: the seed run's step count equals the oracle's, x^1 within 1e-9, the
seeded x^2.. within max(1e-9, 10 x the oracle's one-ulp sensitivity), the
kept basis orthonormal to 1e-12, alpha and beta within 1e-9 of the oracle's,
and the CG on the seeded systems as in the other parity tests.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I
from test_gpu_parity import REL_X, compare_full, csr_ctx, run_gpu, self_sensitivity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("side,freq,passes,nrhs", [
    (61, 1, 2, 16),    # n = 3721: 233 blocks of 16 rows, the last with 9
    (70, 3, 1, 5),     # n = 4900: 16-row blocks would need 307 > 304, so 154 blocks of 32, the last with 4
    (98, 7, 2, 3),     # n = 9604: 301 blocks of 32
    (99, 2, 2, 2),     # n = 9801: past the run's limit, step kernels
])
def test_reorth_run_matches_oracle(seedlib, orc, side, freq, passes, nrhs):
    rp, ci, v = I.laplacian_2d_csr(side, side)
    n = side * side
    B = I.gaussian_rhs(n, nrhs, seed=side)
    kw = dict(m_max=2000, reorth_freq=freq, reorth_passes=passes)
    ctx = csr_ctx(seedlib, rp, ci, v, tol_seed=1e-12, tol_rest=1e-8, keep_basis=1, **kw)
    info1, info2, Xs, X = run_gpu(seedlib, ctx, B)
    op = orc.Operator.csr(rp, ci, v)
    ref = orc.seed_solve_all(op, B, tol_seed=1e-12, tol_rest=1e-8, **kw)
    s_seed, s_final = self_sensitivity(orc, op, B, ref, cols=(1,), tol=1e-12, **kw)
    compare_full(ref, info1, info2, Xs.real, X.real, "lap%d-f%d" % (side, freq),
                 seeded_tol=max(REL_X, 10 * s_seed), final_tol=max(REL_X, 10 * s_final))
    a, b = seedlib.seed_get_tridiag(ctx)
    assert np.abs(a - ref["seed"]["alpha"]).max() < 1e-9 * np.abs(ref["seed"]["alpha"]).max()
    assert np.abs(b - ref["seed"]["beta"]).max() < 1e-9 * np.abs(ref["seed"]["beta"]).max()
    m = info1[0]["iters"]
    V = seedlib.seed_get_basis(ctx, m)
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-12
    seedlib.seed_destroy(ctx)


def test_reorth_run_agrees_with_step_kernels(seedlib):
    """kernel_path 0 (the one-launch run) and 1 (step kernels) on the 64x64
    Laplacian with full reorthogonalization: the same step count, and the same
    x^1 and seeded x^j up to rounding."""
    rp, ci, v = I.laplacian_2d_csr(64, 64)
    B = I.gaussian_rhs(4096, 4, seed=0)
    out = {}
    for kp in (0, 1):
        ctx = csr_ctx(seedlib, rp, ci, v, m_max=4096, reorth_freq=1, tol_seed=1e-12, kernel_path=kp)
        info1, _, Xs, _ = run_gpu(seedlib, ctx, B, rest=False)
        out[kp] = (info1[0]["iters"], Xs.real)
        seedlib.seed_destroy(ctx)
    assert out[0][0] == out[1][0]
    x0, x1 = out[0][1], out[1][1]
    assert np.linalg.norm(x0[:, 0] - x1[:, 0]) <= 1e-10 * np.linalg.norm(x1[:, 0])
    assert np.linalg.norm(x0[:, 1:] - x1[:, 1:]) <= 1e-8 * np.linalg.norm(x1[:, 1:])


def test_reorth_run_stops_at_mmax_and_on_indefinite(seedlib, orc):
    """The one-launch run's other stops: m_max reached (20 steps of a 300-entry
    diagonal, reorthogonalization every 2 steps, one right-hand side and two),
    x^1 as the oracle's after the same 20 steps; an indefinite matrix makes
    delta_i <= 0 inside the launch: SEED_ENOTSPD, not a fault."""
    from test_gpu_parity import dev_cols, seeded_only_sensitivity, relerr
    d = np.linspace(0.01, 1.0, 300)
    rp, ci, v = I.diagonal_csr(d)
    op = orc.Operator.csr(rp, ci, v)
    for nrhs in (1, 2):
        B = I.gaussian_rhs(300, nrhs, seed=1)
        ctx = csr_ctx(seedlib, rp, ci, v, m_max=20, reorth_freq=2, tol_seed=1e-12)
        info1, _, _, X = run_gpu(seedlib, ctx, B, rest=False)
        assert info1[0]["iters"] == 20 and info1[0]["converged"] == 0
        ref = orc.seed_first(op, B, m_max=20, reorth_freq=2, tol=1e-12)
        assert relerr(X[:, 0].real, ref["X"][:, 0].real) < REL_X
        if nrhs > 1:
            sens = seeded_only_sensitivity(orc, op, B, m_max=20, reorth_freq=2, tol=1e-12)
            assert relerr(X[:, 1:].real, ref["X"][:, 1:].real) < max(REL_X, 10 * sens)
        seedlib.seed_destroy(ctx)
    dn = d.copy()
    dn[:150] *= -1.0
    ctx2 = csr_ctx(seedlib, *I.diagonal_csr(dn), m_max=300, reorth_freq=1)
    B = I.gaussian_rhs(300, 2, seed=1)
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_solve_first(ctx2, dev_cols(B), dev_cols(np.zeros_like(B)))
    assert e.value.status == seedlib.SEED_ENOTSPD
    seedlib.seed_destroy(ctx2)
