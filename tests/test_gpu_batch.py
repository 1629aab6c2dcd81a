"""Batched uneven problems (seed_batch_solve) and the CSR launch-shape autotuner.

 * A batch of independent shifted 2-d / 3-d Laplacians with different sizes
   and right-hand side counts gives, problem by problem, bitwise the results
   of solving each problem alone with the same parameters, on the step-kernel
   path (kernel_path 1) and with persistent seed runs side by side
   (kernel_path 0): the batch only changes when the work runs.
 * Two problems of the batch against the oracle: seed step counts equal,
   CG iteration counts within 5 %, true residuals <= 1.5 tol_rest.
 * Every autotuned launch shape gives the apply to 1e-13 of the oracle's.
"""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRM = dict(m_max=600, reorth_freq=25, tol_seed=1e-10, tol_rest=1e-8, kernel_path=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().t()


def host(t):
    return t.t().cpu().numpy().T


def make(seedlib, p, **prm):
    rp, ci, v, B = I.batch_problem_arrays(p)
    ctx = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                  torch.from_numpy(v).cuda(), seedlib.seed_params_default(**prm))
    return ctx, (rp, ci, v), B


@pytest.mark.parametrize("kernel_path", [1, 0])
def test_batch_equals_solo_solves_and_oracle(seedlib, orc, kernel_path):
    probs = I.batch_problems(count=7, n_min=300, n_max=20000, seed=3)
    probs[1] = dict(probs[1], nrhs=1)          # a single right-hand side in the mix
    prm = dict(PRM, kernel_path=kernel_path)
    ctxs, ops, Bs, Xs = [], [], [], []
    for p in probs:
        c, op, B = make(seedlib, p, **prm)
        ctxs.append(c), ops.append(op), Bs.append(dev(B))
        Xs.append(torch.full_like(Bs[-1].t(), 7.0).t())   # overwritten (x0_zero)
    infos = seedlib.seed_batch_solve(ctxs, Bs, Xs, workers=4)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        c, _, _ = make(seedlib, p, **prm)
        X = torch.zeros_like(Bs[i].t()).t()
        a = seedlib.seed_solve_first(c, Bs[i], X)
        b = seedlib.seed_solve_rest(c, Bs[i], X)
        torch.cuda.synchronize()
        assert torch.equal(X, Xs[i]), i
        assert infos[i][0]["iters"] == a[0]["iters"]
        assert [x["iters"] for x in infos[i][1:]] == [x["iters"] for x in b[1:]]
    for i in (0, 3):
        B = host(Bs[i])
        op = orc.Operator.csr(*ops[i])
        ref = orc.seed_solve_all(op, B, m_max=600, reorth_freq=25, tol_seed=1e-10, tol_rest=1e-8)
        assert infos[i][0]["iters"] == ref["seed"]["iters"]
        X = host(Xs[i]).real
        for j, r in enumerate(ref["rest"], start=1):
            assert abs(infos[i][j]["iters"] - r["iters"]) <= max(1, 0.05 * r["iters"])
            assert np.linalg.norm(B[:, j] - op.apply(X[:, j]).real) <= 1.5e-8 * np.linalg.norm(B[:, j])


def test_batch_one_launch_reorthogonalizing_runs_side_by_side(seedlib, orc):
    """Small problems that reorthogonalize every 3 steps run their whole seed
    run as one cooperative launch each (up to 4 at a time from the batch's
    workers): bitwise the solo results, and one problem against the oracle."""
    probs = I.batch_problems(count=6, n_min=300, n_max=9000, seed=11)
    prm = dict(m_max=600, reorth_freq=3, tol_seed=1e-10, tol_rest=1e-8, kernel_path=0)
    ctxs, ops, Bs, Xs = [], [], [], []
    for p in probs:
        c, op, B = make(seedlib, p, **prm)
        ctxs.append(c), ops.append(op), Bs.append(dev(B))
        Xs.append(torch.zeros_like(Bs[-1].t()).t())
    infos = seedlib.seed_batch_solve(ctxs, Bs, Xs, workers=4)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        c, _, _ = make(seedlib, p, **prm)
        X = torch.zeros_like(Bs[i].t()).t()
        a = seedlib.seed_solve_first(c, Bs[i], X)
        seedlib.seed_solve_rest(c, Bs[i], X)
        torch.cuda.synchronize()
        assert torch.equal(X, Xs[i]), i
        assert infos[i][0]["iters"] == a[0]["iters"]
    B = host(Bs[0])
    op = orc.Operator.csr(*ops[0])
    ref = orc.seed_solve_all(op, B, m_max=600, reorth_freq=3, tol_seed=1e-10, tol_rest=1e-8)
    assert infos[0][0]["iters"] == ref["seed"]["iters"]
    X = host(Xs[0]).real
    for j in range(1, B.shape[1]):
        assert np.linalg.norm(B[:, j] - op.apply(X[:, j]).real) <= 1.5e-8 * np.linalg.norm(B[:, j])


def test_batch_reports_failing_problem(seedlib):
    probs = I.batch_problems(count=3, n_min=300, n_max=3000, seed=5)
    ctxs, Bs, Xs = [], [], []
    for p in probs:
        c, _, B = make(seedlib, p, **PRM)
        ctxs.append(c), Bs.append(dev(B)), Xs.append(torch.zeros_like(dev(B).t()).t())
    # problem 1: an indefinite matrix (negative shift) -> SEED_ENOTSPD, the others still solve
    rp, ci, v, B = I.batch_problem_arrays(probs[1])
    v = v.copy()
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    v[ci == rows] -= 20.0
    ctxs[1] = seedlib.seed_create_csr(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                                      torch.from_numpy(v).cuda(), seedlib.seed_params_default(**PRM))
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_batch_solve(ctxs, Bs, Xs)
    assert "problem 1" in str(e.value)
    with pytest.raises(ValueError):
        seedlib.seed_batch_solve(ctxs, Bs[:2], Xs)
    with pytest.raises(seedlib.SeedError):
        seedlib.seed_batch_solve([ctxs[0], ctxs[0]], [Bs[0], Bs[0]], [Xs[0], Xs[0]])


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_shape_apply_matches_oracle(seedlib, orc, precision):
    p = I.batch_problems(count=1, n_min=40000, n_max=40001, seed=7)[0]
    c, op, B = make(seedlib, p, m_max=4, autotune=1, precision=precision)
    st = seedlib.seed_get_stats(c)
    assert (st["csr_tpr"], st["csr_block"]) in [(1, 256), (1, 128), (1, 512), (2, 256), (4, 256), (8, 256)]
    X = B[:, :2]
    Y = torch.zeros_like(dev(X).t()).t()
    seedlib.seed_apply(c, 0, dev(X), Y)
    torch.cuda.synchronize()
    o = orc.Operator.csr(*op)
    for j in range(2):
        ref = o.apply(X[:, j]).real
        assert np.abs(host(Y)[:, j] - ref).max() <= 1e-13 * np.abs(ref).max()
