"""Differentiable seed solve for the Wilson normal operator (torch.autograd).

    X = WilsonSeedSolve.apply(kappa, B, links, dims, bc_t, params, seeded_backward)

solves A(kappa) X = B with A = D^H D by the seed method (seed_solve_first on
column 1, seed_solve_rest on the others), keeping the Lanczos basis.  The
backward pass solves the adjoint systems A Lambda = G (A is Hermitian) for the
incoming gradient G = dL/dX: their initial guesses are the Galerkin projection
of G over the forward basis (seed_project, Sec. 2.1's projection reused for new
right-hand sides), finished by lockstep CG (seed_solve_cg) -- when
seeded_backward is set.  It is off by default: the projection costs two FP64
passes over the forward basis (V^H G and V c, bound by the FP64 pipe on this
GPU) and on the 16^4 adjoint workload (kappa 0.150, 8 right-hand sides) it
saved only 3 % of the backward CG iterations, so the seeded backward took
longer (467 ms against 453 ms unseeded); by default the adjoint solves start
from zero and the forward basis is not kept.  Then

    dL/dB     = Lambda,
    dL/dkappa = -sum_j Re <Lambda_j, (dA/dkappa) X_j>   (seed_grad_kappa),

in PyTorch's conjugate-Wirtinger convention (dL = Re <grad, dz>).  With
params["precision"] = 1 both the forward and the adjoint solves run in mixed
precision (FP32 iterations, FP64 reliable updates, the same FP64 tolerances);
the FP32 basis is not used for the backward projection, so those adjoint
solves start from zero.  Every step runs in the library's kernels; this module
only marshals tensors.
"""
from __future__ import annotations

import torch

from . import binding as S


def _colmajor(t: torch.Tensor) -> torch.Tensor:
    """The same values as an (n, p) column-major tensor (stride (1, n))."""
    return t.t().contiguous().t() if t.stride(0) != 1 else t


class WilsonSeedSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa: torch.Tensor, B: torch.Tensor, links: torch.Tensor, dims, bc_t: int = 0,
                params: dict | None = None, seeded_backward: bool = False):
        prm = dict(params or {})
        prm["keep_basis"] = 1 if seeded_backward else 0
        p = S.seed_params_default(**prm)
        sc = S.seed_create_wilson(tuple(dims), float(kappa), links, p, bc_t=bc_t)
        Bc = _colmajor(B.detach())
        X = torch.empty((Bc.shape[1], Bc.shape[0]), dtype=Bc.dtype, device=Bc.device).t()
        ctx.info_forward = [S.seed_solve_first(sc, Bc, X)[0]] + S.seed_solve_rest(sc, Bc, X)[1:]
        ctx.sc = sc
        ctx.seeded = seeded_backward and int(prm.get("precision", 0)) == 0
        ctx.kappa_meta = (kappa.dtype, kappa.device) if isinstance(kappa, torch.Tensor) else (torch.float64, "cpu")
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX: torch.Tensor):
        (X,) = ctx.saved_tensors
        sc = ctx.sc
        G = _colmajor(gX.detach().to(X.dtype))
        Lam = torch.zeros_like(X.t()).t()
        if ctx.seeded:
            S.seed_project(sc, G, Lam)
        ctx.info_backward = S.seed_solve_cg(sc, G, Lam)
        gk = -S.seed_grad_kappa(sc, Lam, X)
        gkappa = torch.tensor(gk, dtype=ctx.kappa_meta[0], device=ctx.kappa_meta[1])
        return gkappa, Lam, None, None, None, None, None


def wilson_seed_solve(kappa: torch.Tensor, B: torch.Tensor, links: torch.Tensor, dims, bc_t: int = 0,
                      params: dict | None = None, seeded_backward: bool = False) -> torch.Tensor:
    """X = A(kappa)^{-1} B with gradients for kappa and B (see module docstring)."""
    return WilsonSeedSolve.apply(kappa, B, links, dims, bc_t, params, seeded_backward)
