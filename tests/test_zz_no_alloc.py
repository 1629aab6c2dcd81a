"""The allocation-free Wilson apply, for callers that cannot call cudaMalloc
while they run (a host loop being captured into a CUDA graph, a service whose
device memory is fixed at start-up, a plug-in in a framework that owns the
device heap).  It must give what the context-based seed_apply gives, on two
calls in a row (the second call finds the first call's leftovers in the shared
scratch array), with periodic and antiperiodic t, and it must accept exactly
the sizes its fixed scratch array holds.  This file is collected last so that
a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_0810_0330_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev_cols(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


@pytest.mark.parametrize("bc_t", [0, 1])
def test_noalloc_apply_matches_seed_apply_twice(seedlib, bc_t):
    for dims, ncols in (((6, 4, 4, 4), 3), ((8, 8, 8, 8), 2)):
        kappa = 0.155
        vol = int(np.prod(dims))
        n = 12 * vol
        U = torch.from_numpy(I.random_su3_links(dims, 0.3, seed=3)).cuda()
        ctx = seedlib.seed_create_wilson(dims, kappa, U, seedlib.seed_params_default(m_max=4), bc_t=bc_t)
        for call in range(2):
            X = _dev_cols(I.gaussian_rhs(n, ncols, seed=10 + call, complex_=True))
            Y_ref = torch.zeros((ncols, n), dtype=torch.complex128, device="cuda").t()
            Y = torch.full((ncols, n), complex(7.0, -7.0), dtype=torch.complex128, device="cuda").t()
            seedlib.seed_apply(ctx, 0, X, Y_ref)
            seedlib.seed_wilson_apply_noalloc(dims, kappa, U, X, Y, bc_t=bc_t)
            torch.cuda.synchronize()
            err = ((Y - Y_ref).abs().max() / Y_ref.abs().max()).item()
            assert err <= 1e-13, (dims, bc_t, call, err)
        seedlib.seed_destroy(ctx)


def test_noalloc_size_limit(seedlib):
    """8^4 needs 128 KiB of neighbour table plus 768 KiB per column: 10 columns
    fit the 8 MiB array, 11 do not and are rejected before any launch."""
    dims = (8, 8, 8, 8)
    vol = int(np.prod(dims))
    n = 12 * vol
    U = torch.from_numpy(I.random_su3_links(dims, 0.3, seed=4)).cuda()
    ctx = seedlib.seed_create_wilson(dims, 0.15, U, seedlib.seed_params_default(m_max=4))
    X = _dev_cols(I.gaussian_rhs(n, 11, seed=5, complex_=True))
    Y = torch.zeros((11, n), dtype=torch.complex128, device="cuda").t()
    Y_ref = torch.zeros((10, n), dtype=torch.complex128, device="cuda").t()
    seedlib.seed_wilson_apply_noalloc(dims, 0.15, U, X[:, :10], Y[:, :10])
    seedlib.seed_apply(ctx, 0, X[:, :10], Y_ref)
    torch.cuda.synchronize()
    assert ((Y[:, :10] - Y_ref).abs().max() / Y_ref.abs().max()).item() <= 1e-13
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_wilson_apply_noalloc(dims, 0.15, U, X, Y)
    assert e.value.status == seedlib.SEED_EINVAL and "limit" in str(e.value)
    seedlib.seed_destroy(ctx)


def test_noalloc_rejects_oversize(seedlib):
    dims = (16, 16, 16, 16)          # one column needs 12 MiB > 8 MiB
    n = 12 * int(np.prod(dims))
    U = torch.zeros((4, int(np.prod(dims)), 3, 3), dtype=torch.complex128, device="cuda")
    X = torch.zeros(n, dtype=torch.complex128, device="cuda")
    Y = torch.zeros(n, dtype=torch.complex128, device="cuda")
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_wilson_apply_noalloc(dims, 0.1, U, X, Y)
    assert e.value.status == seedlib.SEED_EINVAL and "limit" in str(e.value)
