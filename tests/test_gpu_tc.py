"""The tensor-core (tcgen05, TF32 with hi/lo split) form of the mixed-precision
seeding products G = V^H R (Sec. 3: every Lanczos vector projected onto every
other right-hand side), through the C ABI's seed_block_products.

 * Small-integer data (exact in TF32, products and sums exact in FP32 and
   FP64): G must equal the exact integer result bit for bit -- any slip in the
   operand layout, the hi/lo or re/im bookkeeping, the tile offsets or the
   reduction shows up exactly.
 * Random FP32 data: G element-wise against FP64 products of the same FP32
   numbers, |G - G64| <= 2e-5 s_qj with s_qj = sqrt(sum_e |v_eq r_ej|^2), the
   scale of rounding errors in a sum of n products (the split keeps ~2^-21 per
   product; the FP32 accumulation over 512 elements per drain gives a few 1e-6
   at the largest entries; plain TF32 operands would give ~2e-4), on shapes
   with ragged step and system tiles, one and many CTAs, and the 16^3 x 32
   workload's block (25 steps x 11 systems).
 * Bitwise reproducible across calls (fixed CTA ranges, fixed-order sums).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cols(a):
    """numpy complex64 (n, k) -> CUDA tensor (n, k), column-major, ld = n."""
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def _exact_case(n, k, nr, seed):
    rng = np.random.default_rng(seed)
    V = (rng.integers(-2, 3, (n, k)) + 1j * rng.integers(-2, 3, (n, k))).astype(np.complex64)
    R = (rng.integers(-2, 3, (n, nr)) + 1j * rng.integers(-2, 3, (n, nr))).astype(np.complex64)
    return V, R


@pytest.mark.parametrize("n,k,nr", [(128, 1, 1), (384 * 5, 7, 3), (4096, 32, 16), (128 * 150, 33, 17),
                                    (128 * 489, 128, 63)])
def test_tc_products_exact_on_small_integers(seedlib, n, k, nr):
    V, R = _exact_case(n, k, nr, seed=n + k)
    G, _ = seedlib.seed_block_products(_cols(V), _cols(R))
    exact = V.astype(np.complex128).conj().T @ R.astype(np.complex128)
    assert np.array_equal(G, exact), np.abs(G - exact).max()


@pytest.mark.parametrize("n,k,nr", [(128 * 7, 5, 2), (49152, 25, 11), (49152, 100, 40), (1572864, 25, 11)])
def test_tc_products_match_fp64(seedlib, n, k, nr):
    rng = np.random.default_rng(7 + k)
    V = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))).astype(np.complex64)
    R = (rng.standard_normal((n, nr)) + 1j * rng.standard_normal((n, nr))).astype(np.complex64)
    V /= np.linalg.norm(V, axis=0)
    G, _ = seedlib.seed_block_products(_cols(V), _cols(R))
    V64, R64 = V.astype(np.complex128), R.astype(np.complex128)
    G64 = V64.conj().T @ R64
    scale = np.sqrt((np.abs(V64) ** 2).T @ (np.abs(R64) ** 2))
    err = (np.abs(G - G64) / scale).max()
    assert err <= 2e-5, err
    # the split matters: plain TF32 rounding of the operands would be far off
    def tf32(x):
        b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x1000) & 0xFFFFE000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    Gt = (tf32(V.real) + 1j * tf32(V.imag)).conj().T @ (tf32(R.real) + 1j * tf32(R.imag))
    assert (np.abs(Gt - G64) / scale).max() > 5 * max(err, 2e-6)


def test_tc_products_reproducible_and_padded_ld(seedlib):
    n, k, nr = 128 * 250, 20, 9
    rng = np.random.default_rng(3)
    V = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))).astype(np.complex64)
    R = (rng.standard_normal((n, nr)) + 1j * rng.standard_normal((n, nr))).astype(np.complex64)
    G1, _ = seedlib.seed_block_products(_cols(V), _cols(R))
    G2, ms = seedlib.seed_block_products(_cols(V), _cols(R), reps=3)
    assert np.array_equal(G1, G2) and ms > 0.0
    # columns with a padded leading dimension (ld = n + 32) give the same bits
    buf = torch.zeros((k, n + 32), dtype=torch.complex64, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()
    G3, _ = seedlib.seed_block_products(buf[:, :n].t(), _cols(R))
    assert np.array_equal(G1, G3)


def test_tc_products_reject_bad_shapes(seedlib):
    V = torch.zeros((2, 100), dtype=torch.complex64, device="cuda").t()   # (100, 2), column-major
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_block_products(V, V)             # n not a multiple of 128
    assert e.value.status == seedlib.SEED_EINVAL
    V = torch.zeros((129, 64), dtype=torch.complex64, device="cuda").t()   # (64, 129): k = 129 > 128
    with pytest.raises(seedlib.SeedError):
        seedlib.seed_block_products(V, V[:, :1])
