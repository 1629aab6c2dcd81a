"""Host-side layout logic (no GPU): the tiled FP32 layout of the mixed path
against the index formula that include/seed.h documents, and the binding's
column length for it."""
import numpy as np
import pytest

from tiled_layout import from_tiled, to_tiled


@pytest.mark.parametrize("sites", [1, 31, 32, 33, 256, 69360, 73695])
def test_tiled_layout_matches_documented_formula(sites):
    rng = np.random.default_rng(sites)
    X = rng.standard_normal((12 * sites, 2)) + 1j * rng.standard_normal((12 * sites, 2))
    T = to_tiled(X, sites)
    tiles = (sites + 31) // 32
    assert T.shape == (384 * tiles, 2)
    s = np.arange(sites)
    for k in range(12):
        idx = ((s // 32) * 12 + k) * 32 + s % 32
        assert np.array_equal(T[idx], X[12 * s + k])
    Y, pad = from_tiled(T, sites)
    assert np.array_equal(Y, X) and np.all(pad == 0) and pad.shape[0] == 32 * tiles - sites


def test_binding_tiled_length():
    pytest.importorskip("torch")
    from paper_0810_0330_gb300.binding import wilson_tiled_length
    for sites in (1, 31, 32, 33, 4096, 69360, 131072):
        assert wilson_tiled_length(12 * sites) == 384 * ((sites + 31) // 32)
