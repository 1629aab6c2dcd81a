"""The mixed solver's tiled FP32 layout (seed_apply ops 6 and 7), written
out on the host: component k = 3*spin + colour of site s at complex index
((s // 32) * 12 + k) * 32 + s % 32 of a column of 384 * ceil(sites / 32)."""
import numpy as np


def to_tiled(X, sites):
    """Site-major columns (n x c, n = 12 sites) -> the solver's tiled FP32
    layout: component k of site s at ((s // 32) * 12 + k) * 32 + s % 32."""
    tiles, c = (sites + 31) // 32, X.shape[1]
    P = np.zeros((tiles * 32, 12, c), dtype=X.dtype)
    P[:sites] = X.reshape(sites, 12, c)
    return np.ascontiguousarray(P.reshape(tiles, 32, 12, c).transpose(0, 2, 1, 3)).reshape(tiles * 384, c)


def from_tiled(T, sites):
    """Inverse of to_tiled: (site-major columns, the padding sites' values)."""
    tiles, c = (sites + 31) // 32, T.shape[1]
    P = T.reshape(tiles, 12, 32, c).transpose(0, 2, 1, 3).reshape(tiles * 32, 12, c)
    return P[:sites].reshape(sites * 12, c), P[sites:]
