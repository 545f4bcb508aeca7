"""Closed form of eq. (1) for Phi(x, xi) = x.xi on uniform grids (oracle).

With x = m/n (m in [0, n)^d) and integer xi in [-n/2, n/2)^d, eq. (1) reads
g(m) = sum_xi exp(2 pi i m.xi / n) f(xi), an inverse DFT of f after shifting
the frequency origin to index 0: g = n^d * ifftn(ifftshift(F)), where F is f
reshaped to the (n,)*d frequency grid.  The paper notes (Sec. 1) that the FFT
evaluates eq. (1) in O(N log N) for this phase.

Parity: a library FFT is the closed form; it is independent of the direct sum
and of the butterfly code, and pins both.
"""
from __future__ import annotations

import numpy as np


def fft_apply(f: np.ndarray, n: int, d: int) -> np.ndarray:
    """g on the uniform X grid (row-major order) for f on the frequency grid."""
    f = np.asarray(f, dtype=np.complex128)
    vec = f.ndim == 1
    if vec:
        f = f[:, None]
    nrhs = f.shape[1]
    F = f.T.reshape((nrhs,) + (n,) * d)
    axes = tuple(range(1, d + 1))
    G = (n ** d) * np.fft.ifftn(np.fft.ifftshift(F, axes=axes), axes=axes)
    g = G.reshape(nrhs, n ** d).T
    return g[:, 0] if vec else g
