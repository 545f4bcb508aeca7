"""Direct summation of eq. (1) and the dense kernel matrix (oracle, FP64).

g(x_i) = sum_j exp(2 pi i Phi(x_i, xi_j)) f(xi_j)   (eq. (1), Sec. 1)

The adjoint is K^H g (conjugate transpose), which the paper's Scenario 2
(Table 1: "applying K and its transpose") presumes available.

Parity: this is the definition itself.  It is pinned against the FFT closed
form (Phi = x.xi on uniform grids, ``fftcheck``) and against rank one
(Phi = 0, separable Phi) in the tests.
"""
from __future__ import annotations

import numpy as np

from .phase import Phase, kernel


def dense_kernel(phase: Phase, rows=None, cols=None) -> np.ndarray:
    """K(rows, cols) as a dense complex128 matrix (all rows/cols by default)."""
    nx = phase.X.shape[0]
    nw = phase.W.shape[0]
    r = np.arange(nx) if rows is None else np.asarray(rows)
    c = np.arange(nw) if cols is None else np.asarray(cols)
    return kernel(phase, r[:, None], c[None, :])


def direct_sum(phase: Phase, f: np.ndarray, rows=None, chunk: int = 256) -> np.ndarray:
    """g = K(rows, :) f by direct summation, f of shape (nw,) or (nw, nrhs)."""
    f = np.asarray(f, dtype=np.complex128)
    vec = f.ndim == 1
    if vec:
        f = f[:, None]
    nx = phase.X.shape[0]
    r = np.arange(nx) if rows is None else np.asarray(rows)
    out = np.empty((r.size, f.shape[1]), dtype=np.complex128)
    cols = np.arange(phase.W.shape[0])
    for s in range(0, r.size, chunk):
        blk = kernel(phase, r[s:s + chunk, None], cols[None, :])
        out[s:s + chunk] = blk @ f
    return out[:, 0] if vec else out


def direct_adjoint(phase: Phase, g: np.ndarray, cols=None, chunk: int = 256) -> np.ndarray:
    """f = K(:, cols)^H g by direct summation, g of shape (nx,) or (nx, nrhs)."""
    g = np.asarray(g, dtype=np.complex128)
    vec = g.ndim == 1
    if vec:
        g = g[:, None]
    nw = phase.W.shape[0]
    c = np.arange(nw) if cols is None else np.asarray(cols)
    out = np.empty((c.size, g.shape[1]), dtype=np.complex128)
    rows = np.arange(phase.X.shape[0])
    for s in range(0, c.size, chunk):
        blk = kernel(phase, rows[:, None], c[None, s:s + chunk])
        out[s:s + chunk] = blk.conj().T @ g
    return out[:, 0] if vec else out


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """Relative L2 error ||a - b|| / ||b||, the epsilon^b of Sec. 4."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
