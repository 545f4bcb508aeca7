"""Phase functions Phi(x, xi) in FP64 (oracle).

* FIO2D: Example 1 of the paper (Sec. 4, eq. for the 2D generalized Radon
  transform): Phi = x.xi + sqrt(c1(x)^2 xi1^2 + c2(x)^2 xi2^2) with
  c1 = (2 + sin 2pi x1 sin 2pi x2)/16, c2 = (2 + cos 2pi x1 cos 2pi x2)/16.
  The paper prints "x . xi'"; the prime is read as a typesetting slip.
* FIO3D: the 3D analogue with c_k = (2 + sin 2pi x_k cos 2pi x_{k+1})/16
  (cyclic index) — a workload of this project, not a paper example.
* FIO2D_JUMP: FIO2D + 0.5 |xi| sign(x1 - 0.5), sign(0) := +1; piecewise smooth
  with one discontinuity (the paper's setting of eq. (1) allows O(1) of them).
* DOT: x.xi (the Fourier kernel of Example 2, Sec. 4).
* DISTANCE: |x - xi|_2.  Example 3 (Sec. 4) uses h |x - xi| on a sphere mesh;
  the workloads pass the points scaled by h, which gives the same Phi.
* ZERO, SEPARABLE: K of rank one; used as pins.
* LOWRANK: Psi(i, j) = sum_t U[i,t] V[j,t], the output form of Algorithm 7.

Parity: pinned by closed forms in tests (DOT against the FFT, ZERO and
SEPARABLE against rank one) and by hand-evaluated points: FIO2D and
FIO2D_JUMP in tests/golden/phase_values.txt, FIO3D in
tests/golden/phase_values_3d.txt (points where every c_k is exact, chosen so
that a wrong cyclic index or swapped sine and cosine change the value),
DISTANCE against exact distances on the sphere mesh.
"""
from __future__ import annotations

import numpy as np

import synth


class Phase:
    """Phi evaluated on index pairs into the point sets X (rows) and W (cols)."""

    def __init__(self, family: int, X: np.ndarray, W: np.ndarray, U=None, V=None):
        self.family = family
        self.X = np.asarray(X, dtype=np.float64)
        self.W = np.asarray(W, dtype=np.float64)
        self.d = self.X.shape[1]
        self.U = None if U is None else np.asarray(U, dtype=np.float64)
        self.V = None if V is None else np.asarray(V, dtype=np.float64)
        if family == synth.PHASE_LOWRANK and (self.U is None or self.V is None):
            raise ValueError("LOWRANK phase needs U and V")

    def __call__(self, ix, iw) -> np.ndarray:
        """Phi(X[ix], W[iw]) with numpy broadcasting of the index arrays."""
        ix = np.asarray(ix)
        iw = np.asarray(iw)
        f = self.family
        if f == synth.PHASE_LOWRANK:
            return np.einsum("...t,...t->...", self.U[ix], self.V[iw])
        x = self.X[ix]
        w = self.W[iw]
        return coordinate_phase(f, x, w)


def coordinate_phase(family: int, x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Phi for coordinate arrays x (..., d) and w (..., d), broadcast together."""
    twopi = 2.0 * np.pi
    dot = np.sum(x * w, axis=-1)
    if family == synth.PHASE_DOT:
        return dot
    if family == synth.PHASE_ZERO:
        return np.zeros(np.broadcast_shapes(x.shape[:-1], w.shape[:-1]))
    if family == synth.PHASE_DISTANCE:
        return np.sqrt(np.sum((x - w) ** 2, axis=-1))
    if family == synth.PHASE_SEPARABLE:
        return np.sum(np.sin(twopi * x), axis=-1) + 0.05 * np.sum(w * w, axis=-1)
    if family in (synth.PHASE_FIO2D, synth.PHASE_FIO2D_JUMP):
        x1, x2 = x[..., 0], x[..., 1]
        c1 = (2.0 + np.sin(twopi * x1) * np.sin(twopi * x2)) / 16.0
        c2 = (2.0 + np.cos(twopi * x1) * np.cos(twopi * x2)) / 16.0
        out = dot + np.sqrt(c1 ** 2 * w[..., 0] ** 2 + c2 ** 2 * w[..., 1] ** 2)
        if family == synth.PHASE_FIO2D_JUMP:
            sgn = np.where(x1 - 0.5 >= 0.0, 1.0, -1.0)
            out = out + 0.5 * np.sqrt(np.sum(w * w, axis=-1)) * sgn
        return out
    if family == synth.PHASE_FIO3D:
        acc = np.zeros(np.broadcast_shapes(x.shape[:-1], w.shape[:-1]))
        for k in range(3):
            ck = (2.0 + np.sin(twopi * x[..., k]) * np.cos(twopi * x[..., (k + 1) % 3])) / 16.0
            acc = acc + ck ** 2 * w[..., k] ** 2
        return dot + np.sqrt(acc)
    raise ValueError(f"unknown phase family {family}")


def kernel(phase: Phase, ix, iw) -> np.ndarray:
    """K(x, xi) = exp(2 pi i Phi(x, xi)), eq. (1).

    Phi is first reduced modulo one (an exact subtraction in FP64 for
    |Phi| < 2^52), which leaves exp(2 pi i Phi) unchanged.
    """
    phi = phase(ix, iw)
    return np.exp(2j * np.pi * (phi - np.rint(phi)))
