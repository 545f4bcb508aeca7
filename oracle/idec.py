"""Linear-scaling interpolative decompositions (oracle), Sec. 3.2.

Column ID of A (m x n) from a row sample s (|s| = t k rows):
  A(s,:) Lambda = Q R,  R = [R1 R2];  T = R1(1:k,1:k)^{-1} [R1(1:k,k+1:tk) R2(1:k,:)],
  V = [I T] Lambda^T,  skeleton q = Lambda(1:k);  A ~ A(:,q) V.
Row ID of A: the column ID of A^T (plain transpose, reading M7: U = V^T with
no conjugation), A ~ U A(q,:).
Adaptive rank (Sec. 3.6): k_eps = min{k : |R(k,k)| <= eps |R(1,1)|}.  Reading:
the columns kept are the pivots strictly above eps |R(1,1)|, i.e. k_eps - 1
of them; keeping the first sub-tolerance pivot as well would make R11 as
ill-conditioned as 1/eps (1e16 for exactly low-rank blocks).  The rank is
capped by kmax (default: no cap) and by min(|s|, n).
The row sample is a Mock-Chebyshev sample (reading M6): a tensor Chebyshev
grid of ceil((tk)^(1/d)) first-kind nodes per axis over the candidates'
bounding box, each node snapped to its nearest candidate, duplicates dropped,
then topped up with seeded uniform random candidates to t k.

The pivoted QR is LAPACK's (scipy.linalg.qr with pivoting), a library step.

Parity: pinned in tests by the ID error bound ||A(s,:) - A(s,q) V|| against
|R(k+1,k+1)| and by exact reproduction of rank-one matrices.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
from scipy.spatial import cKDTree


def chebyshev_nodes(lo: np.ndarray, hi: np.ndarray, p: int) -> np.ndarray:
    """Tensor grid of p first-kind Chebyshev nodes per axis over the box [lo, hi]."""
    d = lo.size
    t = (1.0 - np.cos((2.0 * np.arange(p) + 1.0) * np.pi / (2.0 * p))) / 2.0
    axes = [lo[k] + (hi[k] - lo[k]) * t for k in range(d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def mock_chebyshev_sample(coords: np.ndarray, count: int, rng: np.random.Generator) -> np.ndarray:
    """Positions (into coords) of a Mock-Chebyshev sample of size >= min(count, len)."""
    ncand = coords.shape[0]
    if ncand <= count:
        return np.arange(ncand)
    d = coords.shape[1]
    p = int(math.ceil(count ** (1.0 / d) - 1e-12))
    nodes = chebyshev_nodes(coords.min(axis=0), coords.max(axis=0), p)
    _, nearest = cKDTree(coords).query(nodes)
    chosen = np.unique(nearest)
    if chosen.size < count:
        rest = np.setdiff1d(np.arange(ncand), chosen)
        extra = rng.choice(rest, size=count - chosen.size, replace=False)
        chosen = np.union1d(chosen, extra)
    return chosen


def column_id(Asub: np.ndarray, tol: float, kmax: int):
    """Column ID from the sampled rows Asub = A(s,:).

    Returns (skel, red, T, rdiag) with A ~ A(:,skel) [I T] re-ordered by
    (skel, red): column skel[i] is reproduced exactly, column red[j] is
    sum_i A(:,skel[i]) T[i,j].  rdiag are |R(j,j)| of the pivoted QR.
    """
    ms, n = Asub.shape
    R, P = scipy.linalg.qr(Asub, mode="r", pivoting=True)
    kk = min(ms, n)
    rdiag = np.abs(np.diag(R[:kk, :kk]))
    # number of pivots strictly above the tolerance (reading of k_eps, see module doc)
    k = int(np.count_nonzero(rdiag > tol * rdiag[0])) if rdiag[0] > 0.0 else 1
    k = max(1, min(k, kmax, kk))
    if rdiag[0] == 0.0:
        T = np.zeros((k, n - k), dtype=np.complex128)
    else:
        T = scipy.linalg.solve_triangular(R[:k, :k], R[:k, k:])
    return P[:k].copy(), P[k:].copy(), T, rdiag


def id_matrix(skel: np.ndarray, red: np.ndarray, T: np.ndarray) -> np.ndarray:
    """The interpolation matrix V = [I T] Lambda^T (k x n)."""
    k = skel.size
    n = k + red.size
    V = np.zeros((k, n), dtype=np.complex128)
    V[np.arange(k), skel] = 1.0
    V[:, red] = T
    return V
