"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the butterfly method: it only draws point
sets, coefficient vectors and sample indices from seeded generators, and names
the workloads (sizes, phase family, tolerances, seeds).  Each side (the CPU
oracle and the GPU library) evaluates phases and kernels with its own code.

Point ordering (a convention of this project; the paper does not fix it):
  * uniform X grid, d=2: x = (i/n, j/n) at index i*n + j; d=3 analogous,
    row-major (i slowest).
  * integer frequency grid, d=2: xi = (k1, k2), k in [-n/2, n/2), at index
    (k1 + n/2)*n + (k2 + n/2); d=3 analogous.
  * random point sets: rows of a PCG64(seed) draw, in the order drawn.
  * sphere mesh: the 12 vertices of the icosahedron, then the edge midpoints of
    each refinement in order of (lower vertex index, higher vertex index) of
    their edge; X is the half with z >= 0 and Omega the half with z < 0, each in
    mesh order.
Complex Gaussian CN(0,1): real and imaginary parts each N(0, 1/2).
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

# Phase family identifiers (the same numbers appear in include/midbf.h).
PHASE_FIO2D = 1        # x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), Example 1 of the paper
PHASE_FIO3D = 2        # x.xi + sqrt(sum_k c_k^2 xi_k^2), c_k=(2+sin2pi x_k cos2pi x_{k+1})/16
PHASE_FIO2D_JUMP = 3   # FIO2D + 0.5 |xi| sign(x1 - 0.5), sign(0) = +1
PHASE_DOT = 4          # x.xi
PHASE_ZERO = 5         # 0
PHASE_SEPARABLE = 6    # sum_k sin(2 pi x_k) + 0.05 sum_k xi_k^2
PHASE_LOWRANK = 7      # Psi = U V^T given per point index
PHASE_DISTANCE = 8     # |x - xi|_2 (the Helmholtz phase h |x - xi| with h folded into the points)


def uniform_grid(n: int, d: int) -> np.ndarray:
    """X = {(i/n, j/n[, l/n])}, row-major, shape (n**d, d), float64."""
    ax = np.arange(n, dtype=np.float64) / n
    mesh = np.meshgrid(*([ax] * d), indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def frequency_grid(n: int, d: int) -> np.ndarray:
    """Omega = integer grid [-n/2, n/2)^d, row-major, shape (n**d, d), float64."""
    ax = np.arange(-(n // 2), n - n // 2, dtype=np.float64)
    mesh = np.meshgrid(*([ax] * d), indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def uniform_random_points(npts: int, d: int, seed: int) -> np.ndarray:
    """npts points uniform in [0,1)^d from PCG64(seed)."""
    return np.random.default_rng(seed).random((npts, d))


def icosphere(level: int):
    """Triangular mesh of the unit sphere: the icosahedron refined `level` times.

    Each refinement splits every triangle into four through its edge midpoints
    and moves the new vertices radially onto the sphere.  Returns (vertices
    (V, 3) float64, faces (F, 3) int64) with V = 10 * 4**level + 2 and
    F = 20 * 4**level.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = len(v) + inv.reshape(3, len(f))          # midpoint index of edges (01, 12, 20)
        v = np.concatenate([v, mid])
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        m01, m12, m20 = m[0], m[1], m[2]
        f = np.concatenate([np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
                            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)])
    return v, f


def hemispheres(vertices: np.ndarray):
    """(X, Omega): the vertices with z >= 0 and those with z < 0, in mesh order."""
    up = vertices[:, 2] >= 0.0
    return vertices[up], vertices[~up]


def complex_gaussian(n: int, nrhs: int, seed: int) -> np.ndarray:
    """CN(0,1) matrix of shape (n, nrhs), column-major use: column r is RHS r."""
    g = np.random.default_rng(seed).standard_normal((n, nrhs, 2)) / math.sqrt(2.0)
    return g[..., 0] + 1j * g[..., 1]


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct sorted indices in [0, n) from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


@functools.lru_cache(maxsize=4)
def _sphere_halves(level: int):
    return hemispheres(icosphere(level)[0])


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: points, phase family, build tolerance, RHS.

    x_kind / w_kind: "grid" (uniform X grid, integer frequency grid Omega),
    "unit" (w_kind only: Omega the same uniform grid in [0,1)^d as X, the
    discretization of Example 1 as the paper states it), "random" (uniform in
    [0,1)^d, seeds x_seed / w_seed) or "sphere" (both
    halves of the icosphere of level n, scaled by h = sqrt(|X|)/10 so that the
    DISTANCE phase |x - xi| is the Helmholtz phase h |x - xi| of the unit sphere).
    """
    name: str
    d: int
    n: int
    phase: int
    tol: float
    n0: int
    nrhs: int
    f_seed: int
    x_kind: str = "grid"        # "grid", "random" or "sphere"
    x_seed: int = 0
    recovered: bool = False     # phase recovered from 8 rows + 8 cols
    sample_rows: int = 0        # 0 = full direct sum, else sampled rows
    sample_seed: int = 3
    w_kind: str = "grid"        # "grid", "unit", "random" or "sphere"
    w_seed: int = 1
    t: float = 2.0              # oversampling of the ID samples (Sec. 3.2)

    @property
    def N(self) -> int:
        """Points per side of the grid and random workloads (|X| for the sphere)."""
        if self.x_kind == "sphere":
            return self.nx
        return self.n ** self.d

    @property
    def nx(self) -> int:
        return len(_sphere_halves(self.n)[0]) if self.x_kind == "sphere" else self.n ** self.d

    @property
    def nw(self) -> int:
        return len(_sphere_halves(self.n)[1]) if self.w_kind == "sphere" else self.n ** self.d

    @property
    def h(self) -> float:
        """Wave number of the sphere workloads (1 otherwise)."""
        return math.sqrt(self.nx) / 10.0 if self.x_kind == "sphere" else 1.0

    def points(self):
        """(X, W, boxX, boxW): coordinates and the domain cubes (lo, side)."""
        if self.x_kind == "sphere":
            X0, W0 = _sphere_halves(self.n)
            h = self.h
            box = (np.full(3, -h), 2.0 * h)
            return h * X0, h * W0, box, box
        if self.x_kind == "grid":
            X = uniform_grid(self.n, self.d)
        else:
            X = uniform_random_points(self.N, self.d, self.x_seed)
        boxX = (np.zeros(self.d), 1.0)
        if self.w_kind == "random":
            W = uniform_random_points(self.N, self.d, self.w_seed)
            boxW = (np.zeros(self.d), 1.0)
        elif self.w_kind == "unit":
            W = uniform_grid(self.n, self.d)
            boxW = (np.zeros(self.d), 1.0)
        else:
            W = frequency_grid(self.n, self.d)
            boxW = (np.full(self.d, -float(self.n // 2)), float(self.n))
        return X, W, boxX, boxW

    def rhs(self, nrhs: int | None = None) -> np.ndarray:
        """f on Omega: (nw, nrhs)."""
        return complex_gaussian(self.nw, self.nrhs if nrhs is None else nrhs, self.f_seed)


# The workloads: Example 1 (2D generalized Radon transform) and a 3D variant of
# it, Example 2 (3D non-uniform Fourier transform, random X and Omega in the
# unit cube) and Example 3 (Helmholtz phase on the two halves of a sphere mesh).
WORKLOADS = {
    "fio2d_n64": Workload("fio2d_n64", 2, 64, PHASE_FIO2D, 1e-6, 64, 1, 0),
    "fio2d_n256_recovered": Workload("fio2d_n256_recovered", 2, 256, PHASE_FIO2D, 1e-6, 64, 64, 0,
                                     recovered=True),
    "fio3d_n32": Workload("fio3d_n32", 3, 32, PHASE_FIO3D, 1e-6, 512, 256, 0,
                          x_kind="random", x_seed=0, sample_rows=512, sample_seed=3),
    "fio2d_jump_n1024": Workload("fio2d_jump_n1024", 2, 1024, PHASE_FIO2D_JUMP, 1e-6, 64, 16, 0,
                                 sample_rows=256, sample_seed=3),
    "nuft3d_n16": Workload("nuft3d_n16", 3, 16, PHASE_DOT, 1e-6, 512, 4, 0, x_kind="random", x_seed=0,
                           w_kind="random", w_seed=1),
    "nuft3d_n32": Workload("nuft3d_n32", 3, 32, PHASE_DOT, 1e-6, 512, 1, 0, x_kind="random", x_seed=0,
                           w_kind="random", w_seed=1, sample_rows=256, sample_seed=3),
    "nuft3d_n64": Workload("nuft3d_n64", 3, 64, PHASE_DOT, 1e-6, 512, 1, 0, x_kind="random", x_seed=0,
                           w_kind="random", w_seed=1, sample_rows=256, sample_seed=3),
    "helmholtz_l5": Workload("helmholtz_l5", 3, 5, PHASE_DISTANCE, 1e-6, 64, 4, 0, x_kind="sphere",
                             w_kind="sphere", t=5.0),
    "helmholtz_l6": Workload("helmholtz_l6", 3, 6, PHASE_DISTANCE, 1e-6, 128, 1, 0, x_kind="sphere",
                             w_kind="sphere", sample_rows=256, sample_seed=3, t=5.0),
}


def batched_instances(count: int = 32, seed: int = 1):
    """Uneven batch: n_i from {64,128,256,512} and nrhs_i in [1, 32], one generator."""
    rng = np.random.default_rng(seed)
    ns = rng.choice([64, 128, 256, 512], count)
    nrhs = rng.integers(1, 33, count)
    out = []
    for i, (n, r) in enumerate(zip(ns.tolist(), nrhs.tolist())):
        out.append(Workload(f"batch{i}_n{n}", 2, int(n), PHASE_FIO2D, 1e-6, 64, int(r), 100 + i,
                            sample_rows=256 if n > 256 else 0))
    return out
