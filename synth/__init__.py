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
Complex Gaussian CN(0,1): real and imaginary parts each N(0, 1/2).
"""
from __future__ import annotations

import dataclasses
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


def complex_gaussian(n: int, nrhs: int, seed: int) -> np.ndarray:
    """CN(0,1) matrix of shape (n, nrhs), column-major use: column r is RHS r."""
    g = np.random.default_rng(seed).standard_normal((n, nrhs, 2)) / math.sqrt(2.0)
    return g[..., 0] + 1j * g[..., 1]


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct sorted indices in [0, n) from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: points, phase family, build tolerance, RHS."""
    name: str
    d: int
    n: int
    phase: int
    tol: float
    n0: int
    nrhs: int
    f_seed: int
    x_kind: str = "grid"        # "grid" or "random"
    x_seed: int = 0
    recovered: bool = False     # phase recovered from 8 rows + 8 cols
    sample_rows: int = 0        # 0 = full direct sum, else sampled rows
    sample_seed: int = 3

    @property
    def N(self) -> int:
        return self.n ** self.d

    def points(self):
        """(X, W, boxX, boxW): coordinates and the domain cubes (lo, side)."""
        if self.x_kind == "grid":
            X = uniform_grid(self.n, self.d)
        else:
            X = uniform_random_points(self.N, self.d, self.x_seed)
        W = frequency_grid(self.n, self.d)
        boxX = (np.zeros(self.d), 1.0)
        boxW = (np.full(self.d, -float(self.n // 2)), float(self.n))
        return X, W, boxX, boxW

    def rhs(self, nrhs: int | None = None) -> np.ndarray:
        return complex_gaussian(self.N, self.nrhs if nrhs is None else nrhs, self.f_seed)


# The five workloads of the build, patterned on Example 1 (2D generalized Radon
# transform) and a 3D variant of it.
WORKLOADS = {
    "fio2d_n64": Workload("fio2d_n64", 2, 64, PHASE_FIO2D, 1e-6, 64, 1, 0),
    "fio2d_n256_recovered": Workload("fio2d_n256_recovered", 2, 256, PHASE_FIO2D, 1e-6, 64, 64, 0,
                                     recovered=True),
    "fio3d_n32": Workload("fio3d_n32", 3, 32, PHASE_FIO3D, 1e-6, 512, 256, 0,
                          x_kind="random", x_seed=0, sample_rows=512, sample_seed=3),
    "fio2d_jump_n1024": Workload("fio2d_jump_n1024", 2, 1024, PHASE_FIO2D_JUMP, 1e-6, 64, 16, 0,
                                 sample_rows=256, sample_seed=3),
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
