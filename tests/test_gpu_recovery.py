"""Vector recovery (Algorithm 4, Sec. 2.3) on the GPU against the oracle.

midbf_recover_vectors runs Algorithm 4 level by level over the runs of a
recovery path (one CTA per vector).  Every edge performs the FP64 operations
of the sequential loop, so the recovered values must equal the oracle's
recovery_vector bit for bit (hence the integer offsets v - u too), and the
flagged sets D must be the same lists in the same order.  The paths come from
the oracle (Algorithm 5: Delaunay, MST, breadth-first order) or are written
out by hand (a chain, a star, pieces cut by Partition2); the inputs include
exact ties u(ed) - v(bg) = +-1/2, where round half away from zero decides.
Then Algorithm 7 through the C ABI with MIDBF_RECOVER_DEVICE must give the
same low-rank phase, bit for bit, as the host recovery.
"""
import numpy as np
import pytest

import synth
from oracle import recovery
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu


def _frac(phi):
    return phi - np.floor(phi)


def _check(path_edges, n, U, tau, V0=None, root=None):
    """Device recovery of the rows of U along path_edges against the oracle."""
    rp = mb.RecoveryPath(n, path_edges, root)
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    v0 = None if V0 is None else torch.from_numpy(np.ascontiguousarray(V0)).cuda()
    v, flags, D = rp.recover(u, tau, v0)
    v = v.cpu().numpy()
    for k in range(U.shape[0]):
        ref, Dref = recovery.recovery_vector(U[k], tau, path_edges, None if V0 is None else V0[k])
        assert np.array_equal(v[k], ref), k
        if path_edges.shape[0]:
            assert D[k] == Dref, (k, D[k][:10], Dref[:10])
        assert np.abs(v[k] - U[k] - np.rint(v[k] - U[k])).max() < 1e-12   # integer offsets (up to rounding)
    return rp, D


@pytest.mark.parametrize("tau", [0.25, 0.1])
def test_random_points_along_oracle_path(tau):
    """Example 2's setting: random points in the unit cube, x.xi with xi
    scaled so that some path increments exceed tau."""
    X = synth.uniform_random_points(4096, 3, 0)
    W = synth.uniform_random_points(8, 3, 1) * 24.0
    P = recovery.recovery_path(X)
    U = np.stack([_frac(X @ w) for w in W])
    rp, D = _check(P, X.shape[0], U, tau)
    assert rp.runs() > 1
    assert max(len(d) for d in D) > 1          # some discontinuities are flagged


def test_nyquist_grid_many_flags():
    """The FIO2D phase on the uniform 32 x 32 grid aliases: many flags."""
    n = 32
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    ph = OPhase(synth.PHASE_FIO2D, X, W)
    P = recovery.recovery_path(X)
    cols = synth.sample_rows(n * n, 8, 5)
    U = np.stack([_frac(ph(np.arange(n * n), np.full(n * n, c))) for c in cols])
    _, D = _check(P, n * n, U, 0.25)
    assert max(len(d) for d in D) > 10


def test_exact_ties_chain_star_and_pieces():
    n = 64
    # chain 0 - 1 - ... - 63: one run per edge; increments of exactly +-1/2
    chain = np.stack([np.arange(n - 1), np.arange(1, n)], 1)
    U = np.stack([np.tile([0.25, 0.75], n // 2), np.tile([0.75, 0.25], n // 2),
                  np.linspace(0.0, 0.96875, n)])
    rp, _ = _check(chain, n, U, 0.25)
    assert rp.runs() == n - 1
    # star around node 5: a single run
    star = np.stack([np.full(n - 1, 5), np.delete(np.arange(n), 5)], 1)
    rp, _ = _check(star, n, U, 0.3)
    assert rp.runs() == 1
    # a balanced binary tree in breadth-first order: one run per depth
    tree = np.stack([(np.arange(1, n) - 1) // 2, np.arange(1, n)], 1)
    rp, D = _check(tree, n, U, 0.2)
    assert rp.runs() == 6
    # the pieces Partition2 cuts at D, each from a given start value at its root
    pieces, _ = recovery.partition(tree, D[2])
    V0 = U + 3.0
    for root, E in pieces:
        if E.shape[0]:
            _check(E, n, U, 1.0, V0, root=root)


def _access(P, nx, nw):
    rows = lambda idx: np.exp(2j * np.pi * P(idx[:, None], np.arange(nw)[None, :]))
    cols = lambda idx: np.exp(2j * np.pi * P(np.arange(nx)[:, None], idx[None, :]))
    return rows, cols


def _same_recovery(X, W, P, **kw):
    rows, cols = _access(P, X.shape[0], W.shape[0])
    host = mb.Phase.recover(X, W, rows, cols, **kw)
    dev = mb.Phase.recover(X, W, rows, cols, device=True, **kw)
    Uh, Vh = host.factors()
    Ud, Vd = dev.factors()
    assert np.array_equal(Uh, Ud) and np.array_equal(Vh, Vd)
    assert host.info == dev.info
    return dev


def test_algorithm7_on_device_equals_host_example2():
    """Example 2 at n = 16 (4096 random points per side), r = 4, q = 2: the
    recovery is exact (Table 4), and the device path changes no bit."""
    X = synth.uniform_random_points(4096, 3, 0)
    W = synth.uniform_random_points(4096, 3, 1)
    ph = _same_recovery(X, W, OPhase(synth.PHASE_DOT, X, W), r=4, q=2, seed=0)
    assert ph.info["mismatches"] == 0


def test_algorithm7_on_device_equals_host_with_pieces():
    """A rank-3 phase with a jump across x1 = 0: several pieces along X, so
    Algorithm 6 recovers block by block."""
    n = 24
    X = synth.uniform_grid(n, 2) * 0.3 - 0.15
    W = synth.frequency_grid(n, 2) * 0.2
    sg = np.where(X[:, 0] >= 0, 1.0, -1.0)
    P = OPhase(synth.PHASE_LOWRANK, X, W, np.stack([X[:, 0], X[:, 1], 0.5 * sg], 1),
               np.stack([W[:, 0], W[:, 1], np.linalg.norm(W, axis=1)], 1))
    ph = _same_recovery(X, W, P, r=4, q=2, seed=3)
    assert ph.info["disc_rows"] > 0 and ph.info["mismatches"] == 0
