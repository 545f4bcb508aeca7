"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: printed
worked examples (tests/golden), closed forms (FFT for Phi = x.xi, rank one
for Phi = 0 or separable Phi), brute force on tiny problems, the ID error
bound of the pivoted QR, and invariants of the recovery (Lemma 3.2, the
mod-1 identity).
"""
import os

import numpy as np
import pytest

import synth
from oracle import direct, fftcheck, idec, midbf, planio, recovery
from oracle.phase import Phase, coordinate_phase, kernel
from oracle.tree import Tree

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid_phase(n, d, family):
    X = synth.uniform_grid(n, d)
    W = synth.frequency_grid(n, d)
    return Phase(family, X, W)


def _boxes(n, d):
    return (np.zeros(d), 1.0), (np.full(d, -n / 2), float(n))


# ---------------------------------------------------------------- phases
def test_phase_hand_values():
    """Example 1's phase at hand-evaluated points (tests/golden/phase_values.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "phase_values.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 5
    for fam, x1, x2, k1, k2, val in rows:
        got = coordinate_phase(int(fam), np.array([float(x1), float(x2)]), np.array([float(k1), float(k2)]))
        assert abs(got - eval(val)) < 1e-14, (fam, x1, x2, k1, k2)


def test_phase_hand_values_3d():
    """The 3D FIO phase at hand-evaluated points (tests/golden/phase_values_3d.txt):
    the cyclic index k+1 and the sin/cos order of c_k are what the values fix."""
    rows = [l.split() for l in open(os.path.join(GOLD, "phase_values_3d.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 4
    for x1, x2, x3, k1, k2, k3, val in rows:
        x = np.array([float(x1), float(x2), float(x3)])
        w = np.array([float(k1), float(k2), float(k3)])
        got = coordinate_phase(synth.PHASE_FIO3D, x, w)
        assert abs(got - float(val)) < 1e-14, (x, w, got, val)


# ---------------------------------------------------------------- direct sum
@pytest.mark.parametrize("n,d", [(16, 2), (32, 2), (8, 3)])
def test_direct_sum_matches_fft(n, d):
    """Eq. (1) with Phi = x.xi on the uniform grids equals an inverse DFT."""
    ph = _grid_phase(n, d, synth.PHASE_DOT)
    f = synth.complex_gaussian(n ** d, 2, 7)
    g = direct.direct_sum(ph, f)
    assert direct.rel_l2(g, fftcheck.fft_apply(f, n, d)) < 1e-12


def test_direct_adjoint_is_conjugate_transpose():
    ph = _grid_phase(8, 2, synth.PHASE_FIO2D)
    K = direct.dense_kernel(ph)
    g = synth.complex_gaussian(64, 3, 1)
    assert np.allclose(direct.direct_adjoint(ph, g), K.conj().T @ g, rtol=0, atol=1e-12)
    # rows/cols subsets agree with the full sums
    f = synth.complex_gaussian(64, 1, 2)[:, 0]
    rows = np.array([3, 17, 40])
    assert np.allclose(direct.direct_sum(ph, f, rows=rows), (K @ f)[rows], atol=1e-12)


# ---------------------------------------------------------------- trees
def test_tree_zorder_matches_fig6():
    rows = np.loadtxt(os.path.join(GOLD, "fig6_zorder.txt"))
    pts = rows[:, :2]
    T = Tree(pts, 2, (np.zeros(2), 1.0))
    for i, z in enumerate(rows[:, 2].astype(int)):
        assert list(T.points(2, z)) == [i]
    # children of node 1 at level 1 are 4..7 (Sec. 3.1: children 4i+t)
    assert T.children(1, 1) == [4, 5, 6, 7]


def test_tree_partitions_points():
    X = synth.uniform_random_points(1000, 3, 4)
    T = Tree(X, 3)
    for lev in range(4):
        allp = np.concatenate([T.points(lev, z) for z in T.level(lev)])
        assert np.array_equal(np.sort(allp), np.arange(1000))
    for lev in range(3):
        for z in T.level(lev):
            kids = np.concatenate([T.points(lev + 1, c) for c in T.children(lev, z)])
            assert np.array_equal(np.sort(kids), np.sort(T.points(lev, z)))


# ---------------------------------------------------------------- IDs
def test_column_id_error_bound():
    """||A - A(:,q) V||_F <= sqrt(n-k) |R(k+1,k+1)| (column pivoting bound), Sec. 3.2."""
    rng = np.random.default_rng(0)
    A = (rng.standard_normal((60, 9)) @ rng.standard_normal((9, 45))).astype(complex)
    A = A + 1e-7 * (rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape))
    for tol in (1e-3, 1e-6, 1e-9):
        skel, red, T, rdiag = idec.column_id(A, tol, 10 ** 9)
        k = skel.size
        V = idec.id_matrix(skel, red, T)
        err = np.linalg.norm(A - A[:, skel] @ V)
        bound = np.sqrt(A.shape[1] - k) * rdiag[k] if k < rdiag.size else 0.0
        assert err <= bound * (1 + 1e-8) + 1e-12 * np.linalg.norm(A)
        assert np.all(rdiag[:k] > tol * rdiag[0]) and (k == rdiag.size or rdiag[k] <= tol * rdiag[0])


def test_column_id_rank_one_exact():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    b = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    A = np.outer(a, b)
    skel, red, T, _ = idec.column_id(A, 1e-9, 10 ** 9)
    assert skel.size == 1
    assert np.allclose(A[:, skel] @ idec.id_matrix(skel, red, T), A, atol=1e-13)


def test_mock_chebyshev_sample_distinct_and_sized():
    rng = np.random.default_rng(2)
    pts = synth.uniform_random_points(500, 2, 3)
    pos = idec.mock_chebyshev_sample(pts, 60, rng)
    assert pos.size >= 60 and np.unique(pos).size == pos.size
    assert np.array_equal(idec.mock_chebyshev_sample(pts[:40], 60, rng), np.arange(40))


# ---------------------------------------------------------------- MIDBF
@pytest.mark.parametrize("family", [synth.PHASE_ZERO, synth.PHASE_SEPARABLE])
@pytest.mark.parametrize("n0,L", [(16, 3), (64, 2)])
def test_midbf_exact_for_rank_one_kernels(family, n0, L):
    """Phi = 0 or a(x) + b(xi) gives a rank-one K; every ID is exact (odd and even L)."""
    n = 32
    ph = _grid_phase(n, 2, family)
    bx, bw = _boxes(n, 2)
    fac = midbf.build(ph, n0=n0, tol=1e-9, boxX=bx, boxW=bw)
    assert fac.L == L
    f = synth.complex_gaussian(n * n, 1, 0)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(ph, f)) < 1e-12
    assert max(r[2] for r in fac.ranks) == 1


@pytest.mark.parametrize("n0,L", [(16, 1), (4, 2), (1, 3)])
def test_midbf_dense_product_tiny(n0, L):
    """All factors multiplied out reproduce the dense K on an 8x8 grid."""
    n = 8
    ph = _grid_phase(n, 2, synth.PHASE_FIO2D)
    bx, bw = _boxes(n, 2)
    fac = midbf.build(ph, n0=n0, tol=1e-10, boxX=bx, boxW=bw)
    assert fac.L == L
    K = direct.dense_kernel(ph)
    P = midbf.dense(fac)
    assert np.linalg.norm(P - K) / np.linalg.norm(K) < 1e-8


@pytest.mark.parametrize("n,family", [(32, synth.PHASE_FIO2D), (64, synth.PHASE_FIO2D),
                                      (32, synth.PHASE_DOT), (32, synth.PHASE_FIO2D_JUMP)])
def test_midbf_matches_direct_sum(n, family):
    ph = _grid_phase(n, 2, family)
    bx, bw = _boxes(n, 2)
    fac = midbf.build(ph, n0=64, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    f = synth.complex_gaussian(n * n, 1, 0)[:, 0]
    g = midbf.apply(fac, f)
    ref = fftcheck.fft_apply(f, n, 2) if family == synth.PHASE_DOT else direct.direct_sum(ph, f)
    assert direct.rel_l2(g, ref) < 2e-5


def test_midbf_3d_random_points():
    n = 8
    X = synth.uniform_random_points(n ** 3, 3, 0)
    W = synth.frequency_grid(n, 3)
    ph = Phase(synth.PHASE_FIO3D, X, W)
    fac = midbf.build(ph, n0=8, tol=1e-7, t=2.0, boxX=(np.zeros(3), 1.0), boxW=(np.full(3, -4.0), 8.0))
    assert fac.L == 2
    f = synth.complex_gaussian(n ** 3, 1, 0)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(ph, f)) < 1e-5


def test_midbf_adjoint_identity_and_dense_adjoint():
    n = 16
    ph = _grid_phase(n, 2, synth.PHASE_FIO2D)
    bx, bw = _boxes(n, 2)
    fac = midbf.build(ph, n0=16, tol=1e-8, boxX=bx, boxW=bw)
    f = synth.complex_gaussian(n * n, 1, 0)[:, 0]
    h = synth.complex_gaussian(n * n, 1, 1)[:, 0]
    lhs = np.vdot(h, midbf.apply(fac, f))
    rhs = np.vdot(midbf.apply_adjoint(fac, h), f)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    K = direct.dense_kernel(ph)
    assert direct.rel_l2(midbf.apply_adjoint(fac, h), K.conj().T @ h) < 1e-6


def test_planio_round_trip_bitwise():
    n = 16
    ph = _grid_phase(n, 2, synth.PHASE_FIO2D)
    bx, bw = _boxes(n, 2)
    fac = midbf.build(ph, n0=16, tol=1e-6, boxX=bx, boxW=bw)
    fac2 = planio.read(planio.write(fac))
    f = synth.complex_gaussian(n * n, 2, 0)
    assert np.array_equal(midbf.apply(fac, f), midbf.apply(fac2, f))
    with pytest.raises(ValueError):
        planio.read(planio.write(fac)[:-3])


# ---------------------------------------------------------------- recovery
def _read_pairs(line):
    return [tuple(int(v) - 1 for v in p.split("-")) for p in line.split(":")[1].split()]


def test_bfs_path_fig3():
    lines = {l.split(":")[0]: l for l in open(os.path.join(GOLD, "fig3_path.txt")) if ":" in l and l[0] != "#"}
    edges = np.array(_read_pairs(lines["tree_edges"]))
    P = recovery.bfs_path(7, edges, root=0)
    assert [tuple(p) for p in P] == _read_pairs(lines["P"])


def test_partition_fig4():
    lines = {l.split(":")[0]: l for l in open(os.path.join(GOLD, "fig4_partition.txt")) if ":" in l and l[0] != "#"}
    P = np.array(_read_pairs(lines["P"]))
    D = [int(v) - 1 for v in lines["D"].split(":")[1].split()]
    pieces, _ = recovery.partition(P, D)
    assert [tuple(e) for e in pieces[0][1]] == _read_pairs(lines["piece 1"])
    assert [tuple(e) for e in pieces[1][1]] == _read_pairs(lines["piece 4"])


def test_mst_is_minimal_on_small_sets():
    """Total MST weight equals the brute-force Prim MST on the complete graph."""
    X = synth.uniform_random_points(40, 2, 9)
    E = recovery.mst_edges(X)
    w = np.linalg.norm(X[E[:, 0]] - X[E[:, 1]], axis=1).sum()
    D = np.linalg.norm(X[:, None] - X[None], axis=2)
    inT = np.zeros(40, bool); inT[0] = True
    best = D[0].copy(); tot = 0.0
    for _ in range(39):
        best[inT] = np.inf
        j = int(np.argmin(best)); tot += best[j]; inT[j] = True
        best = np.minimum(best, D[j])
    assert abs(w - tot) < 1e-12
    P = recovery.recovery_path(X)
    assert sorted(P[:, 1].tolist()) == list(range(1, 40))


def test_recovery_vector_is_prefix_sum_of_wrapped_increments():
    rng = np.random.default_rng(3)
    X = synth.uniform_random_points(200, 2, 1)
    P = recovery.recovery_path(X)
    phi = 7.0 * rng.standard_normal() + 3.0 * X[:, 0] - 2.0 * X[:, 1] ** 2
    u = phi - np.rint(phi)
    v, _ = recovery.recovery_vector(u, 1.0, P)
    parent = np.full(200, -1); parent[P[:, 1]] = P[:, 0]
    ref = np.empty(200)
    for node in range(200):          # walk to the root, summing wrapped increments
        acc, c = 0.0, node
        while parent[c] >= 0:
            t = u[c] - u[parent[c]]
            acc += t - np.sign(t) * np.floor(np.abs(t) + 0.5)
            c = parent[c]
        ref[node] = u[c] + acc
    assert np.allclose(v, ref, atol=1e-12)


def test_low_rank_phase_recovers_smooth_phase():
    """Small path increments: Psi = Phi + integer row/column offsets, e^{2 pi i Psi} = K."""
    n = 24
    X = synth.uniform_grid(n, 2) * 0.3
    W = synth.frequency_grid(n, 2)
    ph = Phase(synth.PHASE_DOT, X, W)
    wr = lambda idx: (lambda p: p - np.rint(p))(ph(idx[:, None], np.arange(n * n)[None, :]))
    wc = lambda idx: (lambda p: p - np.rint(p))(ph(np.arange(n * n)[:, None], idx[None, :]))
    U, V, rec = recovery.low_rank_phase(wr, wc, X, W, r=4, q=2, seed=0)
    assert rec.mismatches == 0 and len(rec.Dr) == 1 and len(rec.Dc) == 1 and rec.tau == 0.25
    # mod-1 identity on recovered rows and columns (exact by construction)
    d = rec.rows - wr(rec.R)
    assert np.abs(d - np.rint(d)).max() < 1e-12
    # Psi - Phi is one integer per recovered row
    diff = rec.rows - ph(rec.R[:, None], np.arange(n * n)[None, :])
    assert np.abs(diff - diff[:, :1]).max() < 1e-9 and np.abs(diff - np.rint(diff)).max() < 1e-9
    S = synth.sample_rows(n * n, 200, 3)
    assert recovery.eps_K(ph, U, V, S) < 1e-9


def _jump_phase(n=24):
    """Phi = x.xi + (1/2) sign(x1) |xi| on a small grid: rank 3, with a jump of
    |xi| across x1 = 0 that is not an integer (a discontinuity for Algorithm 4),
    and path increments below 1/4 elsewhere."""
    X = synth.uniform_grid(n, 2) * 0.3 - 0.15
    W = synth.frequency_grid(n, 2) * 0.2
    sg = np.where(X[:, 0] >= 0, 1.0, -1.0)
    U = np.stack([X[:, 0], X[:, 1], 0.5 * sg], 1)
    V = np.stack([W[:, 0], W[:, 1], np.linalg.norm(W, axis=1)], 1)
    return X, W, Phase(synth.PHASE_LOWRANK, X, W, U, V)


def test_recovery_partitions_at_a_jump():
    """Algorithm 6: the jump is detected along the X path, Partition2 splits
    the tree there, and each piece is recovered from its own root, so rows and
    columns still agree (Lemma 3.2: zero mismatches at tau = 1/4) and
    exp(2 pi i Psi) reproduces K to rounding for r >= 4 (rank 3 plus the
    integer offsets); r = 3 cannot hold the offsets."""
    X, W, ph = _jump_phase()
    N = X.shape[0]
    wr = lambda idx: (lambda p: p - np.rint(p))(ph(idx[:, None], np.arange(N)[None, :]))
    wc = lambda idx: (lambda p: p - np.rint(p))(ph(np.arange(N)[:, None], idx[None, :]))
    S = synth.sample_rows(N, 200, 3)
    for r, exact in ((3, False), (4, True), (5, True)):
        U, V, rec = recovery.low_rank_phase(wr, wc, X, W, r=r, q=2, seed=0, max_disc=64)
        assert len(rec.Dr) > 1 and rec.tau == 0.25 and rec.mismatches == 0
        ek = recovery.eps_K(ph, U, V, S)
        assert (ek < 1e-12) if exact else (ek > 0.1), (r, ek)
