"""Multidimensional phase recovery (oracle, FP64), Sec. 2.1 and 2.3.

* ``recovery_path``     — Algorithm 5: P = BFS(MST(DT(X))), Def. 3.1-3.3.
                          Library steps: scipy Delaunay, csgraph MST.  BFS is
                          written out; neighbours are visited in ascending
                          index order, which reproduces the worked example
                          of Fig. 3 (P = [1,3;1,4;1,7;3,6;4,2;4,5]).
* ``recovery_vector``   — Algorithm 4: v(ed) = u(ed) - round(u(ed) - v(bg))
                          along the path; |v(ed) - v(bg)| >= tau flags ed.
                          Reading R1: round half away from zero.  Reading R2:
                          D starts with the path's root.
* ``partition``         — Partition2 (Sec. 2.3.4, Fig. 4): cut the tree at
                          every node of D; each piece keeps its edges in path
                          order.  Worked example of Fig. 4 pinned in tests.
* ``recovery_matrix``   — Algorithm 6 with the block order of its lines.
* ``rsvd_restricted``   — Algorithm 1 restricted to the known rows R and
                          columns C (reading R4: Pi_col within C, Pi_row
                          within R, S_row = R minus Pi_row, S_col likewise).
* ``low_rank_phase``    — Algorithm 7: R, C, recovery, rSVD, V <- V Sigma.
                          Reading R3: R and C contain index 0 (the path root)
                          plus seeded random indices.  Reading R6: tau starts
                          at 1/4 and grows by 1/40 while a vector has more
                          than ``max_disc`` flags, at most to 1/2.

Parity: pinned in tests by the worked examples of Fig. 3 and Fig. 4, by the
mod-1 identity e^{2 pi i Psi} = K on recovered rows/columns, by the closed
form of Algorithm 4 as a tree prefix sum of wrapped increments, by Lemma 3.2
(no row/column mismatch at tau <= 1/4), and by exact recovery of rank-r
phases with small path increments.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import minimum_spanning_tree
from scipy.spatial import Delaunay


def matlab_round(x):
    """Round half away from zero (MATLAB's round)."""
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def mst_edges(X: np.ndarray):
    """Edges (i, j) of a Euclidean MST taken from the Delaunay graph (Def. 3.1, 3.2)."""
    n, d = X.shape
    if n == 1:
        return np.zeros((0, 2), dtype=np.int64)
    if n <= d + 1:
        ii, jj = np.triu_indices(n, 1)
    else:
        tri = Delaunay(X)
        simp = tri.simplices
        pairs = []
        for a in range(d + 1):
            for b in range(a + 1, d + 1):
                pairs.append(np.stack([simp[:, a], simp[:, b]], axis=1))
        e = np.concatenate(pairs)
        e = np.sort(e, axis=1)
        e = np.unique(e, axis=0)
        ii, jj = e[:, 0], e[:, 1]
    w = np.linalg.norm(X[ii] - X[jj], axis=1)
    # zero-length edges would vanish in the sparse graph: shift all weights by one
    G = coo_matrix((w + 1.0, (ii, jj)), shape=(n, n)).tocsr()
    T = minimum_spanning_tree(G).tocoo()
    return np.stack([T.row, T.col], axis=1).astype(np.int64)


def bfs_path(n: int, edges: np.ndarray, root: int = 0) -> np.ndarray:
    """Recovery path matrix P ((n-1) x 2, [parent, child]) by BFS from root (Def. 3.3)."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    for lst in adj:
        lst.sort()
    seen = np.zeros(n, dtype=bool)
    seen[root] = True
    queue = [root]
    head = 0
    P = []
    while head < len(queue):
        u = queue[head]
        head += 1
        for v in adj[u]:
            if not seen[v]:
                seen[v] = True
                P.append((u, v))
                queue.append(v)
    if len(P) != n - 1:
        raise ValueError("the graph is not connected")
    return np.asarray(P, dtype=np.int64).reshape(-1, 2)


def recovery_path(X: np.ndarray, root: int = 0) -> np.ndarray:
    """Algorithm 5: P = bfsearch(minspantree(delaunay(X)))."""
    return bfs_path(X.shape[0], mst_edges(np.asarray(X, dtype=np.float64)), root)


def recovery_vector(u: np.ndarray, tau: float, P: np.ndarray, v0=None):
    """Algorithm 4.  u: observed values mod 1; returns (v, D).

    v starts as a copy of u (or of v0 when the caller has already fixed some
    entries, e.g. the path's root); each edge fixes v at its child from v at
    its parent.
    """
    v = np.array(u if v0 is None else v0, dtype=np.float64, copy=True)
    D = [int(P[0, 0])] if P.shape[0] else []
    for bg, ed in P:
        v[ed] = u[ed] - matlab_round(u[ed] - v[bg])
        if abs(v[ed] - v[bg]) >= tau:
            D.append(int(ed))
    return v, D


def partition(P: np.ndarray, D):
    """Partition2: split the path at the nodes of D (D[0] is the root).

    Returns a list of (root, edges) in the order of D, each edges array in
    path order, parent and child both inside the piece.
    """
    Dset = set(int(x) for x in D)
    owner = {int(P[0, 0]) if P.shape[0] else int(D[0]): int(D[0])}
    owner[int(D[0])] = int(D[0])
    pieces = {int(x): [] for x in D}
    for bg, ed in P:
        bg, ed = int(bg), int(ed)
        if ed in Dset:
            owner[ed] = ed
            continue
        owner[ed] = owner[bg]
        pieces[owner[bg]].append((bg, ed))
    return [(int(r), np.asarray(pieces[int(r)], dtype=np.int64).reshape(-1, 2)) for r in D], owner


@dataclasses.dataclass
class Recovered:
    R: np.ndarray            # recovered row indices
    C: np.ndarray            # recovered column indices
    rows: np.ndarray         # Psi(R, :)
    cols: np.ndarray         # Psi(:, C)
    Dr: list
    Dc: list
    tau: float
    mismatches: int          # entries (i in R, j in C) where rows and cols disagree


def _detect(u, P, tau, max_disc):
    t = tau
    while True:
        _, D = recovery_vector(u, t, P)
        if len(D) - 1 <= max_disc or t >= 0.5:
            return D, t
        t = min(0.5, t + 1.0 / 40.0)


def recovery_matrix(wrapped_rows, wrapped_cols, R, C, P1, P2, tau=0.25, max_disc=16) -> Recovered:
    """Algorithm 6.

    wrapped_rows(idx) -> (len(idx), nw) values mod 1 of Phi rows; wrapped_cols
    likewise for columns (nx, len(idx)).  R and C must contain the path roots.
    """
    root_x, root_w = int(P1[0, 0]), int(P2[0, 0])
    col0 = wrapped_cols(np.array([root_w]))[:, 0]
    row0 = wrapped_rows(np.array([root_x]))[0]
    Dr, tau_r = _detect(col0, P1, tau, max_disc)
    Dc, tau_c = _detect(row0, P2, tau, max_disc)
    R = np.array(list(dict.fromkeys([int(x) for x in list(R) + Dr])), dtype=np.int64)
    C = np.array(list(dict.fromkeys([int(x) for x in list(C) + Dc])), dtype=np.int64)
    U_rows = wrapped_rows(R)            # |R| x nw, mod-1 observations
    U_cols = wrapped_cols(C)            # nx x |C|
    rows = U_rows.copy()
    cols = U_cols.copy()
    rpos = {int(r): i for i, r in enumerate(R)}
    cpos = {int(c): j for j, c in enumerate(C)}
    pieces1, own1 = partition(P1, Dr)
    pieces2, own2 = partition(P2, Dc)
    own1_arr = np.array([own1[i] for i in range(P1.shape[0] + 1)])
    own2_arr = np.array([own2[j] for j in range(P2.shape[0] + 1)])
    for rs, E1 in pieces1:
        for ct, E2 in pieces2:
            # root row of block (s,t) along P2.B_t, start value = observation
            i0, j0 = rpos[rs], cpos[ct]
            rows[i0], _ = recovery_vector(U_rows[i0], 1.0, E2, rows[i0]) if E2.size else (rows[i0], None)
            # root column along P1.B_s, starting from the recovered (rs, ct)
            v0 = cols[:, j0].copy()
            v0[rs] = rows[i0, ct]
            cols[:, j0] = recovery_vector(U_cols[:, j0], 1.0, E1, v0)[0] if E1.size else v0
            # sampled rows of piece s over piece t, start from the root column
            for r in R:
                if own1_arr[r] != rs or r == rs:
                    continue
                i = rpos[int(r)]
                v0 = rows[i].copy()
                v0[ct] = cols[r, j0]
                rows[i] = recovery_vector(U_rows[i], 1.0, E2, v0)[0] if E2.size else v0
            # sampled columns of piece t over piece s, start from the root row
            for c in C:
                if own2_arr[c] != ct or c == ct:
                    continue
                j = cpos[int(c)]
                v0 = cols[:, j].copy()
                v0[rs] = rows[i0, c]
                cols[:, j] = recovery_vector(U_cols[:, j], 1.0, E1, v0)[0] if E1.size else v0
    mism = int(np.count_nonzero(np.abs(rows[:, C] - cols[R, :]) > 1e-9))
    return Recovered(R, C, rows, cols, Dr, Dc, max(tau_r, tau_c), mism)


def pivots(A: np.ndarray, r: int) -> np.ndarray:
    """First r column pivots of a column-pivoted QR (library step)."""
    _, P = scipy.linalg.qr(A, mode="r", pivoting=True)
    return P[:r]


def rsvd_restricted(rec: Recovered, r: int):
    """Algorithm 1 on Psi with only rows R and columns C known (reading R4).

    Returns (U, S, V) with Psi ~ U diag(S) V^T, U (nx x r), V (nw x r).
    """
    R, C = rec.R, rec.C
    A_RC = rec.rows[:, C]                       # Psi(R, C)
    pc = pivots(A_RC, r)                        # Pi_col within C (positions)
    pr = pivots(A_RC.T, r)                      # Pi_row within R (positions)
    Pi_col, Pi_row = C[pc], R[pr]
    Q1, _ = np.linalg.qr(rec.cols[:, pc])       # basis of Psi(:, Pi_col), nx x r
    Q2, _ = np.linalg.qr(rec.rows[pr].T)        # basis of Psi(Pi_row, :)^T, nw x r
    I = np.concatenate([Pi_row, np.setdiff1d(R, Pi_row)])
    J = np.concatenate([Pi_col, np.setdiff1d(C, Pi_col)])
    rpos = {int(x): i for i, x in enumerate(R)}
    A_IJ = rec.rows[[rpos[int(i)] for i in I]][:, J]
    M = np.linalg.pinv(Q1[I]) @ A_IJ @ np.linalg.pinv(Q2[J].T)
    UM, SM, VMh = np.linalg.svd(M)
    U = Q1 @ UM[:, :r]
    V = Q2 @ VMh.conj().T[:, :r]
    return U, SM[:r], V


def low_rank_phase(wrapped_rows, wrapped_cols, X1, X2, r: int, q: int, seed: int,
                   tau=0.25, max_disc=16, P1=None, P2=None):
    """Algorithm 7: returns (U, V, Recovered) with Psi ~ U V^T (V <- V Sigma)."""
    nx, nw = X1.shape[0], X2.shape[0]
    rng = np.random.default_rng(seed)
    R = np.concatenate([[0], rng.choice(np.arange(1, nx), size=r * q - 1, replace=False)])
    C = np.concatenate([[0], rng.choice(np.arange(1, nw), size=r * q - 1, replace=False)])
    P1 = recovery_path(X1) if P1 is None else P1
    P2 = recovery_path(X2) if P2 is None else P2
    rec = recovery_matrix(wrapped_rows, wrapped_cols, R, C, P1, P2, tau, max_disc)
    U, S, V = rsvd_restricted(rec, r)
    return U, V * S[None, :], rec


def eps_K(phase_true, U, V, S_idx) -> float:
    """epsilon^K of Sec. 4 on the index set S (rows and columns)."""
    phi = phase_true(S_idx[:, None], S_idx[None, :])
    psi = U[S_idx] @ V[S_idx].T
    A = np.exp(2j * np.pi * phi)
    B = np.exp(2j * np.pi * psi)
    return float(np.linalg.norm(A - B, 2) / np.linalg.norm(A, 2))
