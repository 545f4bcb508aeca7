"""Plain MIDBF construction and apply (oracle, FP64), Sec. 3.

Structure (Sec. 3.1, 3.3-3.5).  Trees T_X, T_Omega of equal depth L (level 0
the root, level L the leaves of about n0 points); b = 2^d.  The paper assumes
L even (Sec. 3.1) and then runs h = L/2 MSCS steps (Sec. 3.5).  Reading M1 for
odd L: one LRCS first (Sec. 3.3), whose middle factor has compressed trees of
depth L-1 (end of Sec. 3.3), then (L-1)/2 MSCS steps.  Both cases are written
as nsteps = ceil(L/2) steps with a shift delta (1 for even L, 0 for odd L);
step s = 1..nsteps pairs

  * X nodes a at level L-s+1 (compressed leaves) with Omega nodes Q at level
    s-1+delta for the row IDs (rID), and
  * Omega nodes beta at level L-s+1 with X nodes P at level s-1+delta for the
    column IDs (cID).

Row IDs come first in a step and run against the columns of the current
middle factor; column IDs then run against the new row skeletons, exactly as
the LRCS of Sec. 3.3 orders them (rID of K(r_i,:), then cID of K(r_hat, c_j)).
At step 1 the rows of an rID are the points of leaf a; at later steps they are
the children's skeletons R_in(a, Q') = [R(c, Q') for c child of a], Q' the
parent of Q.  Columns symmetrically.  After the last step the middle factor S
has one dense block per pair (P, Q) at level nsteps-1+delta whose entries are
kernel values at skeleton points (Sec. 3.5): rows [R(a, Q) for a child of P],
columns [C(beta, P) for beta child of Q].  The M3 reading of the garbled
index formula of S^L_ij is this one.

Factor product (eq. (finishIDBF)): K ~ U^1 ... U^nsteps S V^nsteps ... V^1,
where V^1 holds the leaf column IDs and U^1 the leaf row IDs.  Each factor is
held as a "stage": a list of blocks with explicit input and output index
lists, so the same data structure describes this oracle's factors and those
read from a plan file (``planio``).

  V block (P', beta):  out = [V_{beta,P_k} in for P_k child of P'],
                       V = [I T] Lambda^T per child (Sec. 3.2);
  S block (P, Q):      out = K(rows, cols) in;
  U block (a, Q'):     out = sum_{Q_l child of Q'} U_{a,Q_l} in_{Q_l},
                       U = Lambda [I T]^T (row ID).

The apply assembles every stage as a sparse matrix and multiplies them in
order; the adjoint multiplies the conjugate transposes in reverse order.

Parity: pinned in tests against the direct sum / FFT within tolerance-scaled
bounds, exactly (1e-13) for rank-one kernels, and as a dense product against
the dense K on tiny trees; the per-ID bound is pinned in ``idec``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import idec
from .phase import Phase, kernel
from .tree import Tree

KIND_V, KIND_S, KIND_U = 0, 1, 2


@dataclasses.dataclass
class Sub:
    """One interpolative decomposition inside a V or U block."""
    skel: np.ndarray   # positions (into the block input for V, output for U)
    red: np.ndarray    # the other positions
    T: np.ndarray      # k x (m - k)


@dataclasses.dataclass
class Block:
    in_idx: np.ndarray
    out_idx: np.ndarray
    subs: list = dataclasses.field(default_factory=list)
    xidx: np.ndarray | None = None    # S blocks: X points of the rows
    widx: np.ndarray | None = None    # S blocks: Omega points of the columns


@dataclasses.dataclass
class Stage:
    kind: int
    in_space: int          # -1: the user input vector; else the producing stage
    out_len: int
    out_user: bool         # output space is the user output vector
    blocks: list


@dataclasses.dataclass
class Factorization:
    d: int
    L: int
    delta: int
    nsteps: int
    tol: float
    phase: Phase
    stages: list
    ranks: list = dataclasses.field(default_factory=list)

    @property
    def nx(self):
        return self.phase.X.shape[0]

    @property
    def nw(self):
        return self.phase.W.shape[0]


def depth_for(npts: int, n0: int, b: int) -> int:
    """L = round(log_b(npts / n0)), at least 0 (Sec. 3.3: m = b^L = N / n0)."""
    if npts <= n0:
        return 0
    return max(0, int(round(math.log(npts / n0, b))))


def sampled_id(rows_of, coords, nsamp, t, tol, kmax, rng):
    """Column ID of A(:, cols) from a Mock-Chebyshev sample of its rows.

    rows_of(pos) returns A(cand[pos], cols) for positions into the candidate
    set.  Sec. 3.2: the sample of t*k rows "is empirically selected and
    gradually increased if not large enough", and Sec. 3.6 updates
    k <- k_eps after each QR.  Reading: the sample starts at nsamp rows
    (t times the running rank estimate) and is regrown to ceil(t * k_eps)
    until it holds at least t*k_eps rows or every candidate.  Returns
    (skel, red, T, next nsamp).
    """
    ncand = coords.shape[0]
    ns = max(1, int(nsamp))
    while True:
        pos = idec.mock_chebyshev_sample(coords, ns, rng)
        skel, red, T, _ = idec.column_id(rows_of(pos), tol, kmax)
        k = skel.size
        need = int(math.ceil(t * k))
        if pos.size >= ncand or pos.size >= need:
            return skel, red, T, need
        ns = min(ncand, need)


def build(phase: Phase, n0: int = 64, tol: float = 1e-6, t: float = 5.0, kest: int = 30,
          kmax: int = 1 << 30, seed: int = 0, boxX=None, boxW=None) -> Factorization:
    """Construct the MIDBF of K = exp(2 pi i Phi) over phase.X x phase.W."""
    X, W = phase.X, phase.W
    d = X.shape[1]
    b = 2 ** d
    L = depth_for(max(X.shape[0], W.shape[0]), n0, b)
    TX = Tree(X, L, boxX)
    TW = Tree(W, L, boxW)
    rng = np.random.default_rng(seed)
    if L == 0:
        blk = Block(in_idx=np.arange(W.shape[0]), out_idx=np.arange(X.shape[0]),
                    xidx=np.arange(X.shape[0]), widx=np.arange(W.shape[0]))
        st = Stage(KIND_S, -1, X.shape[0], True, [blk])
        return Factorization(d, 0, 1, 0, tol, phase, [st])
    delta = 1 if L % 2 == 0 else 0
    nsteps = (L + 1) // 2
    nsamp = int(math.ceil(t * kest))

    # Keys are (level of a, a, level of Q, Q) with Z-indices a, Q.
    R = {}     # -> X point indices of the row skeleton of a w.r.t. Q
    C = {}     # (level of beta, beta, level of P, P) -> Omega skeleton points
    Ufac = {}  # -> Sub relative to R_in(a, parent(Q))
    Vfac = {}  # -> Sub relative to C_in(beta, parent(P))
    ranks = []

    def parent_or_none(lev, z):
        return None if lev == 0 else z >> d

    for s in range(1, nsteps + 1):
        la = L - s + 1          # level of the compressed leaves
        lq = s - 1 + delta      # level of the paired nodes
        # ---- row IDs: (a at la) x (Q at lq) ----
        col_cand = {}
        for Q in TW.level(lq):
            Qp = parent_or_none(lq, Q)
            for a in TX.level(la):
                if s == 1:
                    rows = TX.points(la, a)
                else:
                    rows = np.concatenate([R[(la + 1, c, lq - 1, Qp)] for c in TX.children(la, a)])
                Pa = None if s == 1 else TX.ancestor(la, a, s - 2 + delta) if s - 2 + delta >= 0 else None
                key = (Q, Pa)
                if key not in col_cand:
                    if s == 1:
                        col_cand[key] = TW.points(lq, Q)
                    else:
                        col_cand[key] = np.concatenate([C[(la + 1, bb, s - 2 + delta, Pa)]
                                                        for bb in TW.descendants(lq, Q, la + 1)])
                cand = col_cand[key]
                skel, red, T, nsamp = sampled_id(lambda pos: kernel(phase, rows[None, :], cand[pos][:, None]),
                                                 W[cand], nsamp, t, tol, kmax, rng)
                R[(la, a, lq, Q)] = rows[skel]
                Ufac[(la, a, lq, Q)] = Sub(skel, red, T)
                ranks.append(("U", s, skel.size))
        # ---- column IDs: (beta at la) x (P at lq) ----
        row_cand = {}
        for P in TX.level(lq):
            Pp = parent_or_none(lq, P)
            for beta in TW.level(la):
                if s == 1:
                    cols = TW.points(la, beta)
                else:
                    cols = np.concatenate([C[(la + 1, c, lq - 1, Pp)] for c in TW.children(la, beta)])
                Qb = TW.ancestor(la, beta, lq)
                key = (P, Qb)
                if key not in row_cand:
                    row_cand[key] = np.concatenate([R[(la, a, lq, Qb)] for a in TX.descendants(lq, P, la)])
                cand = row_cand[key]
                skel, red, T, nsamp = sampled_id(lambda pos: kernel(phase, cand[pos][:, None], cols[None, :]),
                                                 X[cand], nsamp, t, tol, kmax, rng)
                C[(la, beta, lq, P)] = cols[skel]
                Vfac[(la, beta, lq, P)] = Sub(skel, red, T)
                ranks.append(("V", s, skel.size))

    # ---- assemble the stages (forward order) ----
    stages = []
    # V stages: y(beta, P_k) segments
    ypos_prev = None
    for s in range(1, nsteps + 1):
        la = L - s + 1
        lq = s - 1 + delta
        lp = s - 2 + delta                 # level of P' (-1: virtual parent of the root)
        blocks, ypos, off = [], {}, 0
        parents = TX.level(lp) if lp >= 0 else [None]
        for Pp in parents:
            kids = TX.children(lp, Pp) if Pp is not None else [0]
            for beta in TW.level(la):
                if s == 1:
                    in_idx = TW.points(la, beta)
                else:
                    in_idx = np.concatenate([np.arange(*ypos_prev[(c, Pp)]) for c in TW.children(la, beta)])
                subs, outs = [], []
                for Pk in kids:
                    sub = Vfac[(la, beta, lq, Pk)]
                    k = sub.skel.size
                    ypos[(beta, Pk)] = (off, off + k)
                    outs.append(np.arange(off, off + k))
                    off += k
                    subs.append(sub)
                blocks.append(Block(in_idx=np.asarray(in_idx), out_idx=np.concatenate(outs), subs=subs))
        stages.append(Stage(KIND_V, len(stages) - 1 if s > 1 else -1, off, False, blocks))
        ypos_prev = ypos
    # S stage
    lS = nsteps - 1 + delta
    blocks, zpos, off = [], {}, 0
    for P in TX.level(lS):
        for Q in TW.level(lS):
            betas = TW.children(lS, Q)
            in_idx = np.concatenate([np.arange(*ypos_prev[(bb, P)]) for bb in betas])
            widx = np.concatenate([C[(lS + 1, bb, lS, P)] for bb in betas])
            outs, xs = [], []
            for a in TX.children(lS, P):
                k = R[(lS + 1, a, lS, Q)].size
                zpos[(a, Q)] = (off, off + k)
                outs.append(np.arange(off, off + k))
                xs.append(R[(lS + 1, a, lS, Q)])
                off += k
            blocks.append(Block(in_idx=in_idx, out_idx=np.concatenate(outs),
                                xidx=np.concatenate(xs), widx=widx))
    stages.append(Stage(KIND_S, len(stages) - 1, off, False, blocks))
    # U stages, s = nsteps .. 1
    for s in range(nsteps, 0, -1):
        la = L - s + 1
        lq = s - 1 + delta
        lp = s - 2 + delta
        blocks, znew, off = [], {}, 0
        parents = TW.level(lp) if lp >= 0 else [None]
        for a in TX.level(la):
            for Qp in parents:
                kids = TW.children(lp, Qp) if Qp is not None else [0]
                in_idx = np.concatenate([np.arange(*zpos[(a, Ql)]) for Ql in kids])
                subs = [Ufac[(la, a, lq, Ql)] for Ql in kids]
                if s == 1:
                    out_idx = TX.points(la, a)
                else:
                    outs = []
                    for c in TX.children(la, a):
                        k = R[(la + 1, c, lp, Qp)].size
                        znew[(c, Qp)] = (off, off + k)
                        outs.append(np.arange(off, off + k))
                        off += k
                    out_idx = np.concatenate(outs)
                blocks.append(Block(in_idx=in_idx, out_idx=np.asarray(out_idx), subs=subs))
        last = s == 1
        stages.append(Stage(KIND_U, len(stages) - 1, X.shape[0] if last else off, last, blocks))
        zpos = znew
    return Factorization(d, L, delta, nsteps, tol, phase, stages, ranks)


def stage_matrix(fac: Factorization, st: Stage, in_len: int) -> sp.csr_matrix:
    """The stage as a sparse (out_len x in_len) matrix, written out entry by entry."""
    rows, cols, vals = [], [], []
    for blk in st.blocks:
        if st.kind == KIND_S:
            Kb = kernel(fac.phase, blk.xidx[:, None], blk.widx[None, :])
            rr, cc = np.meshgrid(blk.out_idx, blk.in_idx, indexing="ij")
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(Kb.ravel())
            continue
        seg = 0
        for sub in blk.subs:
            k = sub.skel.size
            if st.kind == KIND_V:
                o = blk.out_idx[seg:seg + k]
                # out_i = in[skel_i] + sum_j T[i,j] in[red_j]
                rows.append(o); cols.append(blk.in_idx[sub.skel]); vals.append(np.ones(k, complex))
                rr, cc = np.meshgrid(o, blk.in_idx[sub.red], indexing="ij")
                rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(sub.T.ravel())
            else:
                i = blk.in_idx[seg:seg + k]
                # out[skel_i] += in_i ; out[red_j] += sum_i T[i,j] in_i
                rows.append(blk.out_idx[sub.skel]); cols.append(i); vals.append(np.ones(k, complex))
                rr, cc = np.meshgrid(blk.out_idx[sub.red], i, indexing="ij")
                rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(sub.T.T.ravel())
            seg += k
    r = np.concatenate(rows) if rows else np.zeros(0, int)
    c = np.concatenate(cols) if cols else np.zeros(0, int)
    v = np.concatenate(vals) if vals else np.zeros(0, complex)
    return sp.coo_matrix((v, (r, c)), shape=(st.out_len, in_len)).tocsr()


def factor_matrices(fac: Factorization):
    """Sparse matrices of all stages in forward order."""
    mats = []
    in_len = fac.nw
    for st in fac.stages:
        M = stage_matrix(fac, st, in_len)
        mats.append(M)
        in_len = st.out_len
    return mats


def apply(fac: Factorization, f: np.ndarray, mats=None) -> np.ndarray:
    """g ~ K f = (prod of factors) f, eq. (finishIDBF)."""
    mats = factor_matrices(fac) if mats is None else mats
    v = np.asarray(f, dtype=np.complex128)
    for M in mats:
        v = M @ v
    return v


def apply_adjoint(fac: Factorization, g: np.ndarray, mats=None) -> np.ndarray:
    """f ~ K^H g: conjugate-transposed factors in reverse order."""
    mats = factor_matrices(fac) if mats is None else mats
    v = np.asarray(g, dtype=np.complex128)
    for M in reversed(mats):
        v = M.conj().T @ v
    return v


def dense(fac: Factorization, mats=None) -> np.ndarray:
    """The dense product of all factors (tiny problems only)."""
    mats = factor_matrices(fac) if mats is None else mats
    P = mats[0].toarray()
    for M in mats[1:]:
        P = M @ P
    return np.asarray(P)


def stored_entries(fac: Factorization) -> dict:
    """Counts of T entries (stored) and S entries (generated) per stage kind."""
    out = {"T": 0, "S": 0, "skel": 0}
    for st in fac.stages:
        for blk in st.blocks:
            if st.kind == KIND_S:
                out["S"] += blk.xidx.size * blk.widx.size
            else:
                for sub in blk.subs:
                    out["T"] += sub.T.size
                    out["skel"] += sub.skel.size
    return out
