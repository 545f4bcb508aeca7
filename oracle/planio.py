"""Reader and writer of the MIDBF level-program file (oracle side).

The file carries the factors of eq. (finishIDBF) as stages of blocks with
explicit index maps (see ``midbf``), so a factorization built here can be
applied by the GPU library, and one built by the library can be applied here.
The library has its own reader/writer; the two share only this layout:

  little-endian throughout
  char[8]  magic "MIDBFPL1"
  i32 d, L, delta, nsteps
  i64 nx, nw
  f64 tol
  i32 phase family, i32 r (low-rank terms, 0 for a closed form)
  f64 X[nx*d], W[nw*d]                 (row-major coordinates)
  if r > 0: f64 U[nx*r], V[nw*r]       (Psi = U V^T, row-major)
  i32 nstages
  per stage:
    i32 kind (0 = V, 1 = S, 2 = U), i32 in_space (-1 = user vector),
    i32 out_user (1 = output is the user vector), i32 pad (0)
    i64 out_len, i64 nblocks
    per block:
      i64 nin, i64 nout, i64 in_idx[nin], i64 out_idx[nout]
      kind S: i64 xidx[nout], i64 widx[nin]
      kind V/U: i32 nsub, i32 pad; per sub: i32 k, i32 m,
                i32 skel[k], i32 red[m-k], c128 T[k*(m-k)] (row-major)
                (m = nin for V, nout for U)

Parity: the reader is pinned in tests by a write/read round trip that must
reproduce the apply bit for bit.
"""
from __future__ import annotations

import io

import numpy as np

from .midbf import Block, Factorization, Stage, Sub, KIND_S, KIND_V
from .phase import Phase

MAGIC = b"MIDBFPL1"


def _w(buf, arr, dtype):
    buf.write(np.ascontiguousarray(np.asarray(arr, dtype=dtype)).tobytes())


def write(fac: Factorization) -> bytes:
    ph = fac.phase
    r = 0 if ph.U is None else ph.U.shape[1]
    buf = io.BytesIO()
    buf.write(MAGIC)
    _w(buf, [fac.d, fac.L, fac.delta, fac.nsteps], "<i4")
    _w(buf, [ph.X.shape[0], ph.W.shape[0]], "<i8")
    _w(buf, [fac.tol], "<f8")
    _w(buf, [ph.family, r], "<i4")
    _w(buf, ph.X, "<f8")
    _w(buf, ph.W, "<f8")
    if r:
        _w(buf, ph.U, "<f8")
        _w(buf, ph.V, "<f8")
    _w(buf, [len(fac.stages)], "<i4")
    for st in fac.stages:
        _w(buf, [st.kind, st.in_space, int(st.out_user), 0], "<i4")
        _w(buf, [st.out_len, len(st.blocks)], "<i8")
        for blk in st.blocks:
            _w(buf, [blk.in_idx.size, blk.out_idx.size], "<i8")
            _w(buf, blk.in_idx, "<i8")
            _w(buf, blk.out_idx, "<i8")
            if st.kind == KIND_S:
                _w(buf, blk.xidx, "<i8")
                _w(buf, blk.widx, "<i8")
                continue
            _w(buf, [len(blk.subs), 0], "<i4")
            for sub in blk.subs:
                k = sub.skel.size
                m = k + sub.red.size
                _w(buf, [k, m], "<i4")
                _w(buf, sub.skel, "<i4")
                _w(buf, sub.red, "<i4")
                _w(buf, sub.T, "<c16")
    return buf.getvalue()


class _Reader:
    def __init__(self, data: bytes):
        self.mv = memoryview(data)
        self.pos = 0

    def take(self, dtype, count):
        dt = np.dtype(dtype)
        nbytes = dt.itemsize * int(count)
        if self.pos + nbytes > len(self.mv):
            raise ValueError("truncated plan file")
        out = np.frombuffer(self.mv[self.pos:self.pos + nbytes], dtype=dt).copy()
        self.pos += nbytes
        return out


def read(data: bytes) -> Factorization:
    rd = _Reader(data)
    if bytes(rd.take("u1", 8)) != MAGIC:
        raise ValueError("not a MIDBF plan file")
    d, L, delta, nsteps = (int(v) for v in rd.take("<i4", 4))
    nx, nw = (int(v) for v in rd.take("<i8", 2))
    tol = float(rd.take("<f8", 1)[0])
    family, r = (int(v) for v in rd.take("<i4", 2))
    X = rd.take("<f8", nx * d).reshape(nx, d)
    W = rd.take("<f8", nw * d).reshape(nw, d)
    U = V = None
    if r:
        U = rd.take("<f8", nx * r).reshape(nx, r)
        V = rd.take("<f8", nw * r).reshape(nw, r)
    phase = Phase(family, X, W, U, V)
    nst = int(rd.take("<i4", 1)[0])
    stages = []
    for _ in range(nst):
        kind, in_space, out_user, _pad = (int(v) for v in rd.take("<i4", 4))
        out_len, nblocks = (int(v) for v in rd.take("<i8", 2))
        blocks = []
        for _b in range(nblocks):
            nin, nout = (int(v) for v in rd.take("<i8", 2))
            in_idx = rd.take("<i8", nin)
            out_idx = rd.take("<i8", nout)
            if kind == KIND_S:
                xidx = rd.take("<i8", nout)
                widx = rd.take("<i8", nin)
                blocks.append(Block(in_idx, out_idx, xidx=xidx, widx=widx))
                continue
            nsub, _p = (int(v) for v in rd.take("<i4", 2))
            subs = []
            for _s in range(nsub):
                k, m = (int(v) for v in rd.take("<i4", 2))
                skel = rd.take("<i4", k).astype(np.int64)
                red = rd.take("<i4", m - k).astype(np.int64)
                T = rd.take("<c16", k * (m - k)).reshape(k, m - k)
                subs.append(Sub(skel, red, T))
            blocks.append(Block(in_idx, out_idx, subs=subs))
        stages.append(Stage(kind, in_space, out_len, bool(out_user), blocks))
    if rd.pos != len(rd.mv):
        raise ValueError("trailing bytes in plan file")
    return Factorization(d, L, delta, nsteps, tol, phase, stages)
