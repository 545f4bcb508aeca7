"""GB300 MIDBF library: Python binding of the C ABI in include/midbf.h.

Argument marshalling only: every step of the apply runs in the library's CUDA
kernels, every step of the construction in its host C++.  The functions named
``midbf_*`` mirror the C entry points one to one; the small classes below own
the handles.  Importing this package loads ``libmidbf.so`` from this directory
and raises if it is missing (build it with ``python
paper_1908_09376_gb300/build.py``); there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmidbf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1908_09376_gb300/build.py`")
_lib = C.CDLL(LIB_PATH)

# ---- constants (include/midbf.h) ------------------------------------------
OK, EINVAL, ENOMEM, ECUDA, ECALLBACK, ERANK, ERECOVERY, ETIMEOUT, EINTERNAL, EFORMAT = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
CHOICE_DEFAULT, CHOICE_COLUMN1, CHOICE_PERSIST, CHOICE_TENSOR, CHOICE_NARROW, CHOICE_CLUSTER = 0, 32, 256, 1024, 64, 128
CHOICE_GEMM = 512
PHASE_FIO2D, PHASE_FIO3D, PHASE_FIO2D_JUMP, PHASE_DOT, PHASE_ZERO, PHASE_SEPARABLE, PHASE_LOWRANK = 1, 2, 3, 4, 5, 6, 7
PHASE_DISTANCE = 8
FP64, FP32, BF16, REFINE = 0, 1, 2, 16
S_ONTHEFLY, S_STORED, S_ONTHEFLY_DF = 0, 1, 2

_i64p = C.POINTER(C.c_int64)
_dblp = C.POINTER(C.c_double)
_vp = C.c_void_p


class midbf_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("n0", C.c_int), ("t", C.c_double), ("kest", C.c_int),
                ("kmax", C.c_int), ("seed", C.c_uint64), ("nthreads", C.c_int), ("use_box", C.c_int),
                ("boxX", C.c_double * 4), ("boxW", C.c_double * 4), ("device_ids", C.c_int),
                ("store_fp32", C.c_int)]


class midbf_stats(C.Structure):
    _fields_ = [("d", C.c_int), ("L", C.c_int), ("delta", C.c_int), ("nsteps", C.c_int), ("nstages", C.c_int),
                ("nx", C.c_int64), ("nw", C.c_int64), ("nblocks", C.c_int64), ("nsubs", C.c_int64),
                ("t_entries", C.c_int64), ("skel_entries", C.c_int64), ("s_entries", C.c_int64),
                ("index_entries", C.c_int64), ("max_rank", C.c_int), ("mean_rank", C.c_double)]


class midbf_recover_info(C.Structure):
    _fields_ = [("rows_requested", C.c_int64), ("cols_requested", C.c_int64), ("disc_rows", C.c_int64),
                ("disc_cols", C.c_int64), ("tau", C.c_double), ("mismatches", C.c_int64)]


ROWS_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, _i64p, C.c_int64, _dblp)


class midbf_access(C.Structure):
    _fields_ = [("rows_fn", ROWS_FN), ("cols_fn", ROWS_FN), ("user", C.c_void_p)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


midbf_last_error = _sig("midbf_last_error", C.c_char_p, [])
midbf_version = _sig("midbf_version", C.c_char_p, [])
midbf_phase_closed_form = _sig("midbf_phase_closed_form", C.c_int,
                               [C.c_int, C.c_int, C.c_int64, _dblp, C.c_int64, _dblp, C.POINTER(_vp)])
midbf_phase_lowrank = _sig("midbf_phase_lowrank", C.c_int,
                           [C.c_int, C.c_int64, _dblp, C.c_int64, _dblp, C.c_int, _dblp, _dblp, C.POINTER(_vp)])
midbf_phase_recover = _sig("midbf_phase_recover", C.c_int,
                           [C.c_int, C.c_int64, _dblp, C.c_int64, _dblp, C.POINTER(midbf_access), C.c_int, C.c_int,
                            C.c_double, C.c_int, C.c_uint64, C.POINTER(_vp), C.POINTER(midbf_recover_info)])
midbf_phase_recover_ex = _sig("midbf_phase_recover_ex", C.c_int,
                              [C.c_int, C.c_int64, _dblp, C.c_int64, _dblp, C.POINTER(midbf_access), C.c_int,
                               C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_int, C.POINTER(_vp),
                               C.POINTER(midbf_recover_info)])
RECOVER_DEVICE = 1
midbf_rpath_create = _sig("midbf_rpath_create", C.c_int, [C.c_int64, C.c_int64, _i64p, C.c_int64, C.POINTER(_vp)])
midbf_rpath_destroy = _sig("midbf_rpath_destroy", None, [_vp])
midbf_rpath_info = _sig("midbf_rpath_info", C.c_int, [_vp, _i64p, _i64p, C.POINTER(C.c_int)])
midbf_recover_vectors = _sig("midbf_recover_vectors", C.c_int,
                             [_vp, C.c_int, _vp, C.c_int64, _vp, C.c_int64, C.c_double, _vp, C.c_int64, _vp,
                              C.c_int64, _vp, _vp])
midbf_phase_eval = _sig("midbf_phase_eval", C.c_int, [_vp, C.c_int64, _i64p, _i64p, _dblp])
midbf_phase_factors = _sig("midbf_phase_factors", C.c_int, [_vp, C.POINTER(C.c_int), _dblp, _dblp])
midbf_phase_destroy = _sig("midbf_phase_destroy", None, [_vp])
midbf_params_default = _sig("midbf_params_default", C.c_int, [C.c_int, C.POINTER(midbf_params)])
midbf_build = _sig("midbf_build", C.c_int, [_vp, C.POINTER(midbf_params), C.POINTER(_vp)])
midbf_plan_export = _sig("midbf_plan_export", C.c_int, [_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)])
midbf_plan_import = _sig("midbf_plan_import", C.c_int, [_vp, C.c_size_t, C.POINTER(_vp)])
midbf_plan_stats = _sig("midbf_plan_stats", C.c_int, [_vp, C.POINTER(midbf_stats)])
midbf_plan_ranks = _sig("midbf_plan_ranks", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int32), C.c_int64,
                                                      C.POINTER(C.c_int64)])
midbf_plan_destroy = _sig("midbf_plan_destroy", None, [_vp])
midbf_free = _sig("midbf_free", None, [_vp])
midbf_dplan_create = _sig("midbf_dplan_create", C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(_vp)])
midbf_dplan_create_ex = _sig("midbf_dplan_create_ex", C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)])
DPLAN_CONSUME = 1
DPLAN_OVERLAP = 2
midbf_dplan_destroy = _sig("midbf_dplan_destroy", None, [_vp])
midbf_workspace_size = _sig("midbf_workspace_size", C.c_int, [_vp, C.c_int, C.POINTER(C.c_size_t)])
midbf_dplan_bytes = _sig("midbf_dplan_bytes", C.c_int, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)])
midbf_apply = _sig("midbf_apply", C.c_int,
                   [_vp, C.c_int, _vp, C.c_int64, _vp, C.c_int64, C.c_int, _vp, _vp, C.c_size_t])
midbf_apply_host = _sig("midbf_apply_host", C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp, _vp, C.c_size_t])
midbf_apply_launches = _sig("midbf_apply_launches", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)])
midbf_dplan_set_overlap = _sig("midbf_dplan_set_overlap", C.c_int, [_vp, C.c_int])
midbf_dplan_overlap = _sig("midbf_dplan_overlap", C.c_int, [_vp, C.POINTER(C.c_int)])
midbf_dplan_status = _sig("midbf_dplan_status", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)])
midbf_dplan_profile = _sig("midbf_dplan_profile", C.c_int, [_vp, C.c_int])
midbf_stage_times = _sig("midbf_stage_times", C.c_int,
                         [_vp, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int), _dblp, C.POINTER(C.c_int)])
midbf_autotune = _sig("midbf_autotune", C.c_int, [_vp, C.c_int, _vp])
midbf_wait_selftest = _sig("midbf_wait_selftest", C.c_int, [_vp, C.c_int, _vp])
midbf_set_choice = _sig("midbf_set_choice", C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int])
midbf_get_choice = _sig("midbf_get_choice", C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)])
midbf_capture_begin = _sig("midbf_capture_begin", C.c_int, [_vp])
midbf_capture_end = _sig("midbf_capture_end", C.c_int, [_vp, C.POINTER(_vp)])
midbf_graph_launch = _sig("midbf_graph_launch", C.c_int, [_vp, _vp])
midbf_graph_destroy = _sig("midbf_graph_destroy", None, [_vp])
midbf_stage_info = _sig("midbf_stage_info", C.c_int,
                        [_vp, C.c_int, C.POINTER(C.c_int), _i64p, _i64p, C.POINTER(C.c_int)])
midbf_batched_workspace_size = _sig("midbf_batched_workspace_size", C.c_int,
                                    [C.c_int, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(C.c_size_t)])
midbf_batched_launches = _sig("midbf_batched_launches", C.c_int,
                              [C.c_int, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)])
midbf_apply_batched = _sig("midbf_apply_batched", C.c_int,
                           [C.c_int, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(_vp), _i64p, C.POINTER(_vp),
                            _i64p, C.POINTER(C.c_int), _vp, _vp, C.c_size_t])
midbf_apply_noalloc = _sig("midbf_apply_noalloc", C.c_int,
                           [_vp, C.c_int, _vp, C.c_int64, _vp, C.c_int64, C.c_int, _vp])
midbf_noalloc_scratch_bytes = _sig("midbf_noalloc_scratch_bytes", C.c_size_t, [])
midbf_pipe_rates = _sig("midbf_pipe_rates", C.c_int, [_vp, _dblp, _dblp, _dblp])


def pipe_rates(stream=None):
    """(FP32 FMAs/s, SFU operations/s, FP64 FMAs/s) measured on the current device."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    check(midbf_pipe_rates(s.cuda_stream, C.byref(a), C.byref(b), C.byref(c)), "midbf_pipe_rates")
    return a.value, b.value, c.value

EXPORTED = [n for n in dir() if n.startswith("midbf_") and callable(globals()[n])
            and not isinstance(globals()[n], type)]


class MidbfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = midbf_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with code {code}: {msg}")


def check(rc, where):
    if rc != OK:
        raise MidbfError(rc, where)


def _f64(a, shape_last=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dblp)


class Phase:
    """Owns a midbf_phase handle."""

    def __init__(self, handle, d, nx, nw):
        self.h = handle
        self.d, self.nx, self.nw = d, nx, nw

    def __del__(self):
        if getattr(self, "h", None):
            midbf_phase_destroy(self.h)
            self.h = None

    @staticmethod
    def closed_form(family, X, W):
        X, px = _f64(X)
        W, pw = _f64(W)
        h = _vp()
        check(midbf_phase_closed_form(family, X.shape[1], X.shape[0], px, W.shape[0], pw, C.byref(h)),
              "midbf_phase_closed_form")
        return Phase(h, X.shape[1], X.shape[0], W.shape[0])

    @staticmethod
    def lowrank(X, W, U, V):
        X, px = _f64(X)
        W, pw = _f64(W)
        U, pu = _f64(U)
        V, pv = _f64(V)
        h = _vp()
        check(midbf_phase_lowrank(X.shape[1], X.shape[0], px, W.shape[0], pw, U.shape[1], pu, pv, C.byref(h)),
              "midbf_phase_lowrank")
        return Phase(h, X.shape[1], X.shape[0], W.shape[0])

    @staticmethod
    def recover(X, W, rows_fn, cols_fn, r=4, q=2, tau=0.25, max_disc=16, seed=0, device=False):
        """Algorithm 7 through the C ABI; rows_fn(idx) -> (len(idx), nw) complex K rows.
        device=True runs every vector recovery (Algorithm 4) on the current CUDA device."""
        X, px = _f64(X)
        W, pw = _f64(W)
        nx, nw = X.shape[0], W.shape[0]

        def _wrap(fn, length):
            def cb(user, idx, cnt, out):
                try:
                    ids = np.ctypeslib.as_array(idx, shape=(cnt,)).copy()
                    vals = np.ascontiguousarray(fn(ids), dtype=np.complex128).reshape(cnt, length)
                    C.memmove(out, vals.ctypes.data, vals.nbytes)
                    return 0
                except Exception:
                    return 1
            return ROWS_FN(cb)

        rcb = _wrap(rows_fn, nw)
        ccb = _wrap(lambda ids: np.asarray(cols_fn(ids)).T, nx)
        acc = midbf_access(rcb, ccb, None)
        info = midbf_recover_info()
        h = _vp()
        check(midbf_phase_recover_ex(X.shape[1], nx, px, nw, pw, C.byref(acc), r, q, tau, max_disc, seed,
                                     RECOVER_DEVICE if device else 0, C.byref(h), C.byref(info)),
              "midbf_phase_recover_ex")
        ph = Phase(h, X.shape[1], nx, nw)
        ph.info = {f: getattr(info, f) for f, _ in midbf_recover_info._fields_}
        return ph

    def eval(self, ix, iw):
        ix = np.ascontiguousarray(ix, dtype=np.int64).ravel()
        iw = np.ascontiguousarray(iw, dtype=np.int64).ravel()
        out = np.empty(ix.size)
        check(midbf_phase_eval(self.h, ix.size, ix.ctypes.data_as(_i64p), iw.ctypes.data_as(_i64p),
                               out.ctypes.data_as(_dblp)), "midbf_phase_eval")
        return out

    def factors(self):
        r = C.c_int()
        check(midbf_phase_factors(self.h, C.byref(r), None, None), "midbf_phase_factors")
        if r.value == 0:
            return None, None
        U = np.empty((self.nx, r.value))
        V = np.empty((self.nw, r.value))
        check(midbf_phase_factors(self.h, C.byref(r), U.ctypes.data_as(_dblp), V.ctypes.data_as(_dblp)),
              "midbf_phase_factors")
        return U, V


class RecoveryPath:
    """A recovery path (Def. 3.3) on the current CUDA device for Algorithm 4:
    edges is an (m, 2) integer array of (parent, child) pairs in path order."""

    def __init__(self, n, edges, root=None):
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 2))
        if root is None:
            root = int(e[0, 0]) if e.shape[0] else 0
        self.n, self.nedges, self.root = int(n), int(e.shape[0]), int(root)
        self.h = _vp()
        check(midbf_rpath_create(self.n, self.nedges, e.ctypes.data_as(_i64p), self.root, C.byref(self.h)),
              "midbf_rpath_create")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            midbf_rpath_destroy(self.h)
            self.h = _vp()

    def runs(self):
        nr = C.c_int()
        check(midbf_rpath_info(self.h, None, None, C.byref(nr)), "midbf_rpath_info")
        return nr.value

    def recover(self, u, tau, v0=None, stream=None):
        """Algorithm 4 for the rows of u (a (nvec, n) float64 CUDA tensor of
        observations modulo one), starting from v0 (default: u).  Returns
        (v, flags, D): recovered values, per-edge flags (uint8) and, per
        vector, the list D of the root and the flagged children."""
        import torch
        u = u.contiguous()
        nvec = u.shape[0]
        v = (u if v0 is None else v0).clone().contiguous()
        flags = torch.zeros((nvec, max(1, self.nedges)), dtype=torch.uint8, device=u.device)
        D = torch.zeros((nvec, self.nedges + 1), dtype=torch.int64, device=u.device)
        nD = torch.zeros(nvec, dtype=torch.int64, device=u.device)
        s = torch.cuda.current_stream(u.device) if stream is None else stream
        check(midbf_recover_vectors(self.h, nvec, u.data_ptr(), self.n, v.data_ptr(), self.n, float(tau),
                                    flags.data_ptr(), flags.shape[1], D.data_ptr(), D.shape[1], nD.data_ptr(),
                                    s.cuda_stream), "midbf_recover_vectors")
        s.synchronize()
        nd = nD.cpu().numpy()
        Dh = D.cpu().numpy()
        return v, flags[:, :self.nedges], [Dh[k, :nd[k]].tolist() for k in range(nvec)]


def params(d, **kw):
    p = midbf_params()
    check(midbf_params_default(d, C.byref(p)), "midbf_params_default")
    boxX = kw.pop("boxX", None)
    boxW = kw.pop("boxW", None)
    for k, v in kw.items():
        setattr(p, k, v)
    if boxX is not None and boxW is not None:
        p.use_box = 1
        for i, v in enumerate(list(boxX[0]) + [boxX[1]]):
            p.boxX[i] = float(v)
        for i, v in enumerate(list(boxW[0]) + [boxW[1]]):
            p.boxW[i] = float(v)
    return p


class Plan:
    """Owns a midbf_plan handle (host butterfly factors)."""

    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            midbf_plan_destroy(self.h)
            self.h = None

    @staticmethod
    def build(phase: Phase, **kw):
        p = params(phase.d, **kw)
        h = _vp()
        check(midbf_build(phase.h, C.byref(p), C.byref(h)), "midbf_build")
        return Plan(h)

    @staticmethod
    def load(data: bytes):
        buf = C.create_string_buffer(data, len(data))
        h = _vp()
        check(midbf_plan_import(buf, len(data), C.byref(h)), "midbf_plan_import")
        return Plan(h)

    def export(self) -> bytes:
        buf = _vp()
        n = C.c_size_t()
        check(midbf_plan_export(self.h, C.byref(buf), C.byref(n)), "midbf_plan_export")
        try:
            if n.value == 0:
                return b""
            arr = np.ctypeslib.as_array(C.cast(buf, C.POINTER(C.c_uint8)), shape=(n.value,))
            return arr.tobytes()
        finally:
            midbf_free(buf)

    def stats(self) -> dict:
        st = midbf_stats()
        check(midbf_plan_stats(self.h, C.byref(st)), "midbf_plan_stats")
        return {f: getattr(st, f) for f, _ in midbf_stats._fields_}

    def ranks(self, stage: int = -1) -> np.ndarray:
        """Ranks k of the interpolative decompositions of one stage (-1: all)."""
        cnt = C.c_int64()
        check(midbf_plan_ranks(self.h, stage, None, 0, C.byref(cnt)), "midbf_plan_ranks")
        out = np.empty(cnt.value, dtype=np.int32)
        check(midbf_plan_ranks(self.h, stage, out.ctypes.data_as(C.POINTER(C.c_int32)), out.size, C.byref(cnt)),
              "midbf_plan_ranks")
        return out


class DevicePlan:
    """Owns a midbf_dplan (plan resident on the current CUDA device)."""

    def __init__(self, plan: Plan, precision=FP32, s_mode=S_ONTHEFLY, consume=False, overlap=False):
        """consume=True releases the host plan's coefficients as they are uploaded
        (midbf_dplan_create_ex with MIDBF_DPLAN_CONSUME); overlap=True prepares the
        overlap of the middle factor with the U stage after it (MIDBF_DPLAN_OVERLAP)."""
        h = _vp()
        flags = (DPLAN_CONSUME if consume else 0) | (DPLAN_OVERLAP if overlap else 0)
        check(midbf_dplan_create_ex(plan.h, precision, s_mode, flags, C.byref(h)), "midbf_dplan_create_ex")
        self.h = h
        self.mode = precision
        self.precision = FP64 if precision == FP64 else FP32   # storage precision of the vectors
        st = plan.stats()
        self.nx, self.nw = st["nx"], st["nw"]

    def __del__(self):
        if getattr(self, "h", None):
            midbf_dplan_destroy(self.h)
            self.h = None

    def wait_selftest(self, ctas=4, stream=None):
        """Failure-detection self-test: bounded waits that run out set MIDBF_ETIMEOUT
        in this plan's status word (read it with status())."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        check(midbf_wait_selftest(self.h, ctas, s.cuda_stream), "midbf_wait_selftest")

    def status(self, reset=True):
        v = C.c_int()
        check(midbf_dplan_status(self.h, int(reset), C.byref(v)), "midbf_dplan_status")
        return v.value

    def workspace_bytes(self, nrhs, host_io=False):
        n = C.c_size_t()
        check(midbf_workspace_size(self.h, nrhs, C.byref(n)), "midbf_workspace_size")
        extra = (self.nx + self.nw) * nrhs * (8 if self.precision == FP32 else 16) if host_io else 0
        return n.value + extra

    def bytes(self):
        fb, ib = C.c_size_t(), C.c_size_t()
        check(midbf_dplan_bytes(self.h, C.byref(fb), C.byref(ib)), "midbf_dplan_bytes")
        return fb.value, ib.value

    def launches(self, nrhs=1):
        n = C.c_int()
        check(midbf_apply_launches(self.h, nrhs, C.byref(n)), "midbf_apply_launches")
        return n.value

    def set_overlap(self, enable=True):
        """Overlap the middle factor with its neighbouring U stage (chunked, on a side stream)."""
        check(midbf_dplan_set_overlap(self.h, int(enable)), "midbf_dplan_set_overlap")

    def overlap(self):
        v = C.c_int()
        check(midbf_dplan_overlap(self.h, C.byref(v)), "midbf_dplan_overlap")
        return v.value

    def profile(self, enable=True):
        check(midbf_dplan_profile(self.h, int(enable)), "midbf_dplan_profile")

    def stage_times(self):
        """[(kind, ms, algorithmic bytes)] of the stages of the last profiled apply."""
        ms = (C.c_float * 64)()
        kinds = (C.c_int * 64)()
        by = (C.c_double * 64)()
        n = C.c_int()
        check(midbf_stage_times(self.h, 64, ms, kinds, by, C.byref(n)), "midbf_stage_times")
        return [(kinds[i], ms[i], by[i]) for i in range(n.value)]

    def autotune(self, nrhs, stream=None):
        """Time every kernel variant of every stage for nrhs RHS and keep the fastest."""
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        check(midbf_autotune(self.h, nrhs, C.c_void_p(s.cuda_stream)), "midbf_autotune")

    def set_choice(self, nrhs, stage, adjoint, choice):
        check(midbf_set_choice(self.h, nrhs, stage, int(adjoint), choice), "midbf_set_choice")

    def choice(self, nrhs, stage, adjoint):
        c = C.c_int()
        check(midbf_get_choice(self.h, nrhs, stage, int(adjoint), C.byref(c)), "midbf_get_choice")
        return c.value

    def stage_info(self):
        """[(kind, factor entries, dense entries)] of every stage in forward order."""
        kinds = (C.c_int * 64)()
        ent = np.zeros(64, np.int64)
        den = np.zeros(64, np.int64)
        n = C.c_int()
        check(midbf_stage_info(self.h, 64, kinds, ent.ctypes.data_as(_i64p), den.ctypes.data_as(_i64p),
                               C.byref(n)), "midbf_stage_info")
        return [(kinds[i], int(ent[i]), int(den[i])) for i in range(n.value)]

    # -- torch helpers (device memory and streams come from PyTorch) --------
    def dtype(self):
        import torch
        return torch.complex64 if self.precision == FP32 else torch.complex128

    def apply(self, x, adjoint=False, out=None, workspace=None, stream=None):
        """y = K x (or K^H x) for a CUDA tensor x of shape (n,) or (nrhs, n) (one RHS per row)."""
        import torch
        if not x.is_cuda:
            raise ValueError("x must be a CUDA tensor")
        if x.dtype != self.dtype():
            raise TypeError(f"x must be {self.dtype()}")
        vec = x.dim() == 1
        xs = x.reshape(1, -1) if vec else x
        xs = xs.contiguous()
        nrhs, nin = xs.shape
        nout = self.nw if adjoint else self.nx
        if nin != (self.nx if adjoint else self.nw):
            raise ValueError("x has the wrong length")
        if out is None:
            out = torch.empty((nrhs, nout), dtype=x.dtype, device=x.device)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes(nrhs), dtype=torch.uint8, device=x.device)
        s = torch.cuda.current_stream(x.device) if stream is None else stream
        check(midbf_apply(self.h, int(adjoint), xs.data_ptr(), nin, out.data_ptr(), nout, nrhs,
                          s.cuda_stream, workspace.data_ptr(), workspace.numel()), "midbf_apply")
        return out.reshape(-1) if vec else out

    def apply_host(self, x: np.ndarray, adjoint=False, workspace=None, stream=None):
        """Host arrays in and out through midbf_apply_host (copies inside the call)."""
        import torch
        dt = np.complex64 if self.precision == FP32 else np.complex128
        xs = np.ascontiguousarray(x, dtype=dt)
        vec = xs.ndim == 1
        xs = xs.reshape(1, -1) if vec else xs
        nrhs = xs.shape[0]
        out = np.empty((nrhs, self.nw if adjoint else self.nx), dtype=dt)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes(nrhs, True), dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream() if stream is None else stream
        check(midbf_apply_host(self.h, int(adjoint), xs.ctypes.data, out.ctypes.data, nrhs, s.cuda_stream,
                               workspace.data_ptr(), workspace.numel()), "midbf_apply_host")
        return out.reshape(-1) if vec else out


class Graph:
    """A recorded sequence of apply calls (midbf_capture_begin/_end), replayed
    with one launch.  The buffers named in the recorded calls must outlive it."""

    def __init__(self, handle, keep):
        self.h = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "h", None):
            midbf_graph_destroy(self.h)
            self.h = None

    def launch(self, stream=None):
        import torch
        s = stream or torch.cuda.current_stream()
        check(midbf_graph_launch(self.h, C.c_void_p(s.cuda_stream)), "midbf_graph_launch")


class capture:
    """Context manager recording the apply calls issued on `stream` (a
    non-default torch.cuda.Stream, made current inside the block) into a
    Graph, available as .graph after the block.  `keep` holds references to
    the tensors the recorded calls use."""

    def __init__(self, stream, keep=()):
        self.stream = stream
        self.keep = list(keep)
        self.graph = None

    def __enter__(self):
        import torch
        self._ctx = torch.cuda.stream(self.stream)
        self._ctx.__enter__()
        check(midbf_capture_begin(C.c_void_p(self.stream.cuda_stream)), "midbf_capture_begin")
        return self

    def __exit__(self, et, ev, tb):
        h = _vp()
        rc = midbf_capture_end(C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self._ctx.__exit__(et, ev, tb)
        if et is None:
            check(rc, "midbf_capture_end")
            self.graph = Graph(h, self.keep)
        elif rc == OK:
            midbf_graph_destroy(h)
        return False


def batched_launches(dplans, adjoints, nrhs):
    """Kernel launches one apply_batched call issues for these instances."""
    n = len(dplans)
    hs = (_vp * n)(*[d.h.value for d in dplans])
    adj = (C.c_int * n)(*[int(a) for a in adjoints])
    nr = (C.c_int * n)(*[int(r) for r in nrhs])
    out = C.c_int()
    check(midbf_batched_launches(n, hs, adj, nr, C.byref(out)), "midbf_batched_launches")
    return out.value


def batched_workspace_bytes(dplans, nrhs):
    n = len(dplans)
    hs = (_vp * n)(*[d.h.value for d in dplans])
    nr = (C.c_int * n)(*[int(r) for r in nrhs])
    need = C.c_size_t()
    check(midbf_batched_workspace_size(n, hs, nr, C.byref(need)), "midbf_batched_workspace_size")
    return need.value


def apply_batched(dplans, xs, adjoints, outs=None, workspace=None, stream=None):
    """Batched apply through midbf_apply_batched.  xs[i]: CUDA tensor (nrhs_i, n_in_i)
    (one RHS per row); returns the outputs (nrhs_i, n_out_i)."""
    import torch
    n = len(dplans)
    xs = [x.reshape(1, -1) if x.dim() == 1 else x for x in xs]
    xs = [x.contiguous() for x in xs]
    nrhs = (C.c_int * n)(*[x.shape[0] for x in xs])
    adj = (C.c_int * n)(*[int(a) for a in adjoints])
    hs = (_vp * n)(*[d.h.value for d in dplans])
    if outs is None:
        outs = [torch.empty((x.shape[0], d.nw if a else d.nx), dtype=x.dtype, device=x.device)
                for d, x, a in zip(dplans, xs, adjoints)]
    ins = (_vp * n)(*[x.data_ptr() for x in xs])
    ots = (_vp * n)(*[o.data_ptr() for o in outs])
    ldi = (C.c_int64 * n)(*[x.shape[1] for x in xs])
    ldo = (C.c_int64 * n)(*[o.shape[1] for o in outs])
    need = C.c_size_t()
    check(midbf_batched_workspace_size(n, hs, nrhs, C.byref(need)), "midbf_batched_workspace_size")
    if workspace is None:
        workspace = torch.empty(need.value, dtype=torch.uint8, device=xs[0].device)
    s = torch.cuda.current_stream(xs[0].device) if stream is None else stream
    check(midbf_apply_batched(n, hs, adj, ins, ldi, ots, ldo, nrhs, s.cuda_stream, workspace.data_ptr(),
                              workspace.numel()), "midbf_apply_batched")
    return outs


def _autograd():
    import torch

    class MIDBFApply(torch.autograd.Function):
        """g = K f with backward grad_f = K^H grad_g (PyTorch's complex convention)."""

        @staticmethod
        def forward(ctx, f, dplan, adjoint):
            ctx.dplan = dplan
            ctx.adjoint = adjoint
            return dplan.apply(f.detach(), adjoint=adjoint)

        @staticmethod
        def backward(ctx, grad):
            return ctx.dplan.apply(grad.contiguous(), adjoint=not ctx.adjoint), None, None

    return MIDBFApply


_MIDBFApply = None


def midbf_matvec(f, dplan: DevicePlan, adjoint: bool = False):
    """Differentiable g = K f (or K^H f) through the hand-written forward and adjoint kernels."""
    global _MIDBFApply
    if _MIDBFApply is None:
        _MIDBFApply = _autograd()
    return _MIDBFApply.apply(f, dplan, adjoint)
