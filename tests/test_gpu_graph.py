"""CUDA-graph recording of apply calls (needs a GB300).

midbf_capture_begin / midbf_capture_end record the kernel launches of a
forward + adjoint apply (or of a batched apply) once; every replay must give
exactly the outputs of the same calls issued directly, for new input
contents in the recorded buffers.  The apply kernels accumulate in a fixed
order (no atomics), so the comparison is bit for bit.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

_P = {}


def _plan(n):
    if n not in _P:
        X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
        _P[n] = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=64,
                              boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    return _P[n]


@pytest.mark.parametrize("mode,s_mode,nrhs", [(mb.FP32, mb.S_ONTHEFLY, 1), (mb.FP32, mb.S_ONTHEFLY, 20),
                                              (mb.BF16 | mb.REFINE, mb.S_ONTHEFLY, 40),
                                              (mb.FP64, mb.S_STORED, 3)])
def test_graph_replay_equals_direct_calls(mode, s_mode, nrhs):
    n = 64
    N = n * n
    dp = mb.DevicePlan(_plan(n), mode, s_mode)
    dt = dp.dtype()
    f = torch.zeros((nrhs, N), dtype=dt, device="cuda")
    g = torch.empty_like(f)
    h = torch.empty_like(f)
    ws = torch.empty(dp.workspace_bytes(nrhs), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with mb.capture(s, keep=(f, g, h, ws)) as cap:
        dp.apply(f, out=g, workspace=ws, stream=s)
        dp.apply(g, adjoint=True, out=h, workspace=ws, stream=s)
    for seed in (0, 1):
        F = torch.from_numpy(synth.complex_gaussian(N, nrhs, 70 + seed).T.copy()).to("cuda", dt)
        f.copy_(F)
        s.wait_stream(torch.cuda.current_stream())
        cap.graph.launch(s)
        s.synchronize()
        g_ref = dp.apply(F)
        h_ref = dp.apply(g_ref, adjoint=True)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref) and torch.equal(h, h_ref), seed
    assert dp.status() == mb.OK


def test_graph_of_batched_apply():
    plans = [_plan(32), _plan(64)]
    dps = [mb.DevicePlan(p, mb.FP32) for p in plans]
    adjoints = [0, 1, 0]
    idx = [0, 1, 1]
    nrhs = [1, 4, 9]
    sizes = [32 * 32, 64 * 64]
    xs = [torch.zeros((r, sizes[i]), dtype=torch.complex64, device="cuda") for i, r in zip(idx, nrhs)]
    outs = [torch.empty_like(x) for x in xs]
    sel = [dps[i] for i in idx]
    hs = (C.c_void_p * len(sel))(*[d.h.value for d in sel])
    nr = (C.c_int * len(sel))(*nrhs)
    need = C.c_size_t()
    mb.check(mb.midbf_batched_workspace_size(len(sel), hs, nr, C.byref(need)), "midbf_batched_workspace_size")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with mb.capture(s, keep=(*xs, *outs, ws)) as cap:
        mb.apply_batched(sel, xs, adjoints, outs=outs, workspace=ws, stream=s)
    for k, x in enumerate(xs):
        x.copy_(torch.from_numpy(synth.complex_gaussian(x.shape[1], x.shape[0], 90 + k).T.copy()).to("cuda"))
    s.wait_stream(torch.cuda.current_stream())
    cap.graph.launch(s)
    s.synchronize()
    for d, x, o, a in zip(sel, xs, outs, adjoints):
        ref = d.apply(x, adjoint=bool(a))
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


def test_host_apply_and_profiling_refused_while_recording():
    n = 32
    dp = mb.DevicePlan(_plan(n), mb.FP32)
    N = n * n
    f = torch.zeros(N, dtype=torch.complex64, device="cuda")
    g = torch.empty_like(f)
    ws = torch.empty(dp.workspace_bytes(1, host_io=True), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    host_in = np.zeros(N, np.complex64)
    host_out = np.zeros(N, np.complex64)
    with mb.capture(s, keep=(f, g, ws)):
        rc = mb.midbf_apply_host(dp.h, 0, host_in.ctypes.data, host_out.ctypes.data, 1, s.cuda_stream,
                                 ws.data_ptr(), ws.numel())
        assert rc == mb.EINVAL
        dp.profile(True)
        with pytest.raises(mb.MidbfError):
            dp.apply(f, out=g, workspace=ws, stream=s)
        dp.profile(False)
        dp.apply(f, out=g, workspace=ws, stream=s)
    torch.cuda.synchronize()
