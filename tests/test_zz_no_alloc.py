"""The allocation-free apply entry point (midbf_apply_noalloc).

Callers that cannot allocate device memory while applying the operator (a
service whose GPU memory belongs to another allocator, a latency-bound loop
where cudaMalloc would synchronize the device) use this call: it keeps its
intermediate vectors in the library's built-in 32 MiB scratch array instead
of a caller workspace.  It must give the same result as midbf_apply, on
repeated calls (the array keeps the previous call's contents), and reject
problems that do not fit the array.  This file is collected last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

import synth
from oracle import midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

TOL = {mb.FP64: 1e-12, mb.FP32: 2e-5}


def _plan():
    n = 32
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=16, tol=1e-6, t=2.0,
                      boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    return fac, mb.Plan.load(planio.write(fac))


@pytest.mark.parametrize("prec", [mb.FP32, mb.FP64])
def test_noalloc_matches_apply_twice(prec):
    fac, plan = _plan()
    dp = mb.DevicePlan(plan, prec)
    dt = torch.complex64 if prec == mb.FP32 else torch.complex128
    s = torch.cuda.current_stream().cuda_stream
    ws = torch.empty(dp.workspace_bytes(3), dtype=torch.uint8, device="cuda")
    for call in range(2):
        for adjoint in (0, 1):
            nin, nout = (fac.nx, fac.nw) if adjoint else (fac.nw, fac.nx)
            x = torch.from_numpy(synth.complex_gaussian(nin, 3, 20 + call + 2 * adjoint).T.copy()).to("cuda", dt)
            y_ref = torch.empty((3, nout), dtype=dt, device="cuda")
            y = torch.full((3, nout), complex(np.nan, np.nan), dtype=dt, device="cuda")
            mb.check(mb.midbf_apply(dp.h, adjoint, x.data_ptr(), nin, y_ref.data_ptr(), nout, 3, s,
                                    ws.data_ptr(), ws.numel()), "midbf_apply")
            mb.check(mb.midbf_apply_noalloc(dp.h, adjoint, x.data_ptr(), nin, y.data_ptr(), nout, 3, s),
                     "midbf_apply_noalloc")
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert np.isfinite(a).all() and err < TOL[prec], (call, adjoint, err)


@pytest.mark.parametrize("mode", [mb.BF16, mb.BF16 | mb.REFINE])
@pytest.mark.parametrize("nrhs", [16, 32])
def test_noalloc_tensor_core_modes_match_apply_twice(mode, nrhs):
    """With 16 or more right-hand sides the BF16 modes run the tensor-core
    kernels, whose RHS images sit in the scratch array after the vector
    buffers; that part of the layout must agree with a caller workspace too.
    Both calls use the same kernels in the same order, so the results agree
    bit for bit."""
    fac, plan = _plan()
    dp = mb.DevicePlan(plan, mode)
    assert dp.workspace_bytes(nrhs) <= mb.midbf_noalloc_scratch_bytes()
    s = torch.cuda.current_stream().cuda_stream
    ws = torch.empty(dp.workspace_bytes(nrhs), dtype=torch.uint8, device="cuda")
    for call in range(2):
        for adjoint in (0, 1):
            nin, nout = (fac.nx, fac.nw) if adjoint else (fac.nw, fac.nx)
            x = torch.from_numpy(synth.complex_gaussian(nin, nrhs, 40 + call + 2 * adjoint).T.copy()).to(
                "cuda", torch.complex64)
            y_ref = torch.empty((nrhs, nout), dtype=torch.complex64, device="cuda")
            y = torch.full((nrhs, nout), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
            mb.check(mb.midbf_apply(dp.h, adjoint, x.data_ptr(), nin, y_ref.data_ptr(), nout, nrhs, s,
                                    ws.data_ptr(), ws.numel()), "midbf_apply")
            mb.check(mb.midbf_apply_noalloc(dp.h, adjoint, x.data_ptr(), nin, y.data_ptr(), nout, nrhs, s),
                     "midbf_apply_noalloc")
            torch.cuda.synchronize()
            assert torch.equal(y, y_ref), (mode, nrhs, call, adjoint)
    assert dp.status() == mb.OK


def test_noalloc_argument_checks_match_apply():
    """The same argument checks as midbf_apply: a null pointer, nrhs <= 0,
    overlapping input and output, and profiling left on while the stream
    records a graph are all rejected with MIDBF_EINVAL."""
    fac, plan = _plan()
    dp = mb.DevicePlan(plan, mb.FP32)
    x = torch.zeros(fac.nw, dtype=torch.complex64, device="cuda")
    y = torch.zeros(fac.nx, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    assert mb.midbf_apply_noalloc(dp.h, 0, None, fac.nw, y.data_ptr(), fac.nx, 1, s.cuda_stream) == mb.EINVAL
    assert mb.midbf_apply_noalloc(dp.h, 0, x.data_ptr(), fac.nw, y.data_ptr(), fac.nx, 0, s.cuda_stream) == mb.EINVAL
    assert mb.midbf_apply_noalloc(dp.h, 0, x.data_ptr(), fac.nw, x.data_ptr(), fac.nx, 1, s.cuda_stream) == mb.EINVAL
    dp.profile(True)
    with mb.capture(s, keep=(x, y)):
        rc = mb.midbf_apply_noalloc(dp.h, 0, x.data_ptr(), fac.nw, y.data_ptr(), fac.nx, 1, s.cuda_stream)
    dp.profile(False)
    torch.cuda.synchronize()
    assert rc == mb.EINVAL
    assert b"profiling" in mb.midbf_last_error()


def test_noalloc_rejects_oversized_problem():
    fac, plan = _plan()
    dp = mb.DevicePlan(plan, mb.FP64)
    cap = mb.midbf_noalloc_scratch_bytes()
    assert cap == 32 << 20
    nrhs = 1
    while dp.workspace_bytes(nrhs) <= cap:
        nrhs *= 2
    x = torch.zeros((nrhs, fac.nw), dtype=torch.complex128, device="cuda")
    y = torch.zeros((nrhs, fac.nx), dtype=torch.complex128, device="cuda")
    rc = mb.midbf_apply_noalloc(dp.h, 0, x.data_ptr(), fac.nw, y.data_ptr(), fac.nx, nrhs,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == mb.EINVAL
    assert b"built-in" in mb.midbf_last_error()
