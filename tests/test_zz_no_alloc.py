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
