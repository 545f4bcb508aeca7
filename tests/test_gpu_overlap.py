"""Overlap of the middle factor with its neighbouring U stage (needs a GB300).

The middle factor S is generated on the fly (arithmetic-bound); the U stage
after it streams T (memory-bound).  The plan groups S's blocks so that each U
block reads the outputs of one group only, and the apply runs the pair chunk
by chunk with the second stage on a side stream.  The kernels and their
accumulation order are the same as with the overlap off, so every result must
be the same bit for bit: forward and adjoint, FP32 and FP64, one RHS and a
few, through midbf_apply, a recorded graph and midbf_apply_noalloc; and the
oracle's apply of the same factors bounds the result as for every apply.
Plans get the overlap only when asked (MIDBF_DPLAN_OVERLAP); without it they
have no chunks.
"""
import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

_C = {}


def _case(n):
    if n not in _C:
        X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=64, tol=1e-6, t=2.0,
                          boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
        _C[n] = (fac, mb.Plan.load(planio.write(fac)), midbf.factor_matrices(fac))
    return _C[n]


@pytest.mark.parametrize("prec,s_mode", [(mb.FP32, mb.S_ONTHEFLY), (mb.FP64, mb.S_ONTHEFLY), (mb.FP32, mb.S_STORED)])
def test_overlap_gives_the_same_bits(prec, s_mode):
    fac, plan, mats = _case(64)
    dp = mb.DevicePlan(plan, prec, s_mode, overlap=True)
    assert dp.overlap() > 1                       # four groups of four blocks at n = 64
    dt = dp.dtype()
    tol = 1e-12 if prec == mb.FP64 else 2e-5
    for nrhs in (1, 3):
        f = torch.from_numpy(synth.complex_gaussian(fac.nw, nrhs, 5).T.copy()).to("cuda", dt)
        if nrhs == 1:
            f = f[0]
        dp.set_overlap(True)
        g_on = dp.apply(f)
        a_on = dp.apply(g_on, adjoint=True)
        base = dp.launches(nrhs)
        dp.set_overlap(False)
        g_off = dp.apply(f)
        a_off = dp.apply(g_on, adjoint=True)
        torch.cuda.synchronize()
        assert torch.equal(g_on, g_off) and torch.equal(a_on, a_off), nrhs
        assert base == dp.launches(nrhs) + 2 * (4 - 1)
        ref = midbf.apply(fac, f.cpu().numpy().astype(np.complex128).T, mats)
        assert direct.rel_l2(g_on.cpu().numpy().T, ref) < tol
    dp.set_overlap(True)


def test_overlap_in_a_graph_and_without_allocation():
    fac, plan, _ = _case(64)
    dp = mb.DevicePlan(plan, mb.FP32, overlap=True)
    assert dp.overlap() > 1
    N = fac.nw
    f = torch.zeros(N, dtype=torch.complex64, device="cuda")
    g = torch.empty_like(f)
    h = torch.empty_like(f)
    ws = torch.empty(dp.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with mb.capture(s, keep=(f, g, h, ws)) as cap:
        dp.apply(f, out=g, workspace=ws, stream=s)
        dp.apply(g, adjoint=True, out=h, workspace=ws, stream=s)
    F = torch.from_numpy(synth.complex_gaussian(N, 1, 9)[:, 0]).to("cuda", torch.complex64)
    f.copy_(F)
    s.wait_stream(torch.cuda.current_stream())
    cap.graph.launch(s)
    s.synchronize()
    dp.set_overlap(False)
    g_ref = dp.apply(F)
    h_ref = dp.apply(g_ref, adjoint=True)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref) and torch.equal(h, h_ref)
    dp.set_overlap(True)
    y = torch.empty_like(f)
    cs = torch.cuda.current_stream().cuda_stream
    mb.check(mb.midbf_apply_noalloc(dp.h, 0, F.data_ptr(), N, y.data_ptr(), N, 1, cs), "midbf_apply_noalloc")
    torch.cuda.synchronize()
    assert torch.equal(y, g_ref)


def test_plans_have_no_overlap_unless_asked():
    fac, plan, _ = _case(64)
    assert mb.DevicePlan(plan, mb.FP32).overlap() == 0
    dp = mb.DevicePlan(plan, mb.FP32, overlap=True)
    assert dp.overlap() == 4
    assert dp.workspace_bytes(1) > mb.DevicePlan(plan, mb.FP32).workspace_bytes(1)   # the third vector
