"""Failure detection without a GPU fault (needs a GB300).

The tensor-core kernels wait on mbarriers with a bounded wait: after 2 s (or
at once when another CTA has already given up) the wait returns, the kernel
writes MIDBF_ETIMEOUT into the plan's status word and exits.  The self-test
runs that same wait on an mbarrier that nothing arrives on, so the wait must
run out.  The host then reads the status word, clears it, and the context
keeps working: the next apply gives the same result as before.
"""
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_survives():
    n = 32
    X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16,
                         boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    dp = mb.DevicePlan(plan, mb.FP32)
    f = torch.from_numpy(synth.complex_gaussian(n * n, 1, 0)[:, 0]).to("cuda", torch.complex64)
    g0 = dp.apply(f)
    torch.cuda.synchronize()
    assert dp.status() == mb.OK
    t0 = time.perf_counter()
    dp.wait_selftest(ctas=4)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert 1.5 < dt < 30.0, dt                 # the 2 s limit, not a hang
    assert dp.status(reset=True) == mb.ETIMEOUT
    assert dp.status() == mb.OK                # cleared
    g1 = dp.apply(f)
    torch.cuda.synchronize()
    assert torch.equal(g0, g1)
    with pytest.raises(mb.MidbfError):
        dp.wait_selftest(ctas=0)


def test_tensor_core_kernels_give_up_once_the_status_word_is_set():
    """A tensor-core apply issued while the plan's status word already reads
    MIDBF_ETIMEOUT (left set by the self-test, not reset) must return without
    waiting out any limit: every bounded wait in the pipelines checks the word
    and gives up at once, the CTAs drain their copies in flight, free their
    tensor memory and exit.  The status stays MIDBF_ETIMEOUT; after a reset the
    next apply gives exactly the result of an apply before the failure."""
    n = 32
    X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16,
                         boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    for mode in (mb.BF16, mb.BF16 | mb.REFINE):
        dp = mb.DevicePlan(plan, mode)
        F = torch.from_numpy(synth.complex_gaussian(n * n, 32, 3).T.copy()).to("cuda", torch.complex64)
        g0 = dp.apply(F)
        a0 = dp.apply(g0, adjoint=True)
        torch.cuda.synchronize()
        assert dp.status() == mb.OK
        dp.wait_selftest(ctas=2)
        torch.cuda.synchronize()
        assert dp.status(reset=False) == mb.ETIMEOUT
        t0 = time.perf_counter()
        dp.apply(F)                              # 32 RHS: every stage on the tensor cores
        dp.apply(g0, adjoint=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert dt < 1.5, dt                      # no CTA waited out the 2 s limit
        assert dp.status(reset=True) == mb.ETIMEOUT
        assert dp.status() == mb.OK
        g1 = dp.apply(F)
        a1 = dp.apply(g1, adjoint=True)
        torch.cuda.synchronize()
        assert dp.status() == mb.OK
        assert torch.equal(g0, g1) and torch.equal(a0, a1)
