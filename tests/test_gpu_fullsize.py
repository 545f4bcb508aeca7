"""Full-size check in the benchmark's launch configuration (needs a GB300).

The n = 256 FIO2D workload (N = 65,536) is built by the library and applied
on the GPU exactly as bench.py does (FP32 and FP64, one RHS, forward and
adjoint, the middle factor on the fly / stored).  The oracle computes sampled
outputs one by one by direct summation (eq. (1)): 256 rows of K f and 256
entries of K^H g.  The bound combines the construction's approximation error
(ID tolerance 1e-6 over 7 factor levels, measured ~1e-6 .. 1e-5 on smaller
grids) with the kernels' rounding.
"""
import numpy as np
import pytest

import synth
from oracle import direct
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

N_GRID = 256


@pytest.fixture(scope="module")
def plan():
    n = N_GRID
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    pl = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=64,
                       boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    return pl, OPhase(synth.PHASE_FIO2D, X, W)


@pytest.mark.parametrize("prec,s_mode", [(mb.FP32, mb.S_ONTHEFLY), (mb.FP64, mb.S_STORED)])
def test_fullsize_sampled_against_direct_sum(plan, prec, s_mode):
    pl, oph = plan
    N = N_GRID ** 2
    dp = mb.DevicePlan(pl, prec, s_mode)
    dt = torch.complex64 if prec == mb.FP32 else torch.complex128
    f = synth.complex_gaussian(N, 1, 0)[:, 0]
    h = synth.complex_gaussian(N, 1, 1)[:, 0]
    g = dp.apply(torch.from_numpy(f).to("cuda", dt)).cpu().numpy()
    a = dp.apply(torch.from_numpy(h).to("cuda", dt), adjoint=True).cpu().numpy()
    rows = synth.sample_rows(N, 256, 3)
    cols = synth.sample_rows(N, 256, 4)
    e_fwd = direct.rel_l2(g[rows], direct.direct_sum(oph, f, rows=rows))
    e_adj = direct.rel_l2(a[cols], direct.direct_adjoint(oph, h, cols=cols))
    assert e_fwd < 5e-5 and e_adj < 5e-5, (e_fwd, e_adj)


def test_fullsize_many_rhs_matches_single(plan):
    """The RHS-tiled kernels (20 RHS: one tile of 16 and a ragged tile of 4)
    give the same columns as 20 one-RHS applies."""
    pl, _ = plan
    N = N_GRID ** 2
    dp = mb.DevicePlan(pl, mb.FP32, mb.S_ONTHEFLY)
    F = torch.from_numpy(synth.complex_gaussian(N, 20, 5).T.copy()).to("cuda", torch.complex64)
    G = dp.apply(F)
    A = dp.apply(G, adjoint=True)
    for r in (0, 7, 16, 19):
        g1 = dp.apply(F[r].contiguous())
        a1 = dp.apply(G[r].contiguous(), adjoint=True)
        assert (torch.linalg.vector_norm(G[r] - g1) / torch.linalg.vector_norm(g1)).item() < 1e-6
        assert (torch.linalg.vector_norm(A[r] - a1) / torch.linalg.vector_norm(a1)).item() < 1e-6


def test_fullsize_tensor_cores_64_rhs(plan):
    """The tensor-core form (BF16 with the hi/lo refinement products) at the
    benchmark's size with 64 RHS: every column within 5e-5 of the FP32 apply of
    the same factors, and sampled rows of three columns within 1e-4 of the
    oracle's direct sum (the mixed-form bound)."""
    pl, oph = plan
    N = N_GRID ** 2
    R = 64
    F = synth.complex_gaussian(N, R, 9)
    Ft = torch.from_numpy(F.T.copy()).to("cuda", torch.complex64)
    d32 = mb.DevicePlan(pl, mb.FP32)
    dtc = mb.DevicePlan(pl, mb.BF16 | mb.REFINE)
    for adj in (False, True):
        g32 = d32.apply(Ft, adjoint=adj)
        gtc = dtc.apply(Ft, adjoint=adj)
        rel = (torch.linalg.vector_norm(gtc - g32) / torch.linalg.vector_norm(g32)).item()
        assert rel < 5e-5, (adj, rel)
    assert dtc.status() == mb.OK
    G = dtc.apply(Ft).cpu().numpy()
    rows = synth.sample_rows(N, 64, 3)
    for r in (0, 31, 63):
        e = direct.rel_l2(G[r][rows], direct.direct_sum(oph, F[:, r], rows=rows))
        assert e < 1e-4, (r, e)
