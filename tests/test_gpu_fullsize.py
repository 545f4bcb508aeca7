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


@pytest.mark.parametrize("R", [64, 256])
def test_fullsize_tensor_cores(plan, R):
    """The tensor-core form (BF16 with the hi/lo refinement products) at the
    benchmark's size with 64 RHS and with 256 RHS (one full pass of the TMEM
    accumulator): every column within 5e-5 of the FP32 apply of the same
    factors (rel-L2, and the largest entry error against the largest entry),
    and sampled rows of three columns within 1e-4 of the oracle's direct sum
    (the mixed-form bound)."""
    pl, oph = plan
    N = N_GRID ** 2
    F = synth.complex_gaussian(N, R, 9)
    Ft = torch.from_numpy(F.T.copy()).to("cuda", torch.complex64)
    d32 = mb.DevicePlan(pl, mb.FP32)
    dtc = mb.DevicePlan(pl, mb.BF16 | mb.REFINE)
    for adj in (False, True):
        g32 = d32.apply(Ft, adjoint=adj)
        gtc = dtc.apply(Ft, adjoint=adj)
        rel = (torch.linalg.vector_norm(gtc - g32) / torch.linalg.vector_norm(g32)).item()
        mx = ((gtc - g32).abs().max() / g32.abs().max()).item()
        assert rel < 5e-5 and mx < 5e-5, (adj, rel, mx)
    assert dtc.status() == mb.OK
    G = dtc.apply(Ft).cpu().numpy()
    rows = synth.sample_rows(N, 64, 3)
    for r in (0, R // 2 - 1, R - 1):
        e = direct.rel_l2(G[r][rows], direct.direct_sum(oph, F[:, r], rows=rows))
        assert e < 1e-4, (r, e)


def test_fullsize_autograd_finite_differences(plan):
    """Autograd through the FP32 apply on the n = 256 plan: the loss
    L(f) = Re <w, K f> is linear in f, so the central difference along each
    of 32 random directions d equals the directional derivative Re <grad, d>
    that the backward pass (the adjoint kernels) gives, up to rounding.  Two
    roundings enter: the FP32 accumulation of the applies (relative 1e-7 per
    stage, divided by the step h) and the difference between the FP32 phase
    of the forward and of the adjoint middle factor (~1e-5 relative, the FP32
    accuracy of the apply).  With h = 1e-2 ||f|| / ||d|| both stay below
    1e-4 of the scale ||w|| ||K d||."""
    pl, _ = plan
    N = N_GRID ** 2
    dp = mb.DevicePlan(pl, mb.FP32)
    rng = np.random.default_rng(2)
    f = torch.from_numpy(synth.complex_gaussian(N, 1, 0)[:, 0]).to("cuda", torch.complex64).requires_grad_(True)
    w = torch.from_numpy(synth.complex_gaussian(N, 1, 1)[:, 0]).to("cuda", torch.complex64)

    def loss(x):
        return torch.real(torch.vdot(w, mb.midbf_matvec(x, dp)))

    loss(f).backward()
    grad = f.grad.detach()
    nf = torch.linalg.vector_norm(f).item()
    nw = torch.linalg.vector_norm(w).item()
    for i in range(32):
        d = torch.from_numpy(rng.standard_normal(N) + 1j * rng.standard_normal(N)).to("cuda", torch.complex64)
        h = 1e-2 * nf / torch.linalg.vector_norm(d).item()
        with torch.no_grad():
            fd = (loss(f + h * d) - loss(f - h * d)) / (2 * h)
            scale = nw * torch.linalg.vector_norm(dp.apply(d)).item()
        dd = torch.real(torch.vdot(grad, d))
        assert abs(fd.item() - dd.item()) <= 1e-4 * scale, (i, fd.item(), dd.item(), scale)


def test_recovered_phase_end_to_end_example2():
    """Scenario 2 of Table 1 on Example 2 (x.xi over 32,768 random points per
    side in the unit cube): Algorithm 7 recovers a rank-4 phase from 8 rows
    and 8 columns of K (Algorithm 4 on the GPU), the library builds the
    factors of exp(2 pi i Psi) and the FP32 apply generates the middle factor
    from the low-rank phase (4 fused multiply-adds per entry).  Expected
    values are the oracle's direct sums of eq. (1) with the TRUE phase x.xi
    on 256 sampled rows and columns; recovery is exact to rounding (Table 4),
    so the bound is the mixed form's FP32 bound."""
    from oracle.phase import kernel as okernel
    w = synth.WORKLOADS["nuft3d_n32"]
    X, W, bx, bw = w.points()
    oph = OPhase(synth.PHASE_DOT, X, W)
    rows_fn = lambda idx: okernel(oph, idx[:, None], np.arange(w.nw)[None, :])
    cols_fn = lambda idx: okernel(oph, np.arange(w.nx)[:, None], idx[None, :])
    ph = mb.Phase.recover(X, W, rows_fn, cols_fn, r=4, q=2, seed=0, device=True)
    assert ph.info["rows_requested"] >= 8 and ph.info["cols_requested"] >= 8 and ph.info["mismatches"] == 0
    pl = mb.Plan.build(ph, tol=w.tol, n0=w.n0, boxX=bx, boxW=bw, device_ids=1)
    dp = mb.DevicePlan(pl, mb.FP32)
    f = w.rhs(1)[:, 0]
    h = synth.complex_gaussian(w.nx, 1, 11)[:, 0]
    g = dp.apply(torch.from_numpy(f).to("cuda", torch.complex64)).cpu().numpy()
    a = dp.apply(torch.from_numpy(h).to("cuda", torch.complex64), adjoint=True).cpu().numpy()
    rows = synth.sample_rows(w.nx, 256, 3)
    cols = synth.sample_rows(w.nw, 256, 4)
    e_fwd = direct.rel_l2(g[rows], direct.direct_sum(oph, f, rows=rows))
    e_adj = direct.rel_l2(a[cols], direct.direct_adjoint(oph, h, cols=cols))
    assert e_fwd < 2e-5 and e_adj < 2e-5, (e_fwd, e_adj)


def test_recovered_phase_paper_discretization():
    """Example 1 as the paper discretizes it (X and Omega both the uniform
    128 x 128 grid in [0,1)^2, Sec. 4) in Scenario 2: the phase recovered with
    r = 10, q = 2 (no discontinuity at tau = 1/4, as Sec. 4 reports), factors
    at the paper's ID tolerance 1e-9, the middle factor stored (10 low-rank
    terms).  The FP64 plain form and the FP32 mixed form against the oracle's
    direct sums with the true phase on 256 sampled rows: the plain form is
    limited by the recovery (eps^K ~ 5e-7 at r = 10), the mixed form by FP32."""
    from oracle.phase import kernel as okernel
    n = 128
    X = synth.uniform_grid(n, 2)
    W = synth.uniform_grid(n, 2)
    N = n * n
    oph = OPhase(synth.PHASE_FIO2D, X, W)
    rows_fn = lambda idx: okernel(oph, idx[:, None], np.arange(N)[None, :])
    cols_fn = lambda idx: okernel(oph, np.arange(N)[:, None], idx[None, :])
    ph = mb.Phase.recover(X, W, rows_fn, cols_fn, r=10, q=2, seed=0, device=True)
    assert ph.info["disc_rows"] == 0 and ph.info["disc_cols"] == 0 and ph.info["tau"] == 0.25
    pl = mb.Plan.build(ph, tol=1e-9, n0=64, t=5.0, boxX=(np.zeros(2), 1.0), boxW=(np.zeros(2), 1.0))
    f = synth.complex_gaussian(N, 1, 0)[:, 0]
    rows = synth.sample_rows(N, 256, 3)
    ref = direct.direct_sum(oph, f, rows=rows)
    for prec, dt, tol in ((mb.FP64, torch.complex128, 2e-6), (mb.FP32, torch.complex64, 2e-5)):
        dp = mb.DevicePlan(pl, prec, mb.S_STORED)
        g = dp.apply(torch.from_numpy(f).to("cuda", dt)).cpu().numpy()
        e = direct.rel_l2(g[rows], ref)
        assert e < tol, (prec, e)


def test_fullsize_accurate_phase(plan):
    """The mixed form with the accurate phase (double-FP32 middle-factor
    phases, MIDBF_S_ONTHEFLY_DF) at the benchmark's size: within 2e-6 of the
    FP64 plain form of the same factors (the ordinary FP32 phase is ~1e-5
    there: its rounding grows with the phase's magnitude, ~35 cycles at
    n = 256), and within 2e-6 of the oracle's direct sums on sampled rows
    (the factors themselves are accurate to ~6e-7)."""
    pl, oph = plan
    N = N_GRID ** 2
    ddf = mb.DevicePlan(pl, mb.FP32, mb.S_ONTHEFLY_DF)
    d64 = mb.DevicePlan(pl, mb.FP64, mb.S_STORED)
    f = synth.complex_gaussian(N, 1, 0)[:, 0]
    for adj in (False, True):
        gdf = ddf.apply(torch.from_numpy(f).to("cuda", torch.complex64), adjoint=adj).to(torch.complex128)
        g64 = d64.apply(torch.from_numpy(f).to("cuda", torch.complex128), adjoint=adj)
        rel = (torch.linalg.vector_norm(gdf - g64) / torch.linalg.vector_norm(g64)).item()
        assert rel < 2e-6, (adj, rel)
    g = ddf.apply(torch.from_numpy(f).to("cuda", torch.complex64)).cpu().numpy()
    rows = synth.sample_rows(N, 256, 3)
    e = direct.rel_l2(g[rows], direct.direct_sum(oph, f, rows=rows))
    assert e < 2e-6, e


def test_paper_grid_many_small_blocks():
    """Example 1 on the paper's grid (X and Omega the uniform 512 x 512 grid in
    [0,1)^2, Sec. 4) with the closed-form phase at ID tolerance 1e-9: 4,096
    leaf blocks of ranks ~10, so the one-RHS column stages run a warp per
    block (k_pattern_c1w) and the row stages the narrow or cluster kernels.
    FP64 and FP32, forward and adjoint, against FP64 direct sums of eq. (1) on
    256 sampled rows and columns."""
    n = 512
    X = synth.uniform_grid(n, 2)
    W = synth.uniform_grid(n, 2)
    N = n * n
    oph = OPhase(synth.PHASE_FIO2D, X, W)
    pl = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-9, n0=64, t=5.0,
                       boxX=(np.zeros(2), 1.0), boxW=(np.zeros(2), 1.0), device_ids=1)
    f = synth.complex_gaussian(N, 1, 0)[:, 0]
    h = synth.complex_gaussian(N, 1, 1)[:, 0]
    rows = synth.sample_rows(N, 256, 3)
    cols = synth.sample_rows(N, 256, 4)
    ref_f = direct.direct_sum(oph, f, rows=rows)
    ref_a = direct.direct_adjoint(oph, h, cols=cols)
    for prec, dt, tol in ((mb.FP64, torch.complex128, 1e-6), (mb.FP32, torch.complex64, 2e-5)):
        dp = mb.DevicePlan(pl, prec, mb.S_STORED)
        g = dp.apply(torch.from_numpy(f).to("cuda", dt)).cpu().numpy()
        a = dp.apply(torch.from_numpy(h).to("cuda", dt), adjoint=True).cpu().numpy()
        e_f, e_a = direct.rel_l2(g[rows], ref_f), direct.rel_l2(a[cols], ref_a)
        assert e_f < tol and e_a < tol, (prec, e_f, e_a)
        assert dp.status() == mb.OK
