"""GPU parity of the MIDBF apply against the CPU FP64 oracle (needs a GB300).

Parity is checked element by element on the SAME factors: plans built by the
oracle (no product code involved in the inputs or the expected values) are
imported into the library and applied on the GPU; the oracle applies them
with its own sparse factor product.  Library-built plans are also checked
against the oracle's apply of the exported file and against the direct sum.

Tolerances (relative L2 over all outputs, and max abs error over max |ref|):
  FP64 plain form   1e-12  (rounding of ~1e3-term sums in FP64; the target
                            is 1e-6, kept 10^6 tighter)
  FP32 mixed form   2e-5   (FP32 storage of T (6e-8) and data, ~10 stages,
                            and FP32 phases of magnitude <= ~50 in the
                            on-the-fly middle factor; the target is 1e-4)
"""
import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

TOL = {mb.FP64: 1e-12, mb.FP32: 2e-5}


def _dt(prec):
    return torch.complex64 if prec == mb.FP32 else torch.complex128


def _check(got, ref, tol, what):
    e = direct.rel_l2(got, ref)
    m = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < tol and m < 10 * tol, f"{what}: rel-L2 {e:.3e}, max {m:.3e}"


def _grid(n, d=2):
    X = synth.uniform_grid(n, d)
    W = synth.frequency_grid(n, d)
    return X, W, (np.zeros(d), 1.0), (np.full(d, -n / 2), float(n))


_CACHE = {}


def oracle_case(name):
    """Oracle-built factorizations spanning odd/even L, ragged ranks, 3D, L=0."""
    if name in _CACHE:
        return _CACHE[name]
    if name == "fio2d_n32_L3":
        X, W, bx, bw = _grid(32)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=16, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    elif name == "fio2d_n64_L3":
        X, W, bx, bw = _grid(64)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=64, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    elif name == "dot_n16_L2":
        X, W, bx, bw = _grid(16)
        fac = midbf.build(OPhase(synth.PHASE_DOT, X, W), n0=4, tol=1e-8, t=2.0, boxX=bx, boxW=bw)
    elif name == "jump_n32_L2":
        X, W, bx, bw = _grid(32)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D_JUMP, X, W), n0=64, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    elif name == "fio3d_n8_L2":
        X = synth.uniform_random_points(512, 3, 0)
        W = synth.frequency_grid(8, 3)
        fac = midbf.build(OPhase(synth.PHASE_FIO3D, X, W), n0=8, tol=1e-7, t=2.0,
                          boxX=(np.zeros(3), 1.0), boxW=(np.full(3, -4.0), 8.0))
    elif name == "lowrank_n32_L3":
        X, W, bx, bw = _grid(32)
        rng = np.random.default_rng(5)
        U = np.concatenate([X, 0.01 * rng.standard_normal((1024, 2))], axis=1)
        V = np.concatenate([W, rng.standard_normal((1024, 2))], axis=1)
        fac = midbf.build(OPhase(synth.PHASE_LOWRANK, X, W, U, V), n0=16, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    elif name == "fio2d_n8_L0":
        X, W, bx, bw = _grid(8)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=64, tol=1e-6, boxX=bx, boxW=bw)
    else:
        raise KeyError(name)
    out = (fac, mb.Plan.load(planio.write(fac)), midbf.factor_matrices(fac))
    _CACHE[name] = out
    return out


CASES = ["fio2d_n32_L3", "fio2d_n64_L3", "dot_n16_L2", "jump_n32_L2", "fio3d_n8_L2", "lowrank_n32_L3",
         "fio2d_n8_L0"]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [mb.FP64, mb.FP32])
@pytest.mark.parametrize("s_mode", [mb.S_ONTHEFLY, mb.S_STORED])
def test_apply_matches_oracle_on_oracle_plans(case, prec, s_mode):
    fac, plan, mats = oracle_case(case)
    dp = mb.DevicePlan(plan, prec, s_mode)
    dev = torch.device("cuda:0")
    for nrhs in (1, 3, 20):
        f = synth.complex_gaussian(fac.nw, nrhs, 11)
        h = synth.complex_gaussian(fac.nx, nrhs, 12)
        g = dp.apply(torch.from_numpy(f.T.copy()).to(dev, _dt(prec))).cpu().numpy().T
        a = dp.apply(torch.from_numpy(h.T.copy()).to(dev, _dt(prec)), adjoint=True).cpu().numpy().T
        g_ref = np.stack([midbf.apply(fac, f[:, r], mats) for r in range(nrhs)], 1)
        a_ref = np.stack([midbf.apply_adjoint(fac, h[:, r], mats) for r in range(nrhs)], 1)
        _check(g, g_ref, TOL[prec], f"{case} forward nrhs={nrhs}")
        _check(a, a_ref, TOL[prec], f"{case} adjoint nrhs={nrhs}")


@pytest.mark.parametrize("prec", [mb.FP64, mb.FP32])
def test_library_plan_matches_oracle_and_direct_sum(prec):
    X, W, bx, bw = _grid(64)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=64, boxX=bx, boxW=bw)
    fac = planio.read(plan.export())
    dp = mb.DevicePlan(plan, prec)
    f = synth.complex_gaussian(4096, 1, 0)[:, 0]
    g = dp.apply(torch.from_numpy(f).cuda().to(_dt(prec))).cpu().numpy()
    _check(g, midbf.apply(fac, f), TOL[prec], "library plan vs oracle apply")
    assert direct.rel_l2(g, direct.direct_sum(OPhase(synth.PHASE_FIO2D, X, W), f)) < 2e-5


def test_adjoint_identity_and_strided_io():
    fac, plan, _ = oracle_case("fio2d_n64_L3")
    dp = mb.DevicePlan(plan, mb.FP64)
    rng = np.random.default_rng(3)
    f = synth.complex_gaussian(fac.nw, 2, 1)
    h = synth.complex_gaussian(fac.nx, 2, 2)
    F = torch.from_numpy(f.T.copy()).cuda()
    H = torch.from_numpy(h.T.copy()).cuda()
    g = dp.apply(F)
    a = dp.apply(H, adjoint=True)
    lhs = torch.vdot(H.reshape(-1), g.reshape(-1)).item()
    rhs = torch.vdot(a.reshape(-1), F.reshape(-1)).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # padded leading dimensions through the raw C entry point
    ld_in, ld_out = fac.nw + 7, fac.nx + 5
    Fp = torch.zeros((2, ld_in), dtype=torch.complex128, device="cuda")
    Fp[:, :fac.nw] = F
    Gp = torch.full((2, ld_out), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    ws = torch.empty(dp.workspace_bytes(2), dtype=torch.uint8, device="cuda")
    mb.check(mb.midbf_apply(dp.h, 0, Fp.data_ptr(), ld_in, Gp.data_ptr(), ld_out, 2,
                            torch.cuda.current_stream().cuda_stream, ws.data_ptr(), ws.numel()), "apply")
    torch.cuda.synchronize()
    assert torch.equal(Gp[:, :fac.nx], g)
    assert torch.isnan(Gp[:, fac.nx:].real).all()   # padding untouched


def test_apply_argument_errors():
    fac, plan, _ = oracle_case("fio2d_n32_L3")
    dp = mb.DevicePlan(plan, mb.FP32)
    x = torch.zeros(fac.nw, dtype=torch.complex64, device="cuda")
    y = torch.zeros(fac.nx, dtype=torch.complex64, device="cuda")
    ws = torch.empty(dp.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert mb.midbf_apply(dp.h, 0, x.data_ptr(), fac.nw - 1, y.data_ptr(), fac.nx, 1, s, ws.data_ptr(),
                          ws.numel()) == mb.EINVAL
    assert mb.midbf_apply(dp.h, 0, x.data_ptr(), fac.nw, y.data_ptr(), fac.nx, 1, s, ws.data_ptr(), 16) == mb.EINVAL
    assert mb.midbf_apply(dp.h, 0, x.data_ptr(), fac.nw, x.data_ptr(), fac.nw, 1, s, ws.data_ptr(),
                          ws.numel()) == mb.EINVAL   # overlapping in/out
    assert mb.midbf_apply(dp.h, 0, x.data_ptr(), fac.nw, y.data_ptr(), fac.nx, 0, s, ws.data_ptr(),
                          ws.numel()) == mb.EINVAL


def test_apply_host_matches_device_apply():
    fac, plan, _ = oracle_case("fio2d_n32_L3")
    dp = mb.DevicePlan(plan, mb.FP32)
    f = synth.complex_gaussian(fac.nw, 2, 4).T.astype(np.complex64)
    g_host = dp.apply_host(f)
    g_dev = dp.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.array_equal(g_host, g_dev)


def test_autograd_finite_differences():
    """g = K f is linear: central differences of a real loss along 32 random
    directions equal the directional derivative from the adjoint kernel."""
    fac, plan, _ = oracle_case("fio2d_n32_L3")
    dp = mb.DevicePlan(plan, mb.FP64)
    rng = np.random.default_rng(2)
    f = torch.from_numpy(synth.complex_gaussian(fac.nw, 1, 0)[:, 0]).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.complex_gaussian(fac.nx, 1, 1)[:, 0]).cuda()

    def loss(x):
        return torch.real(torch.vdot(w, mb.midbf_matvec(x, dp)))

    L0 = loss(f)
    L0.backward()
    grad = f.grad.detach()
    for i in range(32):
        d = torch.from_numpy(rng.standard_normal(fac.nw) + 1j * rng.standard_normal(fac.nw)).cuda()
        h = 1e-3
        with torch.no_grad():
            fd = (loss(f + h * d) - loss(f - h * d)) / (2 * h)
        dd = torch.real(torch.vdot(grad, d))
        assert abs(fd.item() - dd.item()) <= 1e-9 * max(1.0, abs(dd.item())), i


# The accurate phase (MIDBF_S_ONTHEFLY_DF): every middle-factor entry's phase
# in double-FP32 arithmetic.  What remains of the FP32 error is the storage of
# T and the vectors in FP32 (6e-8 relative), FP32 accumulation over ~10
# stages, and the SFU sine/cosine (absolute error ~4e-7): bound 2e-6, ten
# times tighter than the FP32 bound, and the result must beat the ordinary
# FP32 phase on the same factors.
DF_TOL = 2e-6


@pytest.mark.parametrize("case", ["fio2d_n32_L3", "fio2d_n64_L3", "jump_n32_L2", "fio3d_n8_L2", "lowrank_n32_L3",
                                  "dot_n16_L2"])
def test_accurate_phase_matches_oracle(case):
    fac, plan, mats = oracle_case(case)
    dp = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY_DF)
    dq = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY)
    for nrhs in (1, 3):
        f = synth.complex_gaussian(fac.nw, nrhs, 30 + nrhs)
        y = synth.complex_gaussian(fac.nx, nrhs, 40 + nrhs)
        F = torch.from_numpy(f.T.copy()).to("cuda", torch.complex64)
        Y = torch.from_numpy(y.T.copy()).to("cuda", torch.complex64)
        g = dp.apply(F).cpu().numpy().T
        a = dp.apply(Y, adjoint=True).cpu().numpy().T
        g_ref = midbf.apply(fac, f, mats)
        a_ref = midbf.apply_adjoint(fac, y, mats)
        _check(g, g_ref, DF_TOL, f"{case} accurate forward nrhs={nrhs}")
        _check(a, a_ref, DF_TOL, f"{case} accurate adjoint nrhs={nrhs}")
        gq = dq.apply(F).cpu().numpy().T
        assert direct.rel_l2(g, g_ref) <= direct.rel_l2(gq, g_ref) * 1.01 + 1e-7, case


def test_accurate_phase_rejections():
    fac, plan, _ = oracle_case("fio2d_n32_L3")
    for prec in (mb.FP64, mb.BF16, mb.BF16 | mb.REFINE):
        with pytest.raises(mb.MidbfError) as e:
            mb.DevicePlan(plan, prec, mb.S_ONTHEFLY_DF)
        assert e.value.code == mb.EINVAL
    dp = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY_DF)
    x = torch.zeros(fac.nw, dtype=torch.complex64, device="cuda")
    with pytest.raises(mb.MidbfError):
        mb.apply_batched([dp], [x], [0])


def _paper_grid_case():
    """Example 1 on the paper's grid (X and Omega both in [0,1)^2), n = 32, ID
    tolerance 1e-9: ranks of ~10-30, so every stage takes the narrow-ID kernels."""
    if "paper_n32" not in _CACHE:
        X, W = synth.uniform_grid(32, 2), synth.uniform_grid(32, 2)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=16, tol=1e-9, t=2.0,
                          boxX=(np.zeros(2), 1.0), boxW=(np.zeros(2), 1.0))
        _CACHE["paper_n32"] = (fac, mb.Plan.load(planio.write(fac)), midbf.factor_matrices(fac))
    return _CACHE["paper_n32"]


@pytest.mark.parametrize("prec", [mb.FP64, mb.FP32])
def test_narrow_id_kernels_match_oracle(prec):
    """One RHS on low-rank factors: the narrow-ID kernels (a warp per ID for
    the row pattern, a lane per column for the column pattern) against the
    oracle, by default on the paper-grid plan (its column stages; its row
    stages have too few IDs per SM and take the cluster kernel) and forced on
    every stage of a plan whose ranks reach 64."""
    fac, plan, mats = _paper_grid_case()
    dp = mb.DevicePlan(plan, prec)
    f = synth.complex_gaussian(fac.nw, 1, 50)[:, 0]
    y = synth.complex_gaussian(fac.nx, 1, 51)[:, 0]
    g = dp.apply(torch.from_numpy(f).to("cuda", _dt(prec))).cpu().numpy()
    a = dp.apply(torch.from_numpy(y).to("cuda", _dt(prec)), adjoint=True).cpu().numpy()
    _check(g, midbf.apply(fac, f, mats), TOL[prec], "paper grid forward")
    _check(a, midbf.apply_adjoint(fac, y, mats), TOL[prec], "paper grid adjoint")
    fac, plan, mats = oracle_case("fio2d_n32_L3")
    # every stage, the stored middle factor included (its blocks are dense
    # sub-blocks with no skeleton: the narrow kernels add no identity part)
    for s_mode in (mb.S_ONTHEFLY, mb.S_STORED):
        dp = mb.DevicePlan(plan, prec, s_mode)
        for q in range(len(dp.stage_info())):
            for adj in (0, 1):
                dp.set_choice(1, q, adj, mb.CHOICE_NARROW)
        f = synth.complex_gaussian(fac.nw, 1, 52)[:, 0]
        g = dp.apply(torch.from_numpy(f).to("cuda", _dt(prec))).cpu().numpy()
        a = dp.apply(torch.from_numpy(f).to("cuda", _dt(prec)), adjoint=True).cpu().numpy()
        _check(g, midbf.apply(fac, f, mats), TOL[prec], f"forced narrow forward, S mode {s_mode}")
        _check(a, midbf.apply_adjoint(fac, f, mats), TOL[prec], f"forced narrow adjoint, S mode {s_mode}")


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,s_mode", [(mb.FP64, mb.S_STORED), (mb.FP32, mb.S_ONTHEFLY), (mb.FP32, mb.S_STORED)])
def test_cluster_row_kernel_matches_oracle(case, prec, s_mode):
    """The one-RHS row pattern on thread-block clusters (the CTAs of a cluster
    split an item's columns; CTA 0 adds the partial rows through distributed
    shared memory in rank order): forced on every stage and direction it runs
    (V forward, U adjoint, the stored middle factor forward), against the
    oracle's apply of the same factors; the result is the same bit for bit on
    a second call.  With 3 RHS the choice falls back to the SIMT tiles."""
    fac, plan, mats = oracle_case(case)
    dp = mb.DevicePlan(plan, prec, s_mode)
    for q in range(len(dp.stage_info())):
        for adj in (0, 1):
            dp.set_choice(1, q, adj, mb.CHOICE_CLUSTER)
            dp.set_choice(3, q, adj, mb.CHOICE_CLUSTER)
    f = synth.complex_gaussian(fac.nw, 3, 60)
    y = synth.complex_gaussian(fac.nx, 3, 61)
    F = torch.from_numpy(f.T.copy()).to("cuda", _dt(prec))
    Y = torch.from_numpy(y.T.copy()).to("cuda", _dt(prec))
    g1, a1 = dp.apply(F[0]), dp.apply(Y[0], adjoint=True)
    g2, a2 = dp.apply(F[0]), dp.apply(Y[0], adjoint=True)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2) and torch.equal(a1, a2)
    _check(g1.cpu().numpy(), midbf.apply(fac, f[:, 0], mats), TOL[prec], f"{case} cluster forward")
    _check(a1.cpu().numpy(), midbf.apply_adjoint(fac, y[:, 0], mats), TOL[prec], f"{case} cluster adjoint")
    g3, a3 = dp.apply(F).cpu().numpy().T, dp.apply(Y, adjoint=True).cpu().numpy().T
    for r in range(3):
        _check(g3[:, r], midbf.apply(fac, f[:, r], mats), TOL[prec], f"{case} 3 RHS forward")
        _check(a3[:, r], midbf.apply_adjoint(fac, y[:, r], mats), TOL[prec], f"{case} 3 RHS adjoint")
    assert dp.status() == mb.OK


@pytest.mark.parametrize("case", ["fio2d_n64_L3", "jump_n32_L2", "fio3d_n8_L2", "lowrank_n32_L3", "dot_n16_L2"])
@pytest.mark.parametrize("s_mode", [mb.S_ONTHEFLY, mb.S_STORED])
def test_gemm_forms_match_oracle(case, s_mode):
    """The FP32 register-tiled complex GEMM forms (4 x 4 micro-tiles per
    thread, RHS in tiles of 64): the middle factor made on the fly (k_s_gemm:
    64 x 32 tiles of S made once in shared memory), and the row and column
    patterns of the V/U stages and of the stored middle factor (k_r_gemm,
    k_c_gemm: T copied by 16-byte cp.async into shared memory).  Forced on every stage for 1,
    5 and 70 RHS (a ragged second RHS tile), and under the default rules at
    40 RHS (the ID stages' GEMM forms), forward and adjoint, against the
    oracle's apply of the same factors; a batched call with a 40-RHS instance
    equals the single apply bit for bit."""
    fac, plan, mats = oracle_case(case)
    dp = mb.DevicePlan(plan, mb.FP32, s_mode)
    for nrhs in (1, 5, 70):
        for q in range(len(dp.stage_info())):
            for adj in (0, 1):
                dp.set_choice(nrhs, q, adj, mb.CHOICE_GEMM)
    for nrhs in (1, 5, 40, 70):
        f = synth.complex_gaussian(fac.nw, nrhs, 70 + nrhs)
        h = synth.complex_gaussian(fac.nx, nrhs, 71 + nrhs)
        g = dp.apply(torch.from_numpy(f.T.copy()).to("cuda", torch.complex64)).cpu().numpy().T
        a = dp.apply(torch.from_numpy(h.T.copy()).to("cuda", torch.complex64), adjoint=True).cpu().numpy().T
        for r in range(0, nrhs, max(1, nrhs // 4)):
            _check(g[:, r], midbf.apply(fac, f[:, r], mats), TOL[mb.FP32], f"{case} gemm forward {nrhs}/{r}")
            _check(a[:, r], midbf.apply_adjoint(fac, h[:, r], mats), TOL[mb.FP32], f"{case} gemm adjoint {nrhs}/{r}")
    x = torch.from_numpy(synth.complex_gaussian(fac.nw, 40, 90).T.copy()).to("cuda", torch.complex64)
    y = torch.from_numpy(synth.complex_gaussian(fac.nx, 3, 91).T.copy()).to("cuda", torch.complex64)
    outs = mb.apply_batched([dp, dp], [x, y], [0, 1])
    assert torch.equal(outs[0], dp.apply(x)) and torch.equal(outs[1], dp.apply(y, adjoint=True))
    assert dp.status() == mb.OK
