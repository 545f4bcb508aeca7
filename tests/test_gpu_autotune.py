"""Kernel choices and the autotuner (needs a GB300).

Every stage of an apply can run several kernel variants (SIMT RHS tiles, the
one-RHS column kernel, each of them one CTA per item or persistent, the
narrow-ID kernels for one RHS and low ranks, the one-RHS row pattern on
thread-block clusters, the FP32 middle factor as a register-tiled GEMM, and
the tensor-core kernels).  Forcing each variant of
each stage in turn must reproduce the oracle's FP64 apply of the same
factors (FP32: 2e-5; tensor cores with refinement: 2e-5; tolerances as in
test_gpu_apply / test_gpu_tensor), and the autotuner must record, for every
stage and direction, one of the variants that apply there.
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


def _case():
    if "c" not in _C:
        n = 64
        X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=64, tol=1e-6, t=2.0,
                          boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
        _C["c"] = (fac, mb.Plan.load(planio.write(fac)), midbf.factor_matrices(fac))
    return _C["c"]


def _ref(fac, mats, f, adjoint):
    fn = midbf.apply_adjoint if adjoint else midbf.apply
    return np.stack([fn(fac, f[:, r], mats) for r in range(f.shape[1])], 1)


@pytest.mark.parametrize("mode,nrhs,choices", [
    (mb.FP32, 1, [1, mb.CHOICE_COLUMN1, 1 | mb.CHOICE_PERSIST, mb.CHOICE_COLUMN1 | mb.CHOICE_PERSIST]),
    (mb.FP32, 1, [mb.CHOICE_NARROW, mb.CHOICE_CLUSTER]),
    (mb.FP32, 20, [1, 2, 4, 8, 16, 16 | mb.CHOICE_PERSIST, mb.CHOICE_GEMM]),
    (mb.BF16 | mb.REFINE, 20, [4, 16 | mb.CHOICE_PERSIST, mb.CHOICE_TENSOR]),
])
def test_every_forced_variant_matches_oracle(mode, nrhs, choices):
    fac, plan, mats = _case()
    dp = mb.DevicePlan(plan, mode)
    ns = len(dp.stage_info())
    f = synth.complex_gaussian(fac.nw, nrhs, 80)
    h = synth.complex_gaussian(fac.nx, nrhs, 81)
    g_ref, a_ref = _ref(fac, mats, f, False), _ref(fac, mats, h, True)
    F = torch.from_numpy(f.T.copy()).to("cuda", torch.complex64)
    H = torch.from_numpy(h.T.copy()).to("cuda", torch.complex64)
    for stage in range(ns):
        for ch in choices:
            dp.set_choice(nrhs, stage, 0, ch)
            dp.set_choice(nrhs, stage, 1, ch)
            g = dp.apply(F).cpu().numpy().T
            a = dp.apply(H, adjoint=True).cpu().numpy().T
            eg, ea = direct.rel_l2(g, g_ref), direct.rel_l2(a, a_ref)
            assert eg < 2e-5 and ea < 2e-5, (stage, ch, eg, ea)
        dp.set_choice(nrhs, stage, 0, mb.CHOICE_DEFAULT)
        dp.set_choice(nrhs, stage, 1, mb.CHOICE_DEFAULT)
    assert dp.status() == mb.OK


@pytest.mark.parametrize("mode,nrhs", [(mb.FP32, 1), (mb.FP32, 12), (mb.FP64, 3), (mb.BF16 | mb.REFINE, 32)])
def test_autotune_records_valid_choices_and_keeps_results(mode, nrhs):
    fac, plan, mats = _case()
    dp = mb.DevicePlan(plan, mode, mb.S_STORED if mode == mb.FP64 else mb.S_ONTHEFLY)
    dt = dp.dtype()
    f = synth.complex_gaussian(fac.nw, nrhs, 82)
    F = torch.from_numpy(f.T.copy()).to("cuda", dt)
    before = dp.apply(F)
    dp.autotune(nrhs)
    info = dp.stage_info()
    simt = {1, 2, 4, 8, 16, mb.CHOICE_COLUMN1}
    for stage in range(len(info)):
        for adj in (0, 1):
            ch = dp.choice(nrhs, stage, adj)
            if ch == mb.CHOICE_TENSOR:
                assert mode & mb.BF16
                continue
            if ch in (mb.CHOICE_NARROW, mb.CHOICE_CLUSTER):   # narrow-ID or cluster kernels: one RHS
                assert nrhs == 1
                continue
            if ch == mb.CHOICE_GEMM:   # the register-tiled FP32 GEMM forms (FP32 data: FP32 and BF16 plans)
                assert mode != mb.FP64 and nrhs >= 8
                continue
            base = ch & ~mb.CHOICE_PERSIST
            assert base in simt, (stage, adj, ch)
            if base == mb.CHOICE_COLUMN1:
                assert nrhs == 1
    after = dp.apply(F)
    tol = 1e-12 if mode == mb.FP64 else 2e-5
    rel = (torch.linalg.vector_norm(after - before) / torch.linalg.vector_norm(before)).item()
    assert rel < tol
    g_ref = _ref(fac, mats, f, False)
    assert direct.rel_l2(after.cpu().numpy().T, g_ref) < tol
    assert dp.status() == mb.OK


def test_batched_apply_uses_tuned_tiles():
    fac, plan, mats = _case()
    dp = mb.DevicePlan(plan, mb.FP32)
    nrhs = 6
    for stage in range(len(dp.stage_info())):
        dp.set_choice(nrhs, stage, 0, 2)
        dp.set_choice(nrhs, stage, 1, 4)
    f = synth.complex_gaussian(fac.nw, nrhs, 83)
    h = synth.complex_gaussian(fac.nx, nrhs, 84)
    xs = [torch.from_numpy(f.T.copy()).to("cuda", torch.complex64),
          torch.from_numpy(h.T.copy()).to("cuda", torch.complex64)]
    outs = mb.apply_batched([dp, dp], xs, [0, 1])
    g_ref, a_ref = _ref(fac, mats, f, False), _ref(fac, mats, h, True)
    assert direct.rel_l2(outs[0].cpu().numpy().T, g_ref) < 2e-5
    assert direct.rel_l2(outs[1].cpu().numpy().T, a_ref) < 2e-5
