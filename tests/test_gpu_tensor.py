"""Tensor-core apply (tcgen05, BF16 operands, FP32 accumulation).

With 16 or more right-hand sides, MIDBF_BF16 plans generate the middle factor
on the fly into shared memory as BF16 and multiply on the tensor cores, and
run the V / U stages as block GEMMs over dense BF16 tile images of their
interpolative decompositions; MIDBF_REFINE adds the refinement products of
the hi/lo split (reading A-R of the design notes).  Checked against the
oracle's FP64 apply of the same factors.  Tolerances: BF16 alone keeps 8
mantissa bits (relative 2^-9 per operand), so a product of five stages
carries a few 1e-3 relative error: bound 2e-2; with refinement each operand
keeps ~16 bits (hi + lo, residual 2^-18) and the dropped lo*lo product is of
the same order, so five stages give ~1e-5: bound 2e-5.  (Rounding every
factor and vector of the fio2d_n64 case this way in numpy, with exact
accumulation, gives 4.7e-3 and 8.4e-6.)
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


def _case(name):
    if name in _C:
        return _C[name]
    if name == "fio2d_n64":
        n = 64
        X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
        fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=64, tol=1e-6, t=2.0,
                          boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    elif name == "fio3d_n8":
        X = synth.uniform_random_points(512, 3, 0)
        W = synth.frequency_grid(8, 3)
        fac = midbf.build(OPhase(synth.PHASE_FIO3D, X, W), n0=8, tol=1e-7, t=2.0,
                          boxX=(np.zeros(3), 1.0), boxW=(np.full(3, -4.0), 8.0))
    else:
        n = 32
        X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
        rng = np.random.default_rng(5)
        U = np.concatenate([X, 0.01 * rng.standard_normal((1024, 2))], axis=1)
        V = np.concatenate([W, rng.standard_normal((1024, 2))], axis=1)
        fac = midbf.build(OPhase(synth.PHASE_LOWRANK, X, W, U, V), n0=16, tol=1e-6, t=2.0,
                          boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -16.0), 32.0))
    _C[name] = (fac, mb.Plan.load(planio.write(fac)), midbf.factor_matrices(fac))
    return _C[name]


def _errors(got, ref):
    """rel-L2 over all entries, and the largest entry error relative to the
    largest reference entry divided by 2: among the ~10^5 - 10^6 entries of a
    case the largest error sits about twice as far out in its distribution's
    tail as the largest reference entry does in its own (measured 1.7x for
    the refined products at 130 RHS), so both ratios are held to the same
    bound."""
    return direct.rel_l2(got, ref), float(np.abs(got - ref).max() / np.abs(ref).max()) / 2.0


# 16: the smallest tensor-core case; 130: a ragged RHS tile (Rpad 144); 256: the
# full TMEM accumulator of one pass (D_top in columns [0, 256), D_bot in
# [256, 512)); 300: more than one pass (a group of 256, then one of 44).
@pytest.mark.parametrize("case", ["fio2d_n64", "fio3d_n8", "lowrank_n32"])
@pytest.mark.parametrize("mode,tol", [(mb.BF16, 2e-2), (mb.BF16 | mb.REFINE, 2e-5)])
def test_tensor_core_middle_factor(case, mode, tol):
    fac, plan, mats = _case(case)
    dp = mb.DevicePlan(plan, mode)
    for nrhs in (16, 130, 256, 300):
        f = synth.complex_gaussian(fac.nw, nrhs, 60)
        h = synth.complex_gaussian(fac.nx, nrhs, 61)
        g = dp.apply(torch.from_numpy(f.T.copy()).to("cuda", torch.complex64)).cpu().numpy().T
        a = dp.apply(torch.from_numpy(h.T.copy()).to("cuda", torch.complex64), adjoint=True).cpu().numpy().T
        g_ref = midbf.apply(fac, f, mats)
        a_ref = midbf.apply_adjoint(fac, h, mats)
        (eg, mg), (ea, ma) = _errors(g, g_ref), _errors(a, a_ref)
        assert max(eg, mg, ea, ma) < tol, (case, mode, nrhs, eg, mg, ea, ma)
    assert dp.status() == mb.OK


def test_tensor_core_groups_agree_with_single_passes():
    """300 RHS run as a pass of 256 and a pass of 44; each column must agree
    with the same column applied in a pass of its own group size (the passes
    share no state but the RHS image buffer, which every pass rewrites).  The
    kernels are the same, so only the FP32 accumulation could differ."""
    fac, plan, _ = _case("fio2d_n64")
    dp = mb.DevicePlan(plan, mb.BF16 | mb.REFINE)
    f = torch.from_numpy(synth.complex_gaussian(fac.nw, 300, 63).T.copy()).to("cuda", torch.complex64)
    g = dp.apply(f)
    g_first = dp.apply(f[:256].contiguous())
    g_rest = dp.apply(f[256:].contiguous())
    torch.cuda.synchronize()
    scale = g.abs().max().item()
    assert (g[:256] - g_first).abs().max().item() <= 1e-6 * scale
    assert (g[256:] - g_rest).abs().max().item() <= 1e-6 * scale


def test_tensor_mode_below_threshold_uses_simt():
    """Fewer than 16 RHS: the BF16 plan runs the FP32 SIMT kernels (FP32 accuracy)."""
    fac, plan, mats = _case("lowrank_n32")
    dp = mb.DevicePlan(plan, mb.BF16)
    f = synth.complex_gaussian(fac.nw, 3, 62)
    g = dp.apply(torch.from_numpy(f.T.copy()).to("cuda", torch.complex64)).cpu().numpy().T
    g_ref = np.stack([midbf.apply(fac, f[:, r], mats) for r in range(3)], 1)
    assert direct.rel_l2(g, g_ref) < 2e-5
