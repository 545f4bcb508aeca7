"""Construction with the decompositions on the GPU (midbf_params.device_ids = 1).

The sampling and regrowth rule stay on the host; kernel samples, pivoted
QRs and T = R11^{-1} R12 run in FP64 on the device.  Rounding differs from
the host QR, so factors are compared by their accuracy against the direct
sum (same bounds as the host build) and by their ranks.
"""
import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu


def _grid(n):
    return (synth.uniform_grid(n, 2), synth.frequency_grid(n, 2), (np.zeros(2), 1.0),
            (np.full(2, -n / 2), float(n)))


@pytest.mark.parametrize("n,family,n0", [(64, synth.PHASE_FIO2D, 64), (32, synth.PHASE_FIO2D_JUMP, 16),
                                         (32, synth.PHASE_ZERO, 16)])
def test_device_build_accuracy(n, family, n0):
    X, W, bx, bw = _grid(n)
    ph = mb.Phase.closed_form(family, X, W)
    dev = mb.Plan.build(ph, tol=1e-6, n0=n0, boxX=bx, boxW=bw, device_ids=1)
    host = mb.Plan.build(ph, tol=1e-6, n0=n0, boxX=bx, boxW=bw)
    sd, sh = dev.stats(), host.stats()
    assert sd["nstages"] == sh["nstages"] and sd["nsubs"] == sh["nsubs"]
    assert abs(sd["mean_rank"] - sh["mean_rank"]) <= 0.05 * sh["mean_rank"] + 1
    fac = planio.read(dev.export())
    f = synth.complex_gaussian(n * n, 1, 0)[:, 0]
    ref = direct.direct_sum(OPhase(family, X, W), f)
    bound = 1e-12 if family == synth.PHASE_ZERO else 2e-5
    assert direct.rel_l2(midbf.apply(fac, f), ref) < bound


def test_device_build_3d_and_lowrank():
    X = synth.uniform_random_points(512, 3, 0)
    W = synth.frequency_grid(8, 3)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO3D, X, W), tol=1e-7, n0=8,
                         boxX=(np.zeros(3), 1.0), boxW=(np.full(3, -4.0), 8.0), device_ids=1)
    fac = planio.read(plan.export())
    f = synth.complex_gaussian(512, 1, 0)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(OPhase(synth.PHASE_FIO3D, X, W), f)) < 1e-5
    n = 32
    X2, W2, bx, bw = _grid(n)
    rng = np.random.default_rng(5)
    U = np.concatenate([X2, 0.01 * rng.standard_normal((1024, 2))], axis=1)
    V = np.concatenate([W2, rng.standard_normal((1024, 2))], axis=1)
    plan = mb.Plan.build(mb.Phase.lowrank(X2, W2, U, V), tol=1e-6, n0=16, boxX=bx, boxW=bw, device_ids=1)
    fac = planio.read(plan.export())
    f = synth.complex_gaussian(1024, 1, 3)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(fac.phase, f)) < 2e-5


def test_device_build_fp32_storage():
    """device_ids with store_fp32: the replies are converted to FP32 one by one;
    the plan has the device build's structure and its coefficients rounded to
    FP32."""
    X, W, bx, bw = _grid(64)
    ph = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    p64 = mb.Plan.build(ph, tol=1e-6, n0=64, boxX=bx, boxW=bw, device_ids=1)
    p32 = mb.Plan.build(ph, tol=1e-6, n0=64, boxX=bx, boxW=bw, device_ids=1, store_fp32=1)
    assert p32.stats() == p64.stats()
    f64, f32 = planio.read(p64.export()), planio.read(p32.export())
    for s64, s32 in zip(f64.stages, f32.stages):
        for b64, b32 in zip(s64.blocks, s32.blocks):
            for u64, u32 in zip(b64.subs, b32.subs):
                assert np.array_equal(u64.skel, u32.skel)
                assert np.array_equal(u32.T, u64.T.astype(np.complex64).astype(np.complex128))


def test_consuming_upload():
    """MIDBF_DPLAN_CONSUME: the device plan equals the one from an ordinary
    upload bit for bit; the consumed host plan keeps its statistics but
    refuses export and further uploads."""
    X, W, bx, bw = _grid(64)
    ph = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    keep = mb.Plan.build(ph, tol=1e-6, n0=64, boxX=bx, boxW=bw, store_fp32=1)
    used = mb.Plan.build(ph, tol=1e-6, n0=64, boxX=bx, boxW=bw, store_fp32=1)
    st = used.stats()
    d1 = mb.DevicePlan(keep, mb.FP32)
    d2 = mb.DevicePlan(used, mb.FP32, consume=True)
    assert used.stats() == st
    F = torch.from_numpy(synth.complex_gaussian(64 * 64, 3, 7).T.copy()).to("cuda", torch.complex64)
    assert torch.equal(d1.apply(F), d2.apply(F))
    assert torch.equal(d1.apply(F, adjoint=True), d2.apply(F, adjoint=True))
    with pytest.raises(mb.MidbfError) as e:
        used.export()
    assert e.value.code == mb.EINVAL
    with pytest.raises(mb.MidbfError) as e:
        mb.DevicePlan(used, mb.FP32)
    assert e.value.code == mb.EINVAL
