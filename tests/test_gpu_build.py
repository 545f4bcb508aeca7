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
