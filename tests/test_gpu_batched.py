"""Batched apply of uneven instances (needs a GB300).

Instances of different sizes, tree depths (odd and even L), directions and
right-hand-side counts go through midbf_apply_batched in one call; each
output must equal the single-instance apply of the same plan (the same kernel
bodies run) and the oracle's apply of the same factors.
"""
import numpy as np
import pytest

import synth
from oracle import midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu


def _fac(n, n0, family=synth.PHASE_FIO2D):
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    return midbf.build(OPhase(family, X, W), n0=n0, tol=1e-6, t=2.0,
                       boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))


@pytest.mark.parametrize("prec", [mb.FP32, mb.FP64])
def test_batched_matches_single_and_oracle(prec):
    facs = [_fac(16, 16), _fac(32, 16), _fac(32, 64), _fac(64, 64), _fac(16, 4, synth.PHASE_DOT)]
    plans = [mb.Plan.load(planio.write(f)) for f in facs]
    dps = [mb.DevicePlan(p, prec) for p in plans]
    dt = torch.complex64 if prec == mb.FP32 else torch.complex128
    adjoints = [0, 1, 0, 1, 0, 1, 1, 0]
    idx = [0, 1, 2, 3, 4, 3, 0, 2]
    nrhs = [1, 3, 20, 1, 2, 5, 1, 1]
    xs = []
    for k, (i, a, r) in enumerate(zip(idx, adjoints, nrhs)):
        n_in = facs[i].nx if a else facs[i].nw
        xs.append(torch.from_numpy(synth.complex_gaussian(n_in, r, 40 + k).T.copy()).to("cuda", dt))
    outs = mb.apply_batched([dps[i] for i in idx], xs, adjoints)
    tol = 1e-12 if prec == mb.FP64 else 2e-5
    for k, (i, a, r) in enumerate(zip(idx, adjoints, nrhs)):
        single = dps[i].apply(xs[k], adjoint=bool(a))
        assert torch.equal(outs[k], single), k
        x = xs[k].cpu().numpy().astype(np.complex128)
        mats = midbf.factor_matrices(facs[i])
        ref = np.stack([(midbf.apply_adjoint if a else midbf.apply)(facs[i], x[q], mats) for q in range(r)])
        got = outs[k].cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < tol, (k, err)


def test_batched_argument_errors():
    fac = _fac(16, 16)
    plan = mb.Plan.load(planio.write(fac))
    d32 = mb.DevicePlan(plan, mb.FP32)
    d64 = mb.DevicePlan(plan, mb.FP64)
    x32 = torch.zeros((1, fac.nw), dtype=torch.complex64, device="cuda")
    x64 = torch.zeros((1, fac.nw), dtype=torch.complex128, device="cuda")
    with pytest.raises(mb.MidbfError) as e:
        mb.apply_batched([d32, d64], [x32, x64], [0, 0])
    assert e.value.code == mb.EINVAL


def test_batched_launch_count():
    """midbf_batched_launches: one launch group per level index and kernel
    variant, so the count lies between the deepest plan's stage count and the
    sum of all stage counts, and stays the same when instances of several
    RHS repeat.  A one-RHS instance's stages that run on the narrow-ID or
    cluster kernels get launches of their own: a repeated one-RHS instance
    adds at most its own stage count."""
    facs = [_fac(16, 16), _fac(32, 16), _fac(32, 64)]
    dps = [mb.DevicePlan(mb.Plan.load(planio.write(f)), mb.FP32) for f in facs]
    nst = [len(d.stage_info()) for d in dps]
    n1 = mb.batched_launches(dps, [0, 1, 0], [2, 3, 20])
    assert max(nst) <= n1 <= sum(nst)
    n2 = mb.batched_launches(dps + dps, [0, 1, 0] * 2, [2, 3, 20] * 2)
    assert n2 == n1
    m1 = mb.batched_launches(dps, [0, 1, 0], [1, 3, 20])
    assert max(nst) <= m1 <= sum(nst)
    m2 = mb.batched_launches(dps + dps[:1], [0, 1, 0, 0], [1, 3, 20, 1])
    assert m1 <= m2 <= m1 + nst[0]
