"""GPU parity on Examples 2 and 3 of Sec. 4 (needs a GB300).

Example 3 (Helmholtz phase h |x - xi| on the two halves of a sphere mesh)
runs the middle factor in the distance form: rows and columns carry their
coordinates relative to the block's first column point, and each entry
takes sqrt(sum_q (C_iq - W_jq)^2).  Example 2 (x.xi over random points in the
unit cube) runs the general phase shape over non-uniform octrees.  Plans
built by the oracle (inputs free of product code) and plans built by the
library (checked against the oracle's apply of the exported file) are both
applied forward and adjoint, SIMT and tensor-core, single and batched.

Tolerances (relative L2, and max abs error over max |ref| within 10x):
  FP64 1e-12 as for the other workloads;
  FP32 3e-5: besides the FP32 storage of T and data (~1e-6), the distance
    form rounds coordinates of magnitude up to 2h to FP32, an absolute phase
    error up to ~2h 2^-23 (3e-6 cycles at h = 7.2; the same arithmetic in
    numpy float32 on 2e5 random pairs of the level-5 mesh gives at most
    2.0e-6 cycles and an rms entry error of 2.9e-6);
  BF16 + refinement 5e-5: the 2e-5 of the refined operands plus that phase
    error.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

torch = pytest.importorskip("torch")
mb = pytest.importorskip("paper_1908_09376_gb300")

pytestmark = pytest.mark.gpu

TOL = {mb.FP64: 1e-12, mb.FP32: 3e-5, mb.BF16 | mb.REFINE: 5e-5}
_C = {}


def _dt(prec):
    return torch.complex128 if prec == mb.FP64 else torch.complex64


def _check(got, ref, tol, what):
    e = direct.rel_l2(got, ref)
    m = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < tol and m < 10 * tol, f"{what}: rel-L2 {e:.3e}, max {m:.3e}"


def _case(name):
    """(factorization, library plan, sparse factor matrices) of one case."""
    if name in _C:
        return _C[name]
    if name == "sphere_l4_oracle":
        X0, W0 = synth.hemispheres(synth.icosphere(4)[0])
        h = math.sqrt(len(X0)) / 10
        box = (np.full(3, -h), 2 * h)
        fac = midbf.build(OPhase(synth.PHASE_DISTANCE, h * X0, h * W0), n0=32, tol=1e-7, t=5.0,
                          boxX=box, boxW=box)
        plan = mb.Plan.load(planio.write(fac))
    elif name == "nuft3d_n8_oracle":
        X = synth.uniform_random_points(512, 3, 0)
        W = synth.uniform_random_points(512, 3, 1)
        box = (np.zeros(3), 1.0)
        fac = midbf.build(OPhase(synth.PHASE_DOT, X, W), n0=8, tol=1e-8, t=2.0, boxX=box, boxW=box)
        plan = mb.Plan.load(planio.write(fac))
    else:
        w = synth.WORKLOADS[name]
        X, W, bx, bw = w.points()
        plan = mb.Plan.build(mb.Phase.closed_form(w.phase, X, W), tol=w.tol, n0=w.n0, boxX=bx, boxW=bw, t=w.t)
        fac = planio.read(plan.export())
    _C[name] = (fac, plan, midbf.factor_matrices(fac))
    return _C[name]


def _run(dp, fac, mats, prec, nrhs, seed, what):
    dev = torch.device("cuda:0")
    f = synth.complex_gaussian(fac.nw, nrhs, seed)
    y = synth.complex_gaussian(fac.nx, nrhs, seed + 1)
    g = dp.apply(torch.from_numpy(f.T.copy()).to(dev, _dt(prec))).cpu().numpy().T
    a = dp.apply(torch.from_numpy(y.T.copy()).to(dev, _dt(prec)), adjoint=True).cpu().numpy().T
    g_ref = np.stack([midbf.apply(fac, f[:, r], mats) for r in range(nrhs)], 1)
    a_ref = np.stack([midbf.apply_adjoint(fac, y[:, r], mats) for r in range(nrhs)], 1)
    _check(g, g_ref, TOL[prec], f"{what} forward nrhs={nrhs}")
    _check(a, a_ref, TOL[prec], f"{what} adjoint nrhs={nrhs}")
    assert dp.status() == mb.OK


@pytest.mark.parametrize("case", ["sphere_l4_oracle", "helmholtz_l5", "nuft3d_n8_oracle", "nuft3d_n16"])
@pytest.mark.parametrize("prec", [mb.FP64, mb.FP32])
@pytest.mark.parametrize("s_mode", [mb.S_ONTHEFLY, mb.S_STORED])
def test_examples_simt(case, prec, s_mode):
    fac, plan, mats = _case(case)
    dp = mb.DevicePlan(plan, prec, s_mode)
    for nrhs in ((1, 2, 4, 9, 20) if s_mode == mb.S_ONTHEFLY else (1, 3)):
        _run(dp, fac, mats, prec, nrhs, 60 + nrhs, f"{case} {s_mode}")


@pytest.mark.parametrize("case", ["sphere_l4_oracle", "helmholtz_l5", "nuft3d_n16"])
def test_examples_tensor_cores(case):
    fac, plan, mats = _case(case)
    dp = mb.DevicePlan(plan, mb.BF16 | mb.REFINE)
    for nrhs in (16, 40):
        _run(dp, fac, mats, mb.BF16 | mb.REFINE, nrhs, 80 + nrhs, f"{case} tensor cores")


def test_helmholtz_library_plan_against_direct_sum():
    """End to end: the library's plan of Example 3 (level 5, t = 5) applied on
    the GPU in FP32 against FP64 direct sums of eq. (1) on sampled rows."""
    w = synth.WORKLOADS["helmholtz_l5"]
    fac, plan, _ = _case("helmholtz_l5")
    dp = mb.DevicePlan(plan, mb.FP32)
    f = w.rhs(1)[:, 0]
    g = dp.apply(torch.from_numpy(f).to("cuda", torch.complex64)).cpu().numpy()
    X, W, _, _ = w.points()
    rows = synth.sample_rows(w.nx, 256, 3)
    ref = direct.direct_sum(OPhase(w.phase, X, W), f, rows=rows)
    assert direct.rel_l2(g[rows], ref) < 2e-5


@pytest.mark.parametrize("prec", [mb.FP32, mb.FP64])
def test_examples_batched(prec):
    """Sphere, random-cube and grid instances in one midbf_apply_batched call:
    each output equals the single-instance apply bit for bit."""
    names = ["sphere_l4_oracle", "nuft3d_n8_oracle", "helmholtz_l5"]
    cases = [_case(n) for n in names]
    dps = [mb.DevicePlan(c[1], prec) for c in cases]
    adjoints = [0, 1, 0, 1, 1, 0]
    idx = [0, 0, 1, 2, 2, 1]
    nrhs = [1, 3, 2, 5, 1, 8]
    xs = []
    for k, (i, a, r) in enumerate(zip(idx, adjoints, nrhs)):
        fac = cases[i][0]
        n_in = fac.nx if a else fac.nw
        xs.append(torch.from_numpy(synth.complex_gaussian(n_in, r, 140 + k).T.copy()).to("cuda", _dt(prec)))
    outs = mb.apply_batched([dps[i] for i in idx], xs, adjoints)
    for k, (i, a, r) in enumerate(zip(idx, adjoints, nrhs)):
        assert torch.equal(outs[k], dps[i].apply(xs[k], adjoint=bool(a))), k
        fac, _, mats = cases[i]
        x = xs[k].cpu().numpy().astype(np.complex128)
        ref = np.stack([(midbf.apply_adjoint if a else midbf.apply)(fac, x[q], mats) for q in range(r)])
        _check(outs[k].cpu().numpy(), ref, TOL[prec], f"batched {k}")


@pytest.mark.parametrize("name", ["helmholtz_l4", "nuft3d_n16"])
def test_device_build_of_examples(name):
    """The IDs' kernel samples and pivoted QRs on the GPU (FP64, the distance
    phase evaluated on the device): the plan, applied by the oracle, against
    the direct sum of eq. (1)."""
    if name == "helmholtz_l4":
        w = synth.Workload(name, 3, 4, synth.PHASE_DISTANCE, 1e-6, 64, 1, 0, x_kind="sphere", w_kind="sphere", t=5.0)
    else:
        w = synth.WORKLOADS[name]
    X, W, bx, bw = w.points()
    plan = mb.Plan.build(mb.Phase.closed_form(w.phase, X, W), tol=w.tol, n0=w.n0, boxX=bx, boxW=bw, t=w.t,
                         device_ids=1)
    fac = planio.read(plan.export())
    f = w.rhs(1)[:, 0]
    rows = synth.sample_rows(w.nx, 256, 3)
    ref = direct.direct_sum(OPhase(w.phase, X, W), f, rows=rows)
    assert direct.rel_l2(midbf.apply(fac, f)[rows], ref) < 2e-5
