"""Examples 2 and 3 of Sec. 4 through the library on the host (no GPU).

The library's DISTANCE phase against the oracle's, its constructions over the
non-uniform octrees of the random cube and the sphere mesh (applied by the
oracle in FP64) against direct sums of eq. (1), and its phase recovery
against the zeros Table 3 prints.
"""
import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

mb = pytest.importorskip("paper_1908_09376_gb300")


def test_library_distance_phase_matches_oracle():
    w = synth.WORKLOADS["helmholtz_l5"]
    X, W, _, _ = w.points()
    ph = mb.Phase.closed_form(synth.PHASE_DISTANCE, X, W)
    rng = np.random.default_rng(2)
    ix, iw = rng.integers(0, w.nx, 4000), rng.integers(0, w.nw, 4000)
    ref = OPhase(synth.PHASE_DISTANCE, X, W)(ix, iw)
    assert np.max(np.abs(ph.eval(ix, iw) - ref)) <= 1e-15 * np.max(ref)


def _library_plan(w, t=None):
    X, W, bx, bw = w.points()
    ph = mb.Phase.closed_form(w.phase, X, W)
    kw = {} if t is None else {"t": t}
    return mb.Plan.build(ph, tol=w.tol, n0=w.n0, boxX=bx, boxW=bw, **kw), OPhase(w.phase, X, W)


def test_library_construction_helmholtz_sphere():
    """Example 3 at level 4 (1313 x 1249 points): the library's plan, applied
    by the oracle in FP64, against the full direct sum (forward and adjoint)."""
    w = synth.Workload("helmholtz_l4", 3, 4, synth.PHASE_DISTANCE, 1e-6, 64, 1, 0, x_kind="sphere",
                       w_kind="sphere", t=5.0)
    plan, P = _library_plan(w, w.t)
    fac = planio.read(plan.export())
    f = w.rhs(1)[:, 0]
    g = midbf.apply(fac, f)
    assert direct.rel_l2(g, direct.direct_sum(P, f)) < 2e-5
    y = synth.complex_gaussian(w.nx, 1, 9)[:, 0]
    assert direct.rel_l2(midbf.apply_adjoint(fac, y), direct.direct_adjoint(P, y)) < 2e-5


def test_library_construction_nuft3d_random():
    """Example 2 at n = 16 (4096 random points on each side): the library's
    plan, applied by the oracle in FP64, against the full direct sum."""
    w = synth.WORKLOADS["nuft3d_n16"]
    plan, P = _library_plan(w)
    fac = planio.read(plan.export())
    f = w.rhs(1)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(P, f)) < 1e-5
    # the printed example is barely oscillatory (|Phi| < 3): ranks stay small
    assert plan.stats()["max_rank"] < 128


def test_library_recovery_tau_study_of_table3():
    """midbf_phase_recover with tau held fixed (no escalation) finds none of
    the discontinuities Table 3 rules out: none at tau = 1/4 for n = 8, 16, 32,
    none at any printed tau for n = 32."""
    for n in (8, 16, 32):
        N = n ** 3
        X = synth.uniform_random_points(N, 3, 0)
        W = synth.uniform_random_points(N, 3, 1)
        P = OPhase(synth.PHASE_DOT, X, W)
        rows = lambda i: np.exp(2j * np.pi * P(i[:, None], np.arange(N)[None, :]))
        cols = lambda i: np.exp(2j * np.pi * P(np.arange(N)[:, None], i[None, :]))
        for tau in ((1 / 4, 1 / 6, 1 / 8, 1 / 10) if n == 32 else (1 / 4,)):
            ph = mb.Phase.recover(X, W, rows, cols, r=4, q=2, tau=tau, max_disc=1 << 30, seed=0)
            assert ph.info["disc_rows"] == 0 and ph.info["disc_cols"] == 0, (n, tau)
            assert ph.info["tau"] == tau and ph.info["mismatches"] == 0


def test_recovered_phase_pipeline_of_table4():
    """Example 2 end to end through the library: recover Psi (Algorithm 7),
    build the MIDBF from it, apply (the oracle applies the exported plan) and
    compare with the direct sum of the true phase.  Table 4 at n = 16: r = 3
    fails (eps^b 0.26), r = 4 and 5 reach eps^b 1.1e-6."""
    n = 16
    N = n ** 3
    X = synth.uniform_random_points(N, 3, 0)
    W = synth.uniform_random_points(N, 3, 1)
    P = OPhase(synth.PHASE_DOT, X, W)
    rows = lambda i: np.exp(2j * np.pi * P(i[:, None], np.arange(N)[None, :]))
    cols = lambda i: np.exp(2j * np.pi * P(np.arange(N)[:, None], i[None, :]))
    f = synth.complex_gaussian(N, 1, 0)[:, 0]
    S = synth.sample_rows(N, 200, 3)
    ref = direct.direct_sum(P, f, rows=S)
    box = (np.zeros(3), 1.0)
    for r, bound in ((3, None), (4, 1.1e-5), (5, 1.1e-5)):
        ph = mb.Phase.recover(X, W, rows, cols, r=r, q=2, tau=0.25, seed=0)
        plan = mb.Plan.build(ph, tol=1e-6, n0=512, boxX=box, boxW=box)
        eb = direct.rel_l2(midbf.apply(planio.read(plan.export()), f)[S], ref)
        if bound is None:
            assert eb > 0.1, (r, eb)
        else:
            assert eb < bound, (r, eb)


def test_helmholtz_accuracy_of_table5():
    """Example 3 with the closed-form phase at the paper's tolerance 1e-9:
    the MIDBF's eps^b on the level-5 mesh (10,242 nodes) is within 10x of
    Table 5's 2.79e-8 for n = 10240."""
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden", "table5_helmholtz.txt")
    eb_paper = {int(l.split()[0]): float(l.split()[1]) for l in open(gold) if l.strip() and not l.startswith("#")}
    w = synth.Workload("helmholtz_l5_tol9", 3, 5, synth.PHASE_DISTANCE, 1e-9, 64, 1, 0, x_kind="sphere",
                       w_kind="sphere", t=5.0)
    plan, P = _library_plan(w, w.t)
    f = w.rhs(1)[:, 0]
    S = synth.sample_rows(w.nx, 200, 3)
    eb = direct.rel_l2(midbf.apply(planio.read(plan.export()), f)[S], direct.direct_sum(P, f, rows=S))
    assert eb < 10 * eb_paper[10240], eb
