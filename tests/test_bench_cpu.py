"""bench.py's accuracy report (no GPU): the sampled direct-sum error is at
rounding level for exact outputs and reports a planted perturbation at its
size, in both directions; the workload defaults follow the configurations."""
import sys

import numpy as np
import pytest

import synth
from oracle import direct
from oracle.phase import Phase as OPhase

mb = pytest.importorskip("paper_1908_09376_gb300")


def _bench():
    sys.argv = ["bench.py"]
    import bench
    return bench


def test_sampled_direct_error_exact_and_perturbed():
    bench = _bench()
    n = 16
    X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
    ph = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    oph = OPhase(synth.PHASE_FIO2D, X, W)
    F = synth.complex_gaussian(n * n, 3, 0)
    Hin = synth.complex_gaussian(n * n, 3, 1)
    G = np.stack([direct.direct_sum(oph, F[:, r]) for r in range(3)], 1)
    H = np.stack([direct.direct_adjoint(oph, Hin[:, r]) for r in range(3)], 1)
    rows = synth.sample_rows(n * n, 20, 3)
    cols = synth.sample_rows(n * n, 20, 4)
    ef, ea = bench.sampled_direct_error(ph, F.T, G.T, Hin.T, H.T, rows, cols)
    assert ef < 1e-13 and ea < 1e-13
    rng = np.random.default_rng(0)
    Gp = G * (1 + 1e-3 * rng.standard_normal(G.shape))
    Hp = H * (1 + 1e-3 * rng.standard_normal(H.shape))
    ef, ea = bench.sampled_direct_error(ph, F.T, Gp.T, Hin.T, Hp.T, rows, cols)
    assert 3e-4 < ef < 3e-3 and 3e-4 < ea < 3e-3
    assert bench.sampled_direct_error(ph, F.T, G.T, Hin.T, H.T, rows, cols[:0])[1] is None


def test_workload_defaults():
    bench = _bench()

    class A:
        workload, n, nrhs, mode, build, store, tune, graph = "fio2d", None, None, None, None, None, None, None
    w, nrhs, mode, build, store, tune, graph = bench.pick_workload(A)
    assert (w.n, nrhs, mode, build, store, tune, graph) == (256, 1, "fp32", "host", "fp64", False, True)
    A.nrhs = 64
    assert bench.pick_workload(A)[6] is False      # the graph default is for the one-RHS step only
    A.nrhs = None
    A.workload = "fio3d_n32"
    w, nrhs, mode, build, store, tune, graph = bench.pick_workload(A)
    assert (w.d, w.N, nrhs, mode, graph) == (3, 32768, 256, "bf16r", False)
    A.workload = "fio2d_jump"
    w, nrhs, mode, build, store, tune, graph = bench.pick_workload(A)
    assert (w.N, nrhs, mode, store, tune, graph) == (1024 * 1024, 16, "fp32", "fp32", True, True)
    A.workload, A.n = "nuft3d", None
    w, nrhs, mode, build, store, tune, graph = bench.pick_workload(A)
    assert (w.d, w.nx, w.nw, nrhs, mode, w.x_kind, w.w_kind) == (3, 64 ** 3, 64 ** 3, 1, "fp32", "random", "random")
    assert graph                                  # every one-RHS step of one plan is replayed as a graph
    A.workload = "helmholtz"
    w, nrhs, mode, build, store, tune, graph = bench.pick_workload(A)
    assert (w.nx, w.nw, nrhs, mode, w.t, w.n0, graph) == (20609, 20353, 1, "fp32", 5.0, 128, True)
    A.workload = "nuft3d_recovered"
    w, nrhs, mode, *_ = bench.pick_workload(A)
    assert w.recovered and (w.nx, w.w_kind, nrhs, mode) == (64 ** 3, "random", 1, "fp32")
    A.workload = "fio2d_paper"
    w, nrhs, mode, *_ = bench.pick_workload(A)
    X, W, bx, bw = w.points()
    assert w.recovered and w.tol == 1e-9 and w.N == 1024 ** 2 and W.max() < 1.0 and W.min() >= 0.0


def test_sampled_direct_error_rectangular():
    """|X| != |Omega| (the sphere halves): rows index X, columns index Omega."""
    bench = _bench()
    X0, W0 = synth.hemispheres(synth.icosphere(2)[0])
    ph = mb.Phase.closed_form(synth.PHASE_DISTANCE, 2.0 * X0, 2.0 * W0)
    oph = OPhase(synth.PHASE_DISTANCE, 2.0 * X0, 2.0 * W0)
    nx, nw = len(X0), len(W0)
    assert nx != nw
    F = synth.complex_gaussian(nw, 2, 0)
    G = np.stack([direct.direct_sum(oph, F[:, r]) for r in range(2)], 1)
    H = np.stack([direct.direct_adjoint(oph, G[:, r]) for r in range(2)], 1)
    ef, ea = bench.sampled_direct_error(ph, F.T, G.T, G.T, H.T, synth.sample_rows(nx, 30, 3),
                                        synth.sample_rows(nw, 30, 4))
    assert ef < 1e-13 and ea < 1e-13


def test_reference_arm_json_line():
    """--impl reference times the oracle on the selected workload (host only)
    and prints the contract's JSON line; the GPU-built workloads say why not."""
    import json
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "helmholtz", "--n", "3", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, env=env, timeout=300, check=True).stdout
    d = json.loads(out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "helmholtz_l3" and (d["config"]["nx"], d["config"]["nw"]) == (337, 305)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "batched"], capture_output=True, text=True, env=env, timeout=300, check=True).stdout
    d = json.loads(out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and "unavailable" in d
