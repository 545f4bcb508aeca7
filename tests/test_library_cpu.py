"""Host-side checks of the library (no GPU): the C ABI loads and exports every
declared symbol, the host construction agrees with the oracle and the direct
sum, the plan file round-trips with the oracle's independent reader/writer,
and malformed input is rejected with the documented status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import direct, midbf, planio
from oracle.phase import Phase as OPhase

mb = pytest.importorskip("paper_1908_09376_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "midbf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(midbf_[a-z_0-9]+)\s*\(", txt))
    names -= {"midbf_rows_fn"}
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(mb.LIB_PATH)
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    for n in names:
        assert n in mb.EXPORTED, f"binding lacks {n}"


def test_binding_constants_match_header():
    """Every MIDBF_* value the header defines equals the binding's constant of
    the same name (status codes, phase families, precisions, middle-factor
    modes, kernel choices, device-plan flags), and the phase ids match synth."""
    txt = open(os.path.join(ROOT, "include", "midbf.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define MIDBF_([A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt)}
    assert len(defs) >= 25
    for name, val in defs.items():
        assert getattr(mb, name) == val, name
    for fam in ("FIO2D", "FIO3D", "FIO2D_JUMP", "DOT", "ZERO", "SEPARABLE", "LOWRANK"):
        assert getattr(synth, "PHASE_" + fam) == defs["PHASE_" + fam]


def _grid(n):
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    return X, W, (np.zeros(2), 1.0), (np.full(2, -n / 2), float(n))


@pytest.mark.parametrize("n,family,n0", [(32, synth.PHASE_FIO2D, 16), (64, synth.PHASE_FIO2D, 64),
                                         (64, synth.PHASE_FIO2D_JUMP, 64), (32, synth.PHASE_DOT, 4)])
def test_host_build_matches_direct_sum(n, family, n0):
    X, W, bx, bw = _grid(n)
    plan = mb.Plan.build(mb.Phase.closed_form(family, X, W), tol=1e-6, n0=n0, boxX=bx, boxW=bw)
    fac = planio.read(plan.export())           # applied by the oracle's own code
    f = synth.complex_gaussian(n * n, 1, 0)[:, 0]
    g = midbf.apply(fac, f)
    gd = direct.direct_sum(OPhase(family, X, W), f)
    assert direct.rel_l2(g, gd) < 2e-5
    st = plan.stats()
    assert st["nx"] == n * n and st["nstages"] == 2 * st["nsteps"] + 1


def test_fp32_storage_keeps_structure_and_accuracy():
    """params.store_fp32 keeps the IDs' coefficients in complex FP32 on the
    host: the same skeletons and ranks as the FP64 build, coefficients equal
    to FP32 rounding, and the oracle's apply of the exported factors within
    FP32 rounding of the FP64 plan's (and within the build tolerance of the
    direct sum)."""
    X, W, bx, bw = _grid(32)
    ph = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    p64 = mb.Plan.build(ph, tol=1e-6, n0=16, boxX=bx, boxW=bw)
    p32 = mb.Plan.build(ph, tol=1e-6, n0=16, boxX=bx, boxW=bw, store_fp32=1)
    assert p32.stats() == p64.stats()
    f64, f32 = planio.read(p64.export()), planio.read(p32.export())
    for s64, s32 in zip(f64.stages, f32.stages):
        for b64, b32 in zip(s64.blocks, s32.blocks):
            for u64, u32 in zip(b64.subs, b32.subs):
                assert np.array_equal(u64.skel, u32.skel) and np.array_equal(u64.red, u32.red)
                assert np.array_equal(u32.T, u64.T.astype(np.complex64).astype(np.complex128))
    f = synth.complex_gaussian(32 * 32, 1, 0)[:, 0]
    g64, g32 = midbf.apply(f64, f), midbf.apply(f32, f)
    assert direct.rel_l2(g32, g64) < 1e-6
    assert direct.rel_l2(g32, direct.direct_sum(OPhase(synth.PHASE_FIO2D, X, W), f)) < 2e-5


def test_host_build_rank_one_exact_and_3d():
    X, W, bx, bw = _grid(32)
    for fam in (synth.PHASE_ZERO, synth.PHASE_SEPARABLE):
        plan = mb.Plan.build(mb.Phase.closed_form(fam, X, W), tol=1e-9, n0=16, boxX=bx, boxW=bw)
        assert plan.stats()["max_rank"] == 1
        fac = planio.read(plan.export())
        f = synth.complex_gaussian(1024, 1, 1)[:, 0]
        assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(OPhase(fam, X, W), f)) < 1e-12
    n = 8
    X3 = synth.uniform_random_points(n ** 3, 3, 0)
    W3 = synth.frequency_grid(n, 3)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO3D, X3, W3), tol=1e-7, n0=8,
                         boxX=(np.zeros(3), 1.0), boxW=(np.full(3, -4.0), 8.0))
    fac = planio.read(plan.export())
    f = synth.complex_gaussian(n ** 3, 1, 0)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(OPhase(synth.PHASE_FIO3D, X3, W3), f)) < 1e-5


def test_lowrank_phase_eval_and_build():
    n = 32
    X, W, bx, bw = _grid(n)
    rng = np.random.default_rng(0)
    U = np.concatenate([X, rng.standard_normal((n * n, 1)) * 0.01], axis=1)
    V = np.concatenate([W, rng.standard_normal((n * n, 1))], axis=1)
    ph = mb.Phase.lowrank(X, W, U, V)
    ix = np.array([0, 5, 700]); iw = np.array([3, 1000, 17])
    assert np.allclose(ph.eval(ix, iw), np.sum(U[ix] * V[iw], axis=1), rtol=0, atol=1e-13)
    U2, V2 = ph.factors()
    assert np.array_equal(U2, U) and np.array_equal(V2, V)
    plan = mb.Plan.build(ph, tol=1e-6, n0=16, boxX=bx, boxW=bw)
    fac = planio.read(plan.export())
    f = synth.complex_gaussian(n * n, 1, 2)[:, 0]
    assert direct.rel_l2(midbf.apply(fac, f), direct.direct_sum(fac.phase, f)) < 2e-5


def test_phase_eval_matches_hand_values():
    X = np.array([[0.25, 0.0], [0.5, 0.0]])
    W = np.array([[3.0, 4.0]])
    p1 = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    assert abs(p1.eval([0], [0])[0] - 1.375) < 1e-14
    p3 = mb.Phase.closed_form(synth.PHASE_FIO2D_JUMP, X, W)
    assert abs(p3.eval([1], [0])[0] - (4 + 13 ** 0.5 / 8)) < 1e-14


def test_phase_eval_matches_hand_values_3d():
    """The library's FP64 evaluation of the 3D FIO phase at the hand-evaluated
    points of tests/golden/phase_values_3d.txt."""
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden", "phase_values_3d.txt"))
            if l.strip() and l[0] != "#"]
    X = np.array([[float(v) for v in r[:3]] for r in rows])
    W = np.array([[float(v) for v in r[3:6]] for r in rows])
    ph = mb.Phase.closed_form(synth.PHASE_FIO3D, X, W)
    got = ph.eval(np.arange(len(rows)), np.arange(len(rows)))
    assert np.abs(got - np.array([float(r[6]) for r in rows])).max() < 1e-14


def test_plan_roundtrip_with_oracle_writer():
    X, W, bx, bw = _grid(32)
    fac = midbf.build(OPhase(synth.PHASE_FIO2D, X, W), n0=16, tol=1e-6, t=2.0, boxX=bx, boxW=bw)
    data = planio.write(fac)
    plan = mb.Plan.load(data)
    assert plan.export() == data


def test_malformed_input_rejected():
    X, W, bx, bw = _grid(16)
    with pytest.raises(mb.MidbfError) as e:
        mb.Phase.closed_form(synth.PHASE_FIO3D, X, W)
    assert e.value.code == mb.EINVAL
    with pytest.raises(mb.MidbfError) as e:
        mb.Phase.closed_form(99, X, W)
    assert e.value.code == mb.EINVAL
    U = np.ones((X.shape[0], 2))
    U[3, 1] = np.nan
    with pytest.raises(mb.MidbfError) as e:
        mb.Phase.lowrank(X, W, U, np.ones((W.shape[0], 2)))
    assert e.value.code == mb.EINVAL
    ph = mb.Phase.closed_form(synth.PHASE_FIO2D, X, W)
    for box in ((np.zeros(2), 0.0), (np.zeros(2), float("nan")), (np.array([0.0, np.inf]), 1.0)):
        with pytest.raises(mb.MidbfError) as e:
            mb.Plan.build(ph, tol=1e-6, n0=16, boxX=box, boxW=bw)
        assert e.value.code == mb.EINVAL
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16, boxX=bx, boxW=bw)
    data = bytearray(plan.export())
    with pytest.raises(mb.MidbfError) as e:
        mb.Plan.load(bytes(data[:-5]))
    assert e.value.code == mb.EFORMAT
    bad = bytearray(data)
    bad[0:8] = b"XXXXXXXX"
    with pytest.raises(mb.MidbfError) as e:
        mb.Plan.load(bytes(bad))
    assert e.value.code == mb.EFORMAT
    # an output position written twice must be caught by validation
    fac = planio.read(bytes(data))
    st = fac.stages[0]
    st.blocks[1].out_idx = st.blocks[0].out_idx.copy()
    with pytest.raises(mb.MidbfError) as e:
        mb.Plan.load(planio.write(fac))
    assert e.value.code == mb.EFORMAT


def test_apply_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X, W, bx, bw = _grid(16)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16, boxX=bx, boxW=bw)
    with pytest.raises(mb.MidbfError) as e:
        mb.DevicePlan(plan, mb.FP32)
    assert e.value.code == mb.ECUDA


def _access(P, n):
    rows = lambda idx: np.exp(2j * np.pi * P(idx[:, None], np.arange(n)[None, :]))
    cols = lambda idx: np.exp(2j * np.pi * P(np.arange(n)[:, None], idx[None, :]))
    return rows, cols


def test_recovery_exact_for_smooth_phase():
    """Algorithm 7 through the C ABI: small path increments -> exact low-rank phase."""
    from oracle import recovery
    n = 32
    X = synth.uniform_grid(n, 2) * 0.3
    W = synth.frequency_grid(n, 2)
    P = OPhase(synth.PHASE_DOT, X, W)
    rows, cols = _access(P, n * n)
    ph = mb.Phase.recover(X, W, rows, cols, r=4, q=2, seed=1)
    info = ph.info
    assert info["mismatches"] == 0 and info["disc_rows"] == 0 and info["disc_cols"] == 0
    assert info["tau"] == 0.25 and info["rows_requested"] >= 8 and info["cols_requested"] >= 8
    U, V = ph.factors()
    S = synth.sample_rows(n * n, 200, 3)
    assert recovery.eps_K(P, U, V, S) < 1e-9


def test_recovery_3d_random_points():
    from oracle import recovery
    X = synth.uniform_random_points(600, 3, 4) * 0.25
    W = synth.uniform_random_points(600, 3, 5) * 2.0
    P = OPhase(synth.PHASE_DOT, X, W)
    rows, cols = _access(P, 600)
    ph = mb.Phase.recover(X, W, rows, cols, r=5, q=2, seed=2)
    U, V = ph.factors()
    assert ph.info["mismatches"] == 0
    assert recovery.eps_K(P, U, V, synth.sample_rows(600, 150, 1)) < 1e-9


def test_recovery_reports_aliasing_on_nyquist_grid():
    """On the uniform FIO grids the phase changes by more than 1/2 per grid
    step near the Nyquist frequency, outside Lemma 3.2's hypothesis: tau is
    driven to 1/2 and recovered rows and columns disagree.  The library must
    report this rather than hide it (the oracle sees the same)."""
    n = 32
    X = synth.uniform_grid(n, 2)
    W = synth.frequency_grid(n, 2)
    P = OPhase(synth.PHASE_FIO2D, X, W)
    rows, cols = _access(P, n * n)
    ph = mb.Phase.recover(X, W, rows, cols, r=4, q=2, seed=0)
    assert ph.info["tau"] == 0.5 and ph.info["mismatches"] > 0


def test_recovery_callback_failure():
    X = synth.uniform_grid(8, 2)
    W = synth.frequency_grid(8, 2)

    def bad(idx):
        raise RuntimeError("no access")

    with pytest.raises(mb.MidbfError) as e:
        mb.Phase.recover(X, W, bad, bad, r=2, q=2)
    assert e.value.code == mb.ECALLBACK
    # values without a phase: NaN, or zero modulus
    for v in (np.nan + 0j, 0j):
        rows = lambda idx: np.full((len(idx), 64), v)
        cols = lambda idx: np.full((64, len(idx)), v)
        with pytest.raises(mb.MidbfError) as e:
            mb.Phase.recover(X, W, rows, cols, r=2, q=2)
        assert e.value.code == mb.ECALLBACK


def test_recovery_path_validation():
    """midbf_rpath_create checks the edges before it touches a device: a parent
    not reached by earlier edges, a child reached twice or an index out of
    range is MIDBF_EINVAL; a valid path without a GPU is MIDBF_ECUDA."""
    for edges in ([[1, 2], [0, 1]], [[0, 1], [0, 1]], [[0, 7]], [[0, 1], [2, 3]]):
        with pytest.raises(mb.MidbfError) as e:
            mb.RecoveryPath(4, np.array(edges), root=0)
        assert e.value.code == mb.EINVAL, edges
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(mb.MidbfError) as e:
            mb.RecoveryPath(4, np.array([[0, 1], [1, 2], [1, 3]]))
        assert e.value.code == mb.ECUDA


def test_recovery_partitions_at_a_jump():
    """Algorithm 6 through the C ABI on a rank-3 phase with a jump of |xi|
    across x1 = 0: discontinuities are flagged along X, tau stays 1/4, rows
    and columns agree, and exp(2 pi i Psi) reproduces K to rounding."""
    from oracle import recovery
    n = 24
    X = synth.uniform_grid(n, 2) * 0.3 - 0.15
    W = synth.frequency_grid(n, 2) * 0.2
    sg = np.where(X[:, 0] >= 0, 1.0, -1.0)
    P = OPhase(synth.PHASE_LOWRANK, X, W, np.stack([X[:, 0], X[:, 1], 0.5 * sg], 1),
               np.stack([W[:, 0], W[:, 1], np.linalg.norm(W, axis=1)], 1))
    rows, cols = _access(P, n * n)
    ph = mb.Phase.recover(X, W, rows, cols, r=4, q=2, seed=0)
    info = ph.info
    assert info["disc_rows"] > 0 and info["tau"] == 0.25 and info["mismatches"] == 0
    U, V = ph.factors()
    assert recovery.eps_K(P, U, V, synth.sample_rows(n * n, 200, 3)) < 1e-12


def test_plan_ranks_agree_with_stats_and_the_oracle_reader():
    """midbf_plan_ranks lists every ID's rank: their count, mean and maximum
    match midbf_plan_stats, and per stage they equal the ranks the oracle's
    independent reader finds in the exported file."""
    n = 32
    X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
    plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16,
                         boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -n / 2), float(n)))
    st = plan.stats()
    allr = plan.ranks()
    assert allr.size == st["nsubs"] and allr.max() == st["max_rank"]
    assert abs(allr.mean() - st["mean_rank"]) < 1e-12
    fac = planio.read(plan.export())
    for q, stage in enumerate(fac.stages):
        ref = [s.skel.size for b in stage.blocks for s in b.subs] if stage.kind != midbf.KIND_S else []
        assert plan.ranks(q).tolist() == ref, q
    with pytest.raises(mb.MidbfError):
        plan.ranks(len(fac.stages))


_FUZZ = r"""
import sys
import numpy as np
import synth
import paper_1908_09376_gb300 as mb
n = 16
X, W = synth.uniform_grid(n, 2), synth.frequency_grid(n, 2)
plan = mb.Plan.build(mb.Phase.closed_form(synth.PHASE_FIO2D, X, W), tol=1e-6, n0=16,
                     boxX=(np.zeros(2), 1.0), boxW=(np.full(2, -8.0), 16.0))
data = plan.export()
rng = np.random.default_rng(int(sys.argv[1]))
loaded = rejected = 0
for it in range(300):
    b = bytearray(data)
    kind = int(rng.integers(0, 4))
    if kind == 0:
        for _ in range(int(rng.integers(1, 4))):
            b[int(rng.integers(0, len(b)))] ^= int(rng.integers(1, 256))
    elif kind == 1:
        pos = int(rng.integers(0, len(b) - 8)) & ~3
        b[pos:pos + 8] = int(rng.choice([-1, 2**31 - 1, 2**40, -2**33, 0])).to_bytes(8, "little", signed=True)
    elif kind == 2:
        b = b[:int(rng.integers(0, len(b)))]
    else:
        pos = int(rng.integers(0, len(b) - 4)) & ~3
        b[pos:pos + 4] = int(rng.choice([-1, 2**31 - 1, 1 << 20, 0, 3])).to_bytes(4, "little", signed=True)
    try:
        mb.Plan.load(bytes(b)).stats()
        loaded += 1
    except mb.MidbfError as e:
        assert e.code in (mb.EFORMAT, mb.EINVAL, mb.ENOMEM), e.code
        rejected += 1
print(loaded, rejected)
"""


def test_corrupted_plan_files_are_rejected_not_crashed():
    """300 random corruptions of a plan file (byte flips, huge or negative
    sizes, truncation): each one loads as a plan that passes validation or is
    rejected with a status code; the process never crashes (run in a child)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", _FUZZ, "7"], capture_output=True, text=True, env=env,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    loaded, rejected = (int(v) for v in out.stdout.split())
    assert loaded + rejected == 300 and rejected > 200
