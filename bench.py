#!/usr/bin/env python3
"""Benchmark of the MIDBF apply on GB300 (one JSON line on stdout).

Default workload: the 2D generalized Radon transform of Example 1 (Sec. 4)
on the n = 256 grid, N = 65,536 points, phase x.xi + sqrt(c1^2 xi1^2 +
c2^2 xi2^2), ID tolerance 1e-6, n0 = 64 (L = 5).  --workload selects the 3D
variant (N = 32,768 random points, 256 RHS, BF16 tensor cores with the
refinement products) or the 2D phase with a jump across x1 = 1/2 on the
n = 1024 grid (16 RHS), Example 2 (3D non-uniform Fourier transform, x.xi over
n^3 random points in the unit cube on both sides) or Example 3 (Helmholtz
phase h |x - xi| on the two halves of a sphere mesh of 10 4^l + 2 nodes).
Synthetic inputs (synth.py), seeded.

A step is one pass of the whole hot path over one batch: the forward apply
g = K f followed by the adjoint apply K^H g, both through all levels (V
levels, the on-the-fly middle factor, U levels), in the mixed form (complex
FP32, or BF16 tensor cores with FP32 accumulation).  value = points*RHS
processed per second over all ranks ((|X| + |Omega|) R per step per rank:
the forward apply produces |X| outputs per RHS, the adjoint |Omega|).  Extra keys
report the rel-L2 error of the step's outputs against FP64 direct sums on
sampled rows, the plain FP64 form, 64 right-hand sides, the roofline of the
dominant kernel, the end-to-end time through the host-buffer C entry point,
and the CPU oracle.

Multi-GPU: the apply does not shard across GPUs here (replicas only); with
torchrun each rank runs its own replica and value sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MIDBF apply points*RHS/s and % roofline at rel-L2<=1e-4, mixed vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="grid size of the 2D workloads")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--skip-extras", action="store_true", help="only the headline measurement")
    ap.add_argument("--sweep", default=None,
                    help="comma-separated grid sizes n: the one-RHS FP32 apply of the FIO2D plan family at each "
                         "(the scaling of Fig. 8), with build times; prints one JSON line with a 'sweep' list")
    ap.add_argument("--cpu-sample-every", type=int, default=32,
                    help="the CPU oracle times every k-th block of every stage and scales by the entry ratio "
                         "(1: the whole apply)")
    ap.add_argument("--workload", default="fio2d",
                    choices=["fio2d", "fio3d_n32", "fio2d_jump", "batched", "nuft3d", "nuft3d_recovered",
                             "fio2d_paper", "helmholtz"],
                    help="fio2d: 2D FIO phase on the n x n grid (--n, default 256); fio3d_n32: 3D, N = 32,768, "
                         "random X; fio2d_jump: 2D with the jump |xi| sign(x1 - 1/2) (--n, default 1024); "
                         "nuft3d: Example 2, N = n^3 random points (--n, default 64); nuft3d_recovered: the same "
                         "with the phase recovered from 8 rows and 8 columns of K (Scenario 2, Algorithm 7, "
                         "r = 4, q = 2) and the middle factor made from the low-rank phase; fio2d_paper: Example 1 "
                         "as the paper discretizes it (X and Omega the n x n grid in [0,1)^2, --n default 1024), "
                         "the phase recovered with r = 10, q = 2, ID tolerance 1e-9 (Table 2's setting); "
                         "helmholtz: Example 3 on "
                         "the sphere mesh of refinement level --n (default 6: 20,609 x 20,353 points)")
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides (default: the workload's)")
    ap.add_argument("--mode", default=None, choices=["fp32", "bf16", "bf16r"],
                    help="arithmetic: complex FP32, or BF16 tensor cores with FP32 accumulation "
                         "(bf16r: with the refinement products); default fp32, bf16r for fio3d_n32")
    ap.add_argument("--build", default=None, choices=["host", "device"],
                    help="where the interpolative decompositions run (default: host for fio2d, else device)")
    ap.add_argument("--tune", default=None, choices=["on", "off"],
                    help="run the autotuner for the RHS count before timing (default: on for fio2d_jump)")
    ap.add_argument("--graph", default=None, choices=["on", "off"],
                    help="time the step as one CUDA-graph replay (default: on for fio2d_jump and the one-RHS steps)")
    ap.add_argument("--store", default=None, choices=["fp64", "fp32"],
                    help="host storage of the IDs' coefficients (default fp64; fp32 for fio2d_jump, whose "
                         "n = 1024 plan does not fit host memory in FP64)")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(total_ms_local, units_per_step_per_rank, steps, pg=None, device=None):
    """Whole-job throughput of `steps` timed steps on every rank: the slowest
    rank's time defines the step time (max over ranks); every rank processed
    its own replica, so the units add up over ranks."""
    total_ms = float(total_ms_local)
    world = 1
    if pg is not None:
        import torch
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        total_ms = tt.item()
        world = pg.get_world_size()
    ms_per_step = total_ms / steps
    return ms_per_step, world * units_per_step_per_rank / (ms_per_step * 1e-3)


def aggregate_sharded(total_ms_local, units_local, steps, pg=None, device=None):
    """Whole-job throughput when the ranks share one batch of instances (no
    replicas): the step time is the slowest rank's, the units are the sum of
    every rank's own instances."""
    total_ms, units = float(total_ms_local), float(units_local)
    if pg is not None:
        import torch
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        uu = torch.tensor([units], dtype=torch.float64, device=device)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        pg.all_reduce(uu, op=pg.ReduceOp.SUM)
        total_ms, units = tt.item(), uu.item()
    ms_per_step = total_ms / steps
    return ms_per_step, units / (ms_per_step * 1e-3)


def shard_instances(work, world, rank):
    """Indices of the instances rank `rank` of `world` applies: the instances
    in decreasing order of work, each to the rank with the least work so far
    (ties to the lower rank).  Every instance goes to exactly one rank and no
    data moves between ranks: the instances are independent problems."""
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += work[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def pick_workload(args):
    """The synthetic workload, its RHS count, arithmetic and build site."""
    if args.workload == "fio2d":
        n = args.n or 256
        w = synth.Workload(f"fio2d_n{n}", 2, n, synth.PHASE_FIO2D, 1e-6, 64, 1, 0, sample_rows=256, sample_seed=3)
    elif args.workload == "fio2d_jump":
        base = synth.WORKLOADS["fio2d_jump_n1024"]
        n = args.n or base.n
        w = synth.Workload(f"fio2d_jump_n{n}", 2, n, base.phase, base.tol, base.n0, base.nrhs, base.f_seed,
                           sample_rows=base.sample_rows, sample_seed=base.sample_seed)
    elif args.workload in ("nuft3d", "nuft3d_recovered"):
        base = synth.WORKLOADS["nuft3d_n64"]
        n = args.n or base.n
        rec = args.workload == "nuft3d_recovered"
        w = synth.Workload(f"nuft3d_n{n}" + ("_recovered" if rec else ""), 3, n, base.phase, base.tol, base.n0, 1,
                           base.f_seed, x_kind="random", x_seed=base.x_seed, w_kind="random", w_seed=base.w_seed,
                           sample_rows=256, sample_seed=3, recovered=rec)
    elif args.workload == "fio2d_paper":
        n = args.n or 1024
        w = synth.Workload(f"fio2d_paper_n{n}", 2, n, synth.PHASE_FIO2D, 1e-9, 64, 1, 0, w_kind="unit",
                           recovered=True, sample_rows=256, sample_seed=3, t=5.0)
    elif args.workload == "helmholtz":
        base = synth.WORKLOADS["helmholtz_l6"]
        lev = args.n or base.n
        w = synth.Workload(f"helmholtz_l{lev}", 3, lev, base.phase, base.tol, base.n0, 1, base.f_seed,
                           x_kind="sphere", w_kind="sphere", sample_rows=256, sample_seed=3, t=base.t)
    else:
        w = synth.WORKLOADS[args.workload]
    nrhs = args.nrhs if args.nrhs is not None else w.nrhs
    mode = args.mode if args.mode is not None else ("bf16r" if w.phase == synth.PHASE_FIO3D else "fp32")
    build = args.build if args.build is not None else ("host" if args.workload == "fio2d" else "device")
    store = args.store if args.store is not None else ("fp32" if args.workload == "fio2d_jump" else "fp64")
    jump = args.workload == "fio2d_jump"
    tune = (args.tune or ("on" if jump else "off")) == "on"
    # the step as one CUDA-graph replay: the default for the one-RHS steps of one plan
    # (the headline's 14 launches cost ~2% of its step when issued one by one, and a
    # larger share of the shorter Example 2 and 3 steps) and for the n = 1024 plan
    one_rhs = nrhs == 1 and args.workload in ("fio2d", "nuft3d", "nuft3d_recovered", "fio2d_paper", "helmholtz")
    graph = (args.graph or ("on" if jump or one_rhs else "off")) == "on"
    return w, nrhs, mode, build, store, tune, graph


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture of the kernel as it stands, keyed by (workload, direction, stage index in
# launch order, stage kind); summaries under profiles/.
NCU_TRAFFIC = {
    ("fio2d_n256", "adj", 4, 0): (1.6237e9, "profiles/k_pattern_c1_fio2d_n256_full.md"),
    ("fio2d_n256", "fwd", 2, 0): (1.6268e9, "profiles/k_pattern_fio2d_n256_full.md"),
    ("fio2d_n256", "fwd", 3, 1): (0.0169e9, "profiles/k_s_fly_fio2d_n256_full.md"),
}

# Table 2 of the paper: T_app (s) for Example 1 at n = 16 ... 4096 with r = 10, k = 30.
TABLE2_T_APP = {16: 2.81e-4, 64: 4.43e-3, 256: 4.00e-2, 1024: 6.86e-1, 4096: 1.64e1}

PHASE_NAMES = {synth.PHASE_FIO2D: "FIO2D closed form", synth.PHASE_FIO3D: "FIO3D closed form",
               synth.PHASE_FIO2D_JUMP: "FIO2D + jump closed form", synth.PHASE_DOT: "x.xi closed form",
               synth.PHASE_DISTANCE: "h |x - xi| closed form (h folded into the points)"}


def sampled_direct_error(ph, F, G, Hin, H, rows, cols, chunk=16):
    """rel-L2 of sampled outputs against FP64 direct sums (eq. (1)).

    G = K F and H = K^H Hin as computed on the GPU ((R, N) arrays); for the
    sampled rows i, sum_j exp(2 pi i Phi(x_i, xi_j)) F_j over every column j,
    and for the sampled columns c, sum_i conj(exp(2 pi i Phi(x_i, xi_c))) Hin_i
    over every row, with Phi from the library's FP64 phase evaluation (no part
    of the apply path).  Empty rows or cols give None for that direction."""
    nx, nw = ph.nx, ph.nw
    Fd = F.T.astype(np.complex128)
    Gd = Hin.T.astype(np.complex128)
    num = den = 0.0
    for r0 in range(0, len(rows), chunk):
        rr = rows[r0:r0 + chunk]
        ix = np.repeat(rr, nw)
        iw = np.tile(np.arange(nw, dtype=np.int64), len(rr))
        K = np.exp(2j * np.pi * ph.eval(ix, iw)).reshape(len(rr), nw)
        ref = K @ Fd
        num += np.sum(np.abs(G[:, rr].T - ref) ** 2)
        den += np.sum(np.abs(ref) ** 2)
    e_fwd = math.sqrt(num / den) if len(rows) else None
    num = den = 0.0
    for c0 in range(0, len(cols), chunk):
        cc = cols[c0:c0 + chunk]
        ix = np.tile(np.arange(nx, dtype=np.int64), len(cc))
        iw = np.repeat(cc, nx)
        K = np.exp(-2j * np.pi * ph.eval(ix, iw)).reshape(len(cc), nx)
        ref = K @ Gd
        num += np.sum(np.abs(H[:, cc].T - ref) ** 2)
        den += np.sum(np.abs(ref) ** 2)
    return e_fwd, (math.sqrt(num / den) if len(cols) else None)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": sorted(reasons)}


def _bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh).get("bf16_tflops", 1900.0)
    return 1900.0


PEAK_BF16 = _bf16_peak()
PEAK_BF16_SOURCE = "measured (burst)" if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else "fallback"


def live_copy_gbps(dev, stream, nbytes=1 << 30, reps=5):
    """HBM copy rate of this GPU now: read + write bytes of one device-to-device
    copy over the best of `reps` event-timed copies."""
    import torch
    a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record(stream)
        b.copy_(a)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b
    return 2 * nbytes / best / 1e9


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return p.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class OracleSample:
    """The oracle's apply (its sparse factor product, FP64) on a bounded sample
    of the plan: every `sample_every`-th block of every stage, forward and
    adjoint, for `nrhs` right-hand sides at once; times scale to the whole plan
    by the fraction of factor entries sampled."""

    def __init__(self, plan_bytes, sample_every=32, nrhs=1):
        from oracle import midbf as omidbf
        from oracle import planio
        fac = planio.read(plan_bytes)
        # the oracle's apply is a chain of scipy CSR products, which run on one
        # thread whatever the core count (no BLAS call is involved)
        self.cores = 1
        self.host_cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        rng = np.random.default_rng(0)
        self.parts = []
        sampled = total = 0
        in_len = fac.nw
        for st in fac.stages:
            ent = [(b.xidx.size * b.widx.size) if st.kind == omidbf.KIND_S else
                   sum(s.T.size + s.skel.size for s in b.subs) for b in st.blocks]
            pick = list(range(0, len(st.blocks), sample_every))
            sub = omidbf.Stage(st.kind, st.in_space, st.out_len, st.out_user, [st.blocks[i] for i in pick])
            M = omidbf.stage_matrix(fac, sub, in_len)
            v = rng.standard_normal((in_len, nrhs)) + 1j * rng.standard_normal((in_len, nrhs))
            w = rng.standard_normal((st.out_len, nrhs)) + 1j * rng.standard_normal((st.out_len, nrhs))
            self.parts.append((M, M.conj().T.tocsr(), v, w))
            total += sum(ent)
            sampled += sum(ent[i] for i in pick)
            in_len = st.out_len
        self.scale = total / max(1, sampled)
        what = ("every block (the whole apply)" if sample_every == 1 else
                f"every {sample_every}th block of each stage ({sampled} of {total} factor entries)")
        self.desc = (f"{what}; forward+adjoint sparse FP64 apply of {nrhs} RHS (scipy CSR products, one thread, "
                     f"{self.host_cores} host cores present)" +
                     ("" if sample_every == 1 else "; time scaled by the entry ratio"))

    def step_seconds(self):
        t0 = time.perf_counter()
        for M, MH, v, w in self.parts:
            M @ v
            MH @ w
        return (time.perf_counter() - t0) * self.scale


def cpu_baseline(plan_bytes, n_points, seconds_budget=15.0, nrhs=1, sample_every=32):
    """n_points: outputs of one forward + adjoint step per RHS (|X| + |Omega|)."""
    smp = OracleSample(plan_bytes, sample_every=sample_every, nrhs=nrhs)
    times = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds_budget or len(times) < 3:
        times.append(smp.step_seconds())
    step_s = statistics.median(times)
    return {"value": n_points * nrhs / step_s, "unit": "points*RHS/s", "cores": smp.cores, "kind": "oracle",
            "sample": smp.desc + f"; median of {len(times)} repetitions"}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle's apply as it stands, on the host cores,
    on this arm's workload (its plan built by the library on the host)."""
    if rank != 0:
        return
    if args.workload in ("batched", "fio2d_jump", "nuft3d_recovered"):
        why = {"batched": "32 plans built on the GPU",
               "fio2d_jump": "the n = 1024 plan (1.6e10 T entries) is built on the GPU and does not fit the host twice",
               "nuft3d_recovered": "its phase is recovered with the GPU's Algorithm 4 (--workload nuft3d times the "
                                   "oracle on the closed-form plan of the same points)"}[args.workload]
        print(json.dumps({"impl": "reference", "unavailable": f"oracle arm not run for {args.workload}: {why}"}),
              flush=True)
        return
    import paper_1908_09376_gb300 as mb
    wl, R1, *_ = pick_workload(args)
    X, W, bx, bw = wl.points()
    plan = mb.Plan.build(mb.Phase.closed_form(wl.phase, X, W), tol=wl.tol, n0=wl.n0, boxX=bx, boxW=bw,
                         nthreads=args.threads, t=wl.t)
    smp = OracleSample(plan.export(), sample_every=max(1, args.cpu_sample_every), nrhs=R1)
    del plan
    units = (wl.nx + wl.nw) * R1
    for _ in range(args.warmup):
        smp.step_seconds()
    times = [smp.step_seconds() for _ in range(args.steps)]
    step_s = sum(times) / len(times)
    v = units / step_s
    cpu = {"value": v, "unit": "points*RHS/s", "cores": smp.cores, "kind": "oracle", "sample": smp.desc}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points*RHS/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": wl.name, "N": wl.N, "nx": wl.nx, "nw": wl.nw, "nrhs": R1, "tol": wl.tol,
                      "n0": wl.n0, "step": "forward + adjoint apply"},
           "cpu_baseline": cpu, "e2e": {"value": v, "unit": "points*RHS/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (phase and elapsed seconds); the JSON line stays alone on stdout."""
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def main_batched(args, ws, rank, dev, pg):
    """32 uneven instances (n from {64, 128, 256, 512}, 1..32 RHS, seed 1), each
    applied forward and adjoint: one midbf_apply_batched call of 64 entries
    per step, every plan autotuned for its RHS count."""
    import torch
    import paper_1908_09376_gb300 as mb
    # the config's 32 instances, RHS counts and seeds, with n capped at 256: with the
    # measured ranks one n = 512 plan takes ~20 min of FP64 QR to build and ~20 GB of HBM
    insts = [w if w.n <= 256 else synth.Workload(w.name.replace("_n512", "_n256"), w.d, 256, w.phase, w.tol, w.n0,
                                                 w.nrhs, w.f_seed, sample_rows=256, sample_seed=w.sample_seed)
             for w in synth.batched_instances(32, 1)]
    n_all = len(insts)
    if ws > 1:
        # the batch is shared out: each rank builds and applies its own instances
        # (work ~ points x RHS), no exchange between ranks
        insts = [insts[i] for i in shard_instances([w.N * w.nrhs for w in insts], ws, rank)]
    t0 = time.perf_counter()
    dps, phs, n0s = [], [], []
    for w in insts:
        X, W, bx, bw = w.points()
        ph = mb.Phase.closed_form(w.phase, X, W)
        n0 = w.n0
        plan = mb.Plan.build(ph, tol=w.tol, n0=n0, boxX=bx, boxW=bw, nthreads=args.threads, device_ids=1,
                             store_fp32=1)
        dp = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY, consume=True)
        del plan
        dps.append(dp)
        phs.append(ph)
        n0s.append(n0)
        log(f"instance {w.name}: n0 {n0}, built and uploaded")
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    for dp, w in zip(dps, insts):
        dp.autotune(w.nrhs)
    t_tune = time.perf_counter() - t0
    sel = dps + dps
    adj = [0] * len(insts) + [1] * len(insts)
    nr = [w.nrhs for w in insts] * 2
    f_host = [synth.complex_gaussian(w.N, w.nrhs, w.f_seed) for w in insts]
    h_host = [synth.complex_gaussian(w.N, w.nrhs, w.f_seed + 1000) for w in insts]
    xs = [torch.from_numpy(a.T.copy()).to(dev, torch.complex64) for a in f_host + h_host]
    outs = [torch.empty_like(x) for x in xs]
    wsb = torch.empty(mb.batched_workspace_bytes(sel, nr), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        mb.apply_batched(sel, xs, adj, outs=outs, workspace=wsb)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    units = sum(2 * w.N * w.nrhs for w in insts)
    ms_per_step, value = aggregate_sharded(sum(a.elapsed_time(b) for a, b in ev), units, args.steps, pg, dev)

    # algorithmic bytes of one step: every instance's stages, forward and adjoint
    total_bytes = 0.0
    for dp, x, o, a in zip(sel, xs, outs, adj):
        dp.profile(True)
        dp.apply(x, adjoint=bool(a), out=o)
        total_bytes += sum(by for _, _, by in dp.stage_times())
        dp.profile(False)
    peak, peak_kind = peaks()
    achieved = total_bytes / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": "whole batched step",
                "peak_source": peak_kind}

    # per-instance accuracy against FP64 direct sums on 32 sampled rows / columns
    step()
    torch.cuda.synchronize()
    errs = []
    if rank == 0:
        k = len(insts)
        for i, w in enumerate(insts):
            rows = synth.sample_rows(w.N, 32, w.sample_seed)
            cols = synth.sample_rows(w.N, 32, w.sample_seed + 1)
            G = outs[i].cpu().numpy()              # K f_i
            A = outs[k + i].cpu().numpy()          # K^H h_i
            e_f, e_a = sampled_direct_error(phs[i], f_host[i].T, G, h_host[i].T, A, rows, cols)
            errs.append({"instance": w.name, "nrhs": w.nrhs, "forward": e_f, "adjoint": e_a})

    # end to end: host inputs in pinned memory, copies inside the timed region
    fh = [torch.from_numpy(a.T.astype(np.complex64).copy()).pin_memory() for a in f_host + h_host]
    oh = [torch.empty(tuple(o.shape), dtype=o.dtype).pin_memory() for o in outs]
    ke = max(3, args.steps // 2)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(ke):
        for x, a in zip(xs, fh):
            x.copy_(a, non_blocking=True)
        step()
        for o, a in zip(outs, oh):
            a.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - te) / ke
    io_bytes = sum(x.numel() * 8 for x in xs)
    _, e2e_value = aggregate_sharded(e2e_s * 1e3, units, 1, pg, dev)
    e2e = {"value": e2e_value, "unit": "points*RHS/s", "h2d_bytes_per_step": io_bytes,
           "d2h_bytes_per_step": io_bytes, "ms_per_step": round(e2e_s * 1e3, 4)}
    launches = mb.batched_launches(sel, adj, nr)
    counts = {}
    for w in insts:
        counts[w.n] = counts.get(w.n, 0) + 1
    out = {"metric": METRIC, "value": value, "unit": "points*RHS/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
           "config": {"workload": "batched32_fio2d_n_le_256", "instances": n_all, "instances_on_rank0": len(insts),
                      "n_counts": counts,
                      "nrhs": [w.nrhs for w in insts], "points_rhs_per_step": units, "mode": "fp32",
                      "step": "forward + adjoint of every instance in one midbf_apply_batched call",
                      "tol": 1e-6, "n0": n0s, "build": "device", "store": "fp32", "autotuned": True,
                      "build_s": round(t_build, 1), "tune_s": round(t_tune, 1),
                      "l2": "flushed (512 MB write) between timed steps",
                      "parallelism": f"instances shared out over {ws} ranks" if ws > 1 else "one GPU"},
           "roofline": roofline, "rel_l2_direct_sampled": {"max_forward": max(e["forward"] for e in errs) if errs else None,
                                                           "max_adjoint": max(e["adjoint"] for e in errs) if errs else None,
                                                           "rows": 32, "per_instance": errs},
           "clocks": clk, "e2e": e2e, "gpu_launches": args.steps * launches, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(out), flush=True)


def fio3d_leg(args, dev, stream, flush):
    """The 3D FIO workload (d = 3, N = 32,768 random points, xi in [-16, 16)^3,
    256 RHS, BF16 tensor cores with the refinement products) measured beside
    the headline: forward + adjoint step time, the tensor-pipe fractions of the
    middle factor, and rel-L2 against FP64 direct sums on 512 sampled rows and
    columns."""
    import torch
    import paper_1908_09376_gb300 as mb
    wl = synth.WORKLOADS["fio3d_n32"]
    X, W, bx, bw = wl.points()
    ph = mb.Phase.closed_form(wl.phase, X, W)
    t0 = time.perf_counter()
    plan = mb.Plan.build(ph, tol=wl.tol, n0=wl.n0, boxX=bx, boxW=bw, nthreads=args.threads, t=wl.t, device_ids=1)
    t_build = time.perf_counter() - t0
    dp = mb.DevicePlan(plan, mb.BF16 | mb.REFINE, mb.S_ONTHEFLY, consume=True)
    del plan
    R = wl.nrhs
    sinfo = dp.stage_info()
    ns = len(sinfo)
    f_host = synth.complex_gaussian(wl.nw, R, wl.f_seed)
    F = torch.from_numpy(f_host.T.copy()).to(dev, torch.complex64)
    G = torch.empty((R, wl.nx), dtype=torch.complex64, device=dev)
    H = torch.empty((R, wl.nw), dtype=torch.complex64, device=dev)
    wsb = torch.empty(dp.workspace_bytes(R), dtype=torch.uint8, device=dev)
    for _ in range(3):
        dp.apply(F, out=G, workspace=wsb)
        dp.apply(G, adjoint=True, out=H, workspace=wsb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    k = 3
    for _ in range(k):
        flush.zero_()
        e0.record(stream)
        dp.apply(F, out=G, workspace=wsb)
        dp.apply(G, adjoint=True, out=H, workspace=wsb)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / k
    dp.profile(True)
    s_rows = []
    for adj in (False, True):
        flush.zero_()
        dp.apply(G if adj else F, adjoint=adj, out=H if adj else G, workspace=wsb)
        for q, (kind, sms, _) in enumerate(dp.stage_times()):
            if kind == 1:
                sidx = ns - 1 - q if adj else q
                alg = 8.0 * sinfo[sidx][1] * R / (sms * 1e-3) / 1e12
                s_rows.append({"dir": "adj" if adj else "fwd", "ms": round(sms, 4), "TFLOPs_algorithmic": round(alg, 1),
                               "TFLOPs_issued": round(3 * alg, 1), "issued_frac": round(3 * alg / PEAK_BF16, 4)})
    dp.profile(False)
    dp.apply(F, out=G, workspace=wsb)
    dp.apply(G, adjoint=True, out=H, workspace=wsb)
    torch.cuda.synchronize()
    rows = synth.sample_rows(wl.nx, wl.sample_rows, wl.sample_seed)
    cols = synth.sample_rows(wl.nw, wl.sample_rows, wl.sample_seed + 1)
    Gn, Hn = G.cpu().numpy(), H.cpu().numpy()
    e_f, e_a = sampled_direct_error(ph, f_host.T, Gn, Gn, Hn, rows, cols)
    out = {"workload": wl.name, "N": wl.N, "nrhs": R, "mode": "bf16r", "ms_per_step": round(ms, 4),
           "value": (wl.nx + wl.nw) * R / (ms * 1e-3), "unit": "points*RHS/s", "build_s": round(t_build, 1),
           "s_stage": s_rows, "peak_TFLOPs": PEAK_BF16, "peak_source": PEAK_BF16_SOURCE,
           "rel_l2_direct_sampled": {"forward": e_f, "adjoint": e_a, "rows": wl.sample_rows},
           "status": dp.status(), "l2": "flushed (512 MB write) between timed steps"}
    del dp, wsb, F, G, H
    torch.cuda.empty_cache()
    return out


def main_sweep(args, ws, rank, dev, pg):
    """Fig. 8's scaling in N: the FIO2D family (Example 1's phase on the n x n
    grid, ID tolerance 1e-6, n0 = 64) at each n of --sweep, one RHS, FP32,
    forward + adjoint per step, L2 flushed between steps; with the build, the
    upload and the sampled rel-L2 against FP64 direct sums beside each n."""
    import torch
    import paper_1908_09376_gb300 as mb
    ns = [int(v) for v in args.sweep.split(",") if v.strip()]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows_out = []
    launches = 0
    clocks = ClockSampler(dev.index)
    clocks.start()
    for n in ns:
        w = synth.Workload(f"fio2d_n{n}", 2, n, synth.PHASE_FIO2D, 1e-6, 64, 1, 0, sample_rows=256, sample_seed=3)
        X, W, bx, bw = w.points()
        ph = mb.Phase.closed_form(w.phase, X, W)
        dev_ids = n >= 512          # the host QRs of the large plans take too long
        t0 = time.perf_counter()
        plan = mb.Plan.build(ph, tol=w.tol, n0=w.n0, boxX=bx, boxW=bw, nthreads=args.threads,
                             device_ids=1 if dev_ids else 0, store_fp32=1 if n >= 1024 else 0)
        t_build = time.perf_counter() - t0
        st = plan.stats()
        t0 = time.perf_counter()
        dp = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY, consume=True)
        t_up = time.perf_counter() - t0
        del plan
        fbytes, ibytes = dp.bytes()
        N = w.N
        f_host = synth.complex_gaussian(N, 1, w.f_seed)
        f = torch.from_numpy(f_host[:, 0].copy()).to(dev, torch.complex64)
        g = torch.empty(N, dtype=torch.complex64, device=dev)
        h = torch.empty(N, dtype=torch.complex64, device=dev)
        wsb = torch.empty(dp.workspace_bytes(1), dtype=torch.uint8, device=dev)
        for _ in range(max(3, args.warmup)):
            dp.apply(f, out=g, workspace=wsb)
            dp.apply(g, adjoint=True, out=h, workspace=wsb)
        torch.cuda.synchronize()
        launches += args.steps * 2 * dp.launches(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            dp.apply(f, out=g, workspace=wsb)
            dp.apply(g, adjoint=True, out=h, workspace=wsb)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        rws = synth.sample_rows(N, 256, 3)
        e_f, e_a = sampled_direct_error(ph, f_host.T, g.reshape(1, N).cpu().numpy(), g.reshape(1, N).cpu().numpy(),
                                        h.reshape(1, N).cpu().numpy(), rws, synth.sample_rows(N, 256, 4))
        rows_out.append({"n": n, "N": N, "L": st["L"], "t_entries": st["t_entries"], "s_entries": st["s_entries"],
                         "mean_rank": round(st["mean_rank"], 1), "max_rank": st["max_rank"],
                         "build": "device IDs" if dev_ids else "host", "build_s": round(t_build, 1),
                         "upload_s": round(t_up, 1), "ms_per_step": round(ms, 4),
                         "points_rhs_per_s": 2 * N / (ms * 1e-3),
                         "factor_GBps": round((fbytes + ibytes) * 2 / (ms * 1e-3) / 1e9, 1),
                         "rel_l2_direct_sampled": {"forward": e_f, "adjoint": e_a}})
        log(f"sweep n={n}: {rows_out[-1]}")
        del dp, wsb, f, g, h
        torch.cuda.empty_cache()
    clk = clocks.stop()
    last = rows_out[-1]
    out = {"metric": METRIC, "value": last["points_rhs_per_s"] * ws, "unit": "points*RHS/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": last["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
           "config": {"workload": "fio2d_sweep", "ns": ns, "nrhs": 1, "mode": "fp32", "tol": 1e-6, "n0": 64,
                      "step": "forward + adjoint apply", "l2": "flushed (512 MB write) between timed steps",
                      "value_at": f"n = {last['n']}", "parallelism": f"replicas x{ws}"},
           "sweep": rows_out, "clocks": clk, "gpu_launches": launches, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.sweep:
        import torch
        torch.cuda.set_device(local)
        main_sweep(args, ws, rank, torch.device("cuda", local), None)
        return
    if args.workload == "batched":
        import torch
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        pg = None
        if ws > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=dev)
            pg = dist
        main_batched(args, ws, rank, dev, pg)
        if pg:
            pg.destroy_process_group()
        return
    import torch
    import paper_1908_09376_gb300 as mb
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    wl, R1, mode_name, build_site, store, tune, use_graph = pick_workload(args)
    n = wl.n
    N = wl.N
    nx, nw = wl.nx, wl.nw
    X, W, bx, bw = wl.points()

    t0 = time.perf_counter()
    recovery = None
    ph_true = mb.Phase.closed_form(wl.phase, X, W)
    if wl.recovered:
        # Scenario 2 (Table 1): the phase is not known; Algorithm 7 recovers a rank-r
        # phase from r q rows and r q columns of K (plus those added for
        # discontinuities), with every vector recovery (Algorithm 4) on the GPU.  The
        # rows and columns of K come from the library's FP64 evaluation of the phase.
        r_rec = 10 if args.workload == "fio2d_paper" else 4

        def k_rows(idx):
            ix = np.repeat(idx, nw)
            iw = np.tile(np.arange(nw, dtype=np.int64), len(idx))
            return np.exp(2j * np.pi * ph_true.eval(ix, iw)).reshape(len(idx), nw)

        def k_cols(idx):
            ix = np.tile(np.arange(nx, dtype=np.int64), len(idx))
            iw = np.repeat(idx, nx)
            return np.exp(2j * np.pi * ph_true.eval(ix, iw)).reshape(len(idx), nx).T

        ph = mb.Phase.recover(X, W, k_rows, k_cols, r=r_rec, q=2, seed=0, device=True)
        t_rec = time.perf_counter() - t0
        # eps^K of Sec. 4 on 256 sampled indices: recovered against the true phase
        S = synth.sample_rows(min(nx, nw), 256, 7)
        Ur, Vr = ph.factors()
        A = np.exp(2j * np.pi * ph_true.eval(np.repeat(S, len(S)), np.tile(S, len(S)))).reshape(len(S), len(S))
        B = np.exp(2j * np.pi * (Ur[S] @ Vr[S].T))
        eps_k = float(np.linalg.norm(A - B, 2) / np.linalg.norm(A, 2))
        recovery = {"r": r_rec, "q": 2, "device_unwrap": True, "recover_s": round(t_rec, 2), "eps_K": eps_k,
                    **{k: (float(v) if k == "tau" else int(v)) for k, v in ph.info.items()}}
        log(f"phase recovered: eps_K {eps_k:.2e}, {ph.info}")
        t0 = time.perf_counter()
    else:
        ph = ph_true
    plan = mb.Plan.build(ph, tol=wl.tol, n0=wl.n0, boxX=bx, boxW=bw, nthreads=args.threads, t=wl.t,
                         device_ids=1 if build_site == "device" else 0, store_fp32=1 if store == "fp32" else 0)
    t_build = time.perf_counter() - t0
    st = plan.stats()
    rk = plan.ranks()
    rank_pcts = {p: int(np.percentile(rk, p)) for p in (10, 50, 90)} if rk.size else None
    log(f"built {wl.name}: {st['t_entries']} T entries, {st['s_entries']} S entries")
    t0 = time.perf_counter()
    mode = {"fp32": mb.FP32, "bf16": mb.BF16, "bf16r": mb.BF16 | mb.REFINE}[mode_name]
    keep_plan = args.workload in ("fio2d", "fio2d_paper") and not args.skip_extras and R1 == 1
    # the on-the-fly middle factor takes at most 8 low-rank phase terms; a rank-10
    # recovered phase runs with the middle factor stored
    s_mode_main = mb.S_STORED if (wl.recovered and recovery and recovery["r"] > 8) else mb.S_ONTHEFLY
    # the oracle's baseline needs the plan file; the small workloads export it before the upload
    # consumes the host copy (the n = 1024 plan is too large to hold twice)
    want_cpu = rank == 0 and ws == 1 and not args.skip_extras and args.workload not in ("fio2d_jump",
                                                                                         "nuft3d_recovered")
    plan_bytes = plan.export() if want_cpu and not keep_plan else None
    # large plans: hand the coefficients to the device as they are uploaded
    dp32 = mb.DevicePlan(plan, mode, s_mode_main, consume=not keep_plan)
    t_up = time.perf_counter() - t0
    log("device plan uploaded")
    if not keep_plan:
        del plan                      # the host copy is no longer needed (large plans)
    fbytes, ibytes = dp32.bytes()
    sinfo = dp32.stage_info()

    f_host = synth.complex_gaussian(nw, R1, wl.f_seed)
    f = torch.from_numpy(f_host.T.copy()).to(dev, torch.complex64)
    g = torch.empty((R1, nx), dtype=torch.complex64, device=dev)
    h = torch.empty((R1, nw), dtype=torch.complex64, device=dev)
    if R1 == 1:
        f, g, h = f[0], g[0], h[0]
    ws1 = torch.empty(dp32.workspace_bytes(R1), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    launches_per_apply = dp32.launches(R1)

    t_tune = 0.0
    if tune:
        t0 = time.perf_counter()
        dp32.autotune(R1)
        t_tune = time.perf_counter() - t0
        log("autotuned")

    def step_direct():
        dp32.apply(f, out=g, workspace=ws1)
        dp32.apply(g, adjoint=True, out=h, workspace=ws1)

    step = step_direct
    if use_graph:
        # the forward + adjoint step recorded once, replayed as one graph launch
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        with mb.capture(cs, keep=(f, g, h, ws1)) as cap:
            dp32.apply(f, out=g, workspace=ws1, stream=cs)
            dp32.apply(g, adjoint=True, out=h, workspace=ws1, stream=cs)
        step_graph = cap.graph

        def step():
            step_graph.launch(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop()
    units = (nx + nw) * R1                  # outputs of the forward and the adjoint apply
    ms_per_step, value = aggregate(sum(step_ms), units, args.steps, pg, dev)

    # the same step with the middle factor and its U stage one after the other
    overlap_chunks = dp32.overlap()
    no_overlap = None
    if overlap_chunks > 1 and not use_graph:
        dp32.set_overlap(False)
        t_off = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            step()
            e_b.record(stream)
            torch.cuda.synchronize()
            t_off.append(e_a.elapsed_time(e_b))
        dp32.set_overlap(True)
        no_overlap = {"ms_per_step": round(statistics.mean(t_off), 5), "chunks": overlap_chunks,
                      "speedup_of_overlap": round(statistics.mean(t_off) / ms_per_step, 3)}
    # the same steps again with CUDA events around every stage launch (profiling runs the
    # stages one after the other, without the overlap).  Reading the stage times waits for
    # the GPU, so before each profiled apply a ~1 ms spin keeps the GPU busy while the host
    # queues the apply's launches: an event then never waits for a launch the host has not
    # issued yet, and the times are the kernels' own.  Each stage reports the median of its
    # launches.
    dp32.profile(True)
    stage_ms = {}
    for i in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(2_000_000)
        dp32.apply(f, out=g, workspace=ws1)
        for q, (kind, ms, by) in enumerate(dp32.stage_times()):
            stage_ms.setdefault(("fwd", q, kind, by), []).append(ms)
        torch.cuda._sleep(2_000_000)
        dp32.apply(g, adjoint=True, out=h, workspace=ws1)
        for q, (kind, ms, by) in enumerate(dp32.stage_times()):
            stage_ms.setdefault(("adj", q, kind, by), []).append(ms)
    dp32.profile(False)

    # dominant kernel and its roofline (algorithmic bytes or flops / event-timed duration)
    peak, peak_kind = peaks()
    ns = len(sinfo)
    tc_active = mode_name != "fp32" and R1 >= 16

    def stage_flops(direction, q):
        """Algorithmic flops of a stage launch: 8 per complex multiply-add of
        the method's factor entries (T of the IDs, or the middle factor) per RHS."""
        sidx = q if direction == "fwd" else ns - 1 - q
        return 8.0 * sinfo[sidx][1] * R1

    dom = max(stage_ms.items(), key=lambda kv: statistics.median(kv[1]))
    (direction, q, kind, by), times = dom
    dom_ms = statistics.median(times)
    all_bytes = sum(k[3] for k in stage_ms.keys())
    stage_rows = []
    for k, v in sorted(stage_ms.items(), key=lambda kv: (kv[0][0] != "fwd", kv[0][1])):
        ms_ = statistics.median(v)
        row = {"dir": k[0], "stage": k[1], "kind": "VSU"[k[2]], "ms": round(ms_, 4),
               "GB": round(k[3] / 1e9, 4), "GBps": round(k[3] / (ms_ * 1e-3) / 1e9, 1)}
        if tc_active:
            row["TFLOPs"] = round(stage_flops(k[0], k[1]) / (ms_ * 1e-3) / 1e12, 1)
        stage_rows.append(row)
    # the middle factor made on the fly with the SIMT kernels is bound by the SFU: every
    # entry needs one sine and one cosine, and for the phases with a square-root term one
    # reciprocal square root; the SFU completes 16 operations per clock per SM
    sfu_ops = 3 if wl.phase in (synth.PHASE_FIO2D, synth.PHASE_FIO3D, synth.PHASE_FIO2D_JUMP,
                                synth.PHASE_DISTANCE) and not wl.recovered else 2
    fma_rate, sfu_rate, dfma_rate = mb.pipe_rates(stream)   # measured on this GPU (midbf_pipe_rates)
    copy_live = live_copy_gbps(dev, stream)
    sfu_peak = sfu_rate / sfu_ops / 1e9             # G entries/s
    s_entries_of = {q_: sinfo[q_][1] for q_ in range(ns) if sinfo[q_][0] == 1}

    def hbm_roofline(exclude_s):
        rows = [(k, v) for k, v in stage_ms.items() if not (exclude_s and k[2] == 1)]
        (d_, q_, kind_, by_), t_ = max(rows, key=lambda kv: statistics.median(kv[1]))
        ms_ = statistics.median(t_)
        a_ = by_ / (ms_ * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(a_, 1), "peak": peak, "unit": "GB/s", "frac": round(a_ / peak, 4),
                "traffic": None, "kernel": f"{d_} stage {q_} ({'VSU'[kind_]})", "peak_source": peak_kind}

    roofline_hbm = None
    if tc_active:
        achieved = stage_flops(direction, q) / (dom_ms * 1e-3) / 1e12
        issued = achieved * (3 if mode_name == "bf16r" else 1)
        roofline = {"bound": "tensor", "achieved": round(achieved, 1), "peak": PEAK_BF16, "unit": "TFLOP/s",
                    "frac": round(achieved / PEAK_BF16, 4), "traffic": None,
                    "kernel": f"{direction} stage {q} ({'VSU'[kind]})", "peak_source": PEAK_BF16_SOURCE,
                    "issued_TFLOPs": round(issued, 1), "issued_frac": round(issued / PEAK_BF16, 4),
                    "flops": "8 per complex multiply-add of the factor entries per RHS; refinement issues 3x"}
    elif kind == 1:
        sidx = q if direction == "fwd" else ns - 1 - q
        achieved = s_entries_of[sidx] / (dom_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(sfu_peak, 1), "unit": "Gentries/s",
                    "frac": round(achieved / sfu_peak, 4), "traffic": None,
                    "kernel": f"{direction} stage {q} (S, made on the fly)",
                    "peak_source": (f"measured SFU rate {sfu_rate / 1e12:.3f}e12 ops/s (midbf_pipe_rates) / {sfu_ops} "
                                    "SFU operations per entry (sine, cosine" +
                                    (", reciprocal square root)" if sfu_ops == 3 else ")")),
                    "fma_rate_per_s": fma_rate, "sfu_rate_per_s": sfu_rate}
        roofline_hbm = hbm_roofline(True)
        roofline_hbm["whole_step_GBps"] = round(all_bytes / (ms_per_step * 1e-3) / 1e9, 1)
    else:
        achieved = by / (dom_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None,
                    "kernel": f"{direction} stage {q} ({'VSU'[kind]})", "peak_source": peak_kind,
                    "whole_step_GBps": round(all_bytes / (ms_per_step * 1e-3) / 1e9, 1),
                    "whole_step_frac": round(all_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4)}

    def fill_traffic(rf, key, alg_bytes):
        if rf is None or key not in NCU_TRAFFIC or R1 != 1 or mode_name != "fp32":
            return
        t, src = NCU_TRAFFIC[key]
        rf["traffic"] = t
        rf["traffic_over_algorithmic"] = round(t / alg_bytes, 4)
        rf["traffic_source"] = src + " (ncu, one launch)"

    fill_traffic(roofline, (wl.name, direction, q, kind), by)
    if roofline_hbm is not None:
        k_ = roofline_hbm["kernel"].split()
        dq = (k_[0], int(k_[2]), "VSU".index(k_[3].strip("()")))
        by_ = next(kk[3] for kk in stage_ms if (kk[0], kk[1], kk[2]) == dq)
        fill_traffic(roofline_hbm, (wl.name,) + dq, by_)
    log("timed")
    # accuracy of this run's outputs against FP64 direct sums on sampled rows / columns
    acc = None
    if rank == 0 and wl.sample_rows:
        torch.cuda.synchronize()
        Gn = g.reshape(R1, nx).cpu().numpy()
        Hn = h.reshape(R1, nw).cpu().numpy()
        rows = synth.sample_rows(nx, wl.sample_rows, wl.sample_seed)
        cols = synth.sample_rows(nw, wl.sample_rows, wl.sample_seed + 1)
        e_f, e_a = sampled_direct_error(ph, f_host.T, Gn, Gn, Hn, rows, cols)
        acc = {"forward": e_f, "adjoint": e_a, "rows": int(wl.sample_rows),
               "reference": "FP64 direct sum over all columns (rows) for sampled outputs"}
        if wl.recovered:
            # end to end: against eq. (1) with the true phase (the recovered phase only
            # fixes K up to integers in Psi, which exp(2 pi i .) does not see)
            t_f, t_a = sampled_direct_error(ph_true, f_host.T, Gn, Gn, Hn, rows, cols)
            acc["forward_vs_true_phase"] = t_f
            acc["adjoint_vs_true_phase"] = t_a
            acc["reference"] += "; Phi = the recovered low-rank phase (*_vs_true_phase: the closed form)"

    extras = {}
    vs_baseline = None
    if args.workload == "fio2d_paper":
        # Table 2 (n, r = 10, k = 30): T_app of the paper's MATLAB code on one 3.2 GHz core,
        # presumably FP64; points/s = N / T_app for one direction, the per-direction rate
        # that value also measures (context: another machine and precision)
        t_app = TABLE2_T_APP.get(n)
        if t_app:
            extras["paper_table2"] = {"T_app_s": t_app, "points_per_s": N / t_app, "hardware": "MATLAB, 1 thread, 3.2 GHz",
                                      "row": f"n = {n}, r = 10, k = 30"}
            vs_baseline = value / (N / t_app)
    if not args.skip_extras and R1 == 1 and args.workload == "fio2d_paper":
        # the plain FP64 form of the same recovered factors (the paper's precision)
        dp64 = mb.DevicePlan(plan, mb.FP64, mb.S_STORED)
        f64 = f.to(torch.complex128)
        g64 = torch.empty(N, dtype=torch.complex128, device=dev)
        h64 = torch.empty(N, dtype=torch.complex128, device=dev)
        ws64 = torch.empty(dp64.workspace_bytes(1), dtype=torch.uint8, device=dev)
        for _ in range(3):
            dp64.apply(f64, out=g64, workspace=ws64)
            dp64.apply(g64, adjoint=True, out=h64, workspace=ws64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot64 = 0.0
        k64 = max(3, args.steps // 2)
        for _ in range(k64):
            flush.zero_()
            e0.record(stream)
            dp64.apply(f64, out=g64, workspace=ws64)
            dp64.apply(g64, adjoint=True, out=h64, workspace=ws64)
            e1.record(stream)
            torch.cuda.synchronize()
            tot64 += e0.elapsed_time(e1)
        ms64 = tot64 / k64
        G64 = g64.reshape(1, N).cpu().numpy()
        H64 = h64.reshape(1, N).cpu().numpy()
        rws = synth.sample_rows(N, 256, wl.sample_seed)
        cls = synth.sample_rows(N, 256, wl.sample_seed + 1)
        e_f, e_a = sampled_direct_error(ph_true, f_host.T, G64, G64, H64, rws, cls)
        extras["plain_fp64"] = {"value": 2 * N / (ms64 * 1e-3), "unit": "points*RHS/s", "ms_per_step": round(ms64, 4),
                                "s_mode": "stored", "rel_l2_vs_true_phase": {"forward": e_f, "adjoint": e_a},
                                "vs_paper_table2": (2 * N / (ms64 * 1e-3)) / (N / t_app) if t_app else None}
        del dp64, ws64
    if not args.skip_extras and R1 == 1 and args.workload == "fio2d":
        # plain FP64 form (middle factor stored: FP64 sincospi on GB300 is slow)
        dp64 = mb.DevicePlan(plan, mb.FP64, mb.S_STORED)
        f64 = f.to(torch.complex128)
        g64 = torch.empty(N, dtype=torch.complex128, device=dev)
        h64 = torch.empty(N, dtype=torch.complex128, device=dev)
        ws64 = torch.empty(dp64.workspace_bytes(1), dtype=torch.uint8, device=dev)
        for _ in range(3):
            dp64.apply(f64, out=g64, workspace=ws64)
            dp64.apply(g64, adjoint=True, out=h64, workspace=ws64)
        torch.cuda.synchronize()
        k64 = max(3, args.steps // 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot64 = 0.0
        for _ in range(k64):
            flush.zero_()
            e0.record(stream)
            dp64.apply(f64, out=g64, workspace=ws64)
            dp64.apply(g64, adjoint=True, out=h64, workspace=ws64)
            e1.record(stream)
            torch.cuda.synchronize()
            tot64 += e0.elapsed_time(e1)
        ms64 = tot64 / k64
        dp32.apply(f, out=g, workspace=ws1)
        dp32.apply(g, adjoint=True, out=h, workspace=ws1)
        dp64.apply(g.to(torch.complex128), adjoint=True, out=h64, workspace=ws64)
        torch.cuda.synchronize()
        rel_fwd = (torch.linalg.vector_norm(g.to(torch.complex128) - g64) / torch.linalg.vector_norm(g64)).item()
        rel_adj = (torch.linalg.vector_norm(h.to(torch.complex128) - h64) / torch.linalg.vector_norm(h64)).item()
        # a complex multiply-add is 4 FP64 FMAs; every stored T and S entry once per direction
        fma64 = 2 * 4.0 * (st["t_entries"] + st["s_entries"])
        extras["plain_fp64"] = {"value": 2 * N / (ms64 * 1e-3), "unit": "points*RHS/s", "ms_per_step": round(ms64, 4),
                                "s_mode": "stored", "bound": "alu(fp64)",
                                "roofline": {"bound": "alu", "achieved": round(fma64 / (ms64 * 1e-3) / 1e9, 1),
                                             "peak": round(dfma_rate / 1e9, 1), "unit": "G FP64 FMA/s",
                                             "frac": round(fma64 / (ms64 * 1e-3) / dfma_rate, 4),
                                             "peak_source": "measured FP64 FMA rate (midbf_pipe_rates)",
                                             "work": "4 FP64 FMAs per complex multiply-add of every T and S entry, "
                                                     "forward and adjoint"}}
        extras["speedup_mixed_vs_plain"] = round(ms64 / ms_per_step, 3)
        extras["rel_l2_fp32_vs_fp64"] = {"forward": rel_fwd, "adjoint": rel_adj}
        # the mixed form with the accurate phase (double-FP32 middle-factor phases)
        dpdf = mb.DevicePlan(plan, mb.FP32, mb.S_ONTHEFLY_DF)
        gdf = torch.empty_like(g)
        hdf = torch.empty_like(h)
        wsdf = torch.empty(dpdf.workspace_bytes(1), dtype=torch.uint8, device=dev)
        for _ in range(3):
            dpdf.apply(f, out=gdf, workspace=wsdf)
            dpdf.apply(gdf, adjoint=True, out=hdf, workspace=wsdf)
        torch.cuda.synchronize()
        totdf = 0.0
        for _ in range(k64):
            flush.zero_()
            e0.record(stream)
            dpdf.apply(f, out=gdf, workspace=wsdf)
            dpdf.apply(gdf, adjoint=True, out=hdf, workspace=wsdf)
            e1.record(stream)
            torch.cuda.synchronize()
            totdf += e0.elapsed_time(e1)
        msdf = totdf / k64
        dpdf.apply(f, out=gdf, workspace=wsdf)
        dpdf.apply(g, adjoint=True, out=hdf, workspace=wsdf)   # the adjoint of the same input as h64
        torch.cuda.synchronize()
        extras["fp32_accurate_phase"] = {
            "value": 2 * N / (msdf * 1e-3), "unit": "points*RHS/s", "ms_per_step": round(msdf, 4),
            "s_mode": "on the fly, double-FP32 phase (MIDBF_S_ONTHEFLY_DF)",
            "rel_l2_vs_fp64": {
                "forward": (torch.linalg.vector_norm(gdf.to(torch.complex128) - g64) / torch.linalg.vector_norm(g64)).item(),
                "adjoint": (torch.linalg.vector_norm(hdf.to(torch.complex128) - h64) / torch.linalg.vector_norm(h64)).item()},
            "speedup_vs_plain": round(ms64 / msdf, 3)}
        del dpdf, wsdf, gdf, hdf
        del dp64, ws64
        torch.cuda.empty_cache()
        # 64 right-hand sides, FP32
        R = 64
        F = torch.from_numpy(synth.complex_gaussian(N, R, 0).T.copy()).to(dev, torch.complex64)
        G = torch.empty((R, N), dtype=torch.complex64, device=dev)
        H = torch.empty((R, N), dtype=torch.complex64, device=dev)
        wsR = torch.empty(dp32.workspace_bytes(R), dtype=torch.uint8, device=dev)
        dp32.apply(F, out=G, workspace=wsR)
        torch.cuda.synchronize()
        kR = 3

        def time_r64():
            tot = 0.0
            for _ in range(kR):
                flush.zero_()
                e0.record(stream)
                dp32.apply(F, out=G, workspace=wsR)
                dp32.apply(G, adjoint=True, out=H, workspace=wsR)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            return tot / kR
        msR = time_r64()
        # the autotuner's choice of kernel variant per stage and direction for 64 RHS
        t0_ = time.perf_counter()
        dp32.autotune(R)
        tuneR = time.perf_counter() - t0_
        dp32.apply(F, out=G, workspace=wsR)
        msRt = time_r64()
        # the tuned step's stages, event-timed one by one (the spin keeps the GPU ahead of the host)
        dp32.profile(True)
        stR = []
        for adj_ in (False, True):
            flush.zero_()
            torch.cuda._sleep(2_000_000)
            dp32.apply(G if adj_ else F, adjoint=adj_, out=H if adj_ else G, workspace=wsR)
            for q_, (kind_, ms_, _) in enumerate(dp32.stage_times()):
                stR.append({"dir": "adj" if adj_ else "fwd", "stage": q_, "kind": "VSU"[kind_], "ms": round(ms_, 3)})
        dp32.profile(False)
        # FP32 FMA roof: 4 FMAs per complex multiply-add of every T and S entry, per RHS,
        # forward and adjoint, against the measured FMA rate
        fmaR = 2 * 4 * float(st["t_entries"] + st["s_entries"]) * R
        extras["nrhs64_fp32"] = {
            "value": 2 * N * R / (msRt * 1e-3), "unit": "points*RHS/s", "ms_per_step": round(msRt, 3),
            "autotuned": True, "tune_s": round(tuneR, 1), "stages": stR,
            "default_rules": {"value": 2 * N * R / (msR * 1e-3), "ms_per_step": round(msR, 3)},
            "roofline": {"bound": "alu", "achieved": round(fmaR / (msRt * 1e-3) / 1e12, 2),
                         "peak": round(fma_rate / 1e12, 2), "unit": "T FP32 FMA/s",
                         "frac": round(fmaR / (msRt * 1e-3) / fma_rate, 4),
                         "peak_source": "measured FP32 FMA rate (midbf_pipe_rates)",
                         "work": "4 FP32 FMAs per complex multiply-add of every T and S entry and RHS, forward and adjoint"}}
        for q_ in range(len(sinfo)):
            for a_ in (0, 1):
                dp32.set_choice(R, q_, a_, mb.CHOICE_DEFAULT)
        # the same with every stage on the tensor cores (BF16 + refinement), at 64 and
        # at 256 RHS (one full pass of the TMEM accumulator); forward and adjoint each
        # timed, and per stage: algorithmic flops (8 per complex multiply-add of the
        # method's factor entries per RHS) and issued flops (3 products refined, over
        # the dense blocks that the tensor cores multiply, identity parts included)
        del wsR
        dptc = mb.DevicePlan(plan, mb.BF16 | mb.REFINE, mb.S_ONTHEFLY)
        Gref = G
        for R in (64, 256):
            F = torch.from_numpy(synth.complex_gaussian(N, R, 0).T.copy()).to(dev, torch.complex64)
            if R != 64:
                Gref = torch.empty((R, N), dtype=torch.complex64, device=dev)
                ws32 = torch.empty(dp32.workspace_bytes(R), dtype=torch.uint8, device=dev)
                dp32.apply(F, out=Gref, workspace=ws32)
                del ws32
            Gt = torch.empty((R, N), dtype=torch.complex64, device=dev)
            Ht = torch.empty((R, N), dtype=torch.complex64, device=dev)
            wsR = torch.empty(dptc.workspace_bytes(R), dtype=torch.uint8, device=dev)   # with the RHS-image area
            dptc.apply(F, out=Gt, workspace=wsR)
            dptc.apply(Gt, adjoint=True, out=Ht, workspace=wsR)
            torch.cuda.synchronize()
            tf = ta = 0.0
            for _ in range(kR):
                flush.zero_()
                e0.record(stream)
                dptc.apply(F, out=Gt, workspace=wsR)
                e1.record(stream)
                torch.cuda.synchronize()
                tf += e0.elapsed_time(e1)
                flush.zero_()
                e0.record(stream)
                dptc.apply(Gt, adjoint=True, out=Ht, workspace=wsR)
                e1.record(stream)
                torch.cuda.synchronize()
                ta += e0.elapsed_time(e1)
            dptc.profile(True)
            srows = {}
            for adj_ in (False, True):
                flush.zero_()
                dptc.apply(Gt if adj_ else F, adjoint=adj_, out=Ht if adj_ else Gt, workspace=wsR)
                for q_, (kind_, ms_, _) in enumerate(dptc.stage_times()):
                    sidx = ns - 1 - q_ if adj_ else q_
                    alg = 8.0 * sinfo[sidx][1] * R / (ms_ * 1e-3) / 1e12
                    iss = 3 * 8.0 * (sinfo[sidx][2] if kind_ != 1 else sinfo[sidx][1]) * R / (ms_ * 1e-3) / 1e12
                    srows.setdefault((q_, kind_), []).append((ms_, alg, iss))
            dptc.profile(False)
            s_rows = [v for (q_, k_), v in srows.items() if k_ == 1][0]
            vu = max(((q_, k_, v) for (q_, k_), v in srows.items() if k_ != 1), key=lambda t: sum(x[0] for x in t[2]))
            rel_tc = (torch.linalg.vector_norm(Gt - Gref) / torch.linalg.vector_norm(Gref)).item()
            msT = (tf + ta) / kR
            extras[f"nrhs{R}_bf16_refine"] = {
                "value": 2 * N * R / (msT * 1e-3), "unit": "points*RHS/s", "ms_per_step": round(msT, 3),
                "fwd_ms": round(tf / kR, 3), "adj_ms": round(ta / kR, 3),
                "s_stage_ms": [round(x[0], 4) for x in s_rows],
                "s_stage_TFLOPs_algorithmic": [round(x[1], 1) for x in s_rows],
                "s_stage_TFLOPs_issued": [round(x[2], 1) for x in s_rows],
                "s_stage_issued_frac_of_bf16_peak": [round(x[2] / PEAK_BF16, 4) for x in s_rows],
                "largest_vu_stage": {"stage": vu[0], "kind": "VSU"[vu[1]], "ms": [round(x[0], 4) for x in vu[2]],
                                     "TFLOPs_issued": [round(x[2], 1) for x in vu[2]]},
                "peak_TFLOPs": PEAK_BF16, "peak_source": PEAK_BF16_SOURCE,
                "rel_l2_vs_fp32": rel_tc, "status": dptc.status()}
            del wsR, F, Gt, Ht
        del G, H, Gref, dptc
        torch.cuda.empty_cache()
        # the 3D FIO workload with 256 RHS on the tensor cores, beside the headline
        extras["fio3d_n32_256rhs_bf16r"] = fio3d_leg(args, dev, stream, flush)

    # end to end through the host-buffer entry point (pinned host memory)
    fh = torch.from_numpy(f_host.T.astype(np.complex64).copy()).pin_memory()
    gh = torch.empty((R1, nx), dtype=torch.complex64).pin_memory()
    hh = torch.empty((R1, nw), dtype=torch.complex64).pin_memory()
    wsh = torch.empty(dp32.workspace_bytes(R1, host_io=True), dtype=torch.uint8, device=dev)
    for _ in range(3):
        mb.check(mb.midbf_apply_host(dp32.h, 0, fh.data_ptr(), gh.data_ptr(), R1, stream.cuda_stream,
                                     wsh.data_ptr(), wsh.numel()), "apply_host")
    ke = max(3, args.steps // 2)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(ke):
        mb.check(mb.midbf_apply_host(dp32.h, 0, fh.data_ptr(), gh.data_ptr(), R1, stream.cuda_stream,
                                     wsh.data_ptr(), wsh.numel()), "apply_host")
        mb.check(mb.midbf_apply_host(dp32.h, 1, gh.data_ptr(), hh.data_ptr(), R1, stream.cuda_stream,
                                     wsh.data_ptr(), wsh.numel()), "apply_host")
    e2e_s = (time.perf_counter() - te) / ke
    e2e = {"value": ws * units / e2e_s, "unit": "points*RHS/s", "h2d_bytes_per_step": (nw + nx) * R1 * 8,
           "d2h_bytes_per_step": (nx + nw) * R1 * 8, "ms_per_step": round(e2e_s * 1e3, 4)}

    cpu = None
    if want_cpu:
        try:
            cpu = cpu_baseline(plan_bytes if plan_bytes is not None else plan.export(), nx + nw, nrhs=R1,
                               sample_every=max(1, args.cpu_sample_every))
        except Exception as e:  # the GPU numbers stand without it
            cpu = {"error": f"{type(e).__name__}: {e}"}

    out = {"metric": METRIC, "value": value, "unit": "points*RHS/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": vs_baseline, "dtype": "c64", "data": "synthetic",
           "config": {"workload": wl.name, "N": N, "nx": nx, "nw": nw, "d": wl.d,
                      "phase": (f"{PHASE_NAMES.get(wl.phase, str(wl.phase)).replace(' closed form', '')} recovered "
                                f"from {2 * recovery['r']} rows + {2 * recovery['r']} columns of K (Algorithm 7, "
                                f"r = {recovery['r']}, q = 2): low-rank UV^T" if wl.recovered
                                else PHASE_NAMES.get(wl.phase, str(wl.phase))),
                      "omega": wl.w_kind, "s_mode": "stored" if s_mode_main == mb.S_STORED else "on the fly",
                      "recovery": recovery,
                      "points": wl.x_kind, "nrhs": R1, "mode": mode_name, "step": "forward + adjoint apply",
                      "tol": wl.tol, "n0": wl.n0, "L": st["L"], "build": build_site, "store": store,
                      "autotuned": tune, "tune_s": round(t_tune, 1), "cuda_graph": use_graph,
                      "choices": ([[dp32.choice(R1, q, 0), dp32.choice(R1, q, 1)] for q in range(len(sinfo))]
                                  if tune else None),
                      "t_entries": st["t_entries"], "s_entries": st["s_entries"], "max_rank": st["max_rank"],
                      "mean_rank": round(st["mean_rank"], 1), "rank_percentiles": rank_pcts,
                      "factor_bytes": fbytes, "index_bytes": ibytes,
                      "l2": "flushed (512 MB write) between timed steps",
                      "parallelism": f"replicas x{ws}", "build_s": round(t_build, 1),
                      "upload_s": round(t_up, 1)},
           "roofline": roofline, "roofline_hbm": roofline_hbm, "stages": stage_rows, "rel_l2_direct_sampled": acc,
           "overlap": {"chunks": overlap_chunks, "without": no_overlap,
                       "note": "middle factor and its U stage run chunk by chunk on two streams (midbf_dplan_set_overlap)"},
           "pipe_rates": {"fma_per_s": fma_rate, "sfu_per_s": sfu_rate, "fp64_fma_per_s": dfma_rate,
                          "source": "midbf_pipe_rates, measured"},
           "hbm_copy_live": {"GBps": round(copy_live, 1),
                             "how": "device-to-device copy of 1 GiB in this process (read + write bytes), best of 5; "
                                    "context for this GPU's HBM beside the roofline's peak"},
           "clocks": clk, "e2e": e2e,
           "gpu_launches": args.steps * 2 * launches_per_apply, "cpu_baseline": cpu}
    out.update(extras)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
