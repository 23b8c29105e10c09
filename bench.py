#!/usr/bin/env python3
"""Constraint steps/s of the fast implicit constraint-resolution scheme.

One step = one time step of Alg. 3 on the largest workload that fits one GPU,
tissue_c3: an ellipsoid of 0.15 x 0.1 x 0.08 m meshed to 20,000 nodes
(60,075 DOF) with 1,500 contacts split between two 0.02 m sphere tools,
5 Newton iterations x 50 PGS sweeps, FP32 with the 3xTF32 tensor-core
contraction: build W_H (reach, supernodal forward solve, pivot scaling,
contraction), then 5 x (device linearisation of the directions,
W = C W_H C^T, PGS, proximity update), then the corrective motion
dq = A^-1 H^T u.  The line also carries the C1-size liver scene (300
contacts) and the contact-dense press_c1 scene as extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl icr|reference]

--impl icr (default) times libicr on the GPU; under torchrun every rank runs
its own replica of the workload on its own GPU (no collective on the data
path) and rank 0 prints one JSON line.  --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

# concurrent scenes run on separate streams; the default of 8 hardware work
# queues would serialise streams that share a queue (must be set before the
# CUDA context exists)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "constraint steps/sec (W_H build+W update+PGS) at stated err vs FP64; p50/p99 lat"
UNIT = "steps/s"
WORKLOAD = "tissue_c3"
EXTRA_WORKLOADS = ("liver_c1", "press_c1")
L2_FLUSH_BYTES = 512 << 20
ORACLE_SAMPLE_COLUMNS = 48      # W_H columns the oracle solves for the CPU baseline and the parity sample
TF32_PER_BF16 = 1.1 / 2.25      # nominal dense tensor rates of the part (TF32 / BF16)

DESCR = {
    "tissue_c3": "tissue_c3: ellipsoid 0.15x0.1x0.08 m, {N} nodes / {n} DOF, {m} contacts split between two "
                 "0.02 m sphere tools (top and +x end, pressed 6 mm, sliding 0.05 m/s), {k} Newton x {s} PGS "
                 "sweeps, seed 3",
    "liver_c1": "liver_c1: ellipsoid 0.15x0.1x0.08 m, {N} nodes / {n} DOF, {m} contacts vs a 0.02 m sphere tool, "
                "{k} Newton x {s} PGS sweeps, seed 1",
    "press_c1": "press_c1: beam 60x10x5 nodes ({n} DOF) held at its top, pressed 0.2-0.3 mm into a plane, {m} "
                "contacts (most loaded, stick and slip mixed), mu U(0.1, 0.6), {k} Newton x {s} PGS sweeps, seed 5",
}


def describe(name, scene) -> str:
    return DESCR[name].format(N=scene.X.shape[0], n=scene.n, m=scene.m, k=scene.n_newton, s=scene.n_sweeps)


def workload_config(scene) -> dict:
    return {
        "workload": describe(WORKLOAD, scene),
        "n_dof": scene.n,
        "contacts": scene.m,
        "newton_iterations": scene.n_newton,
        "pgs_sweeps": scene.n_sweeps,
        "supernodes": int(scene.factor.sym.nsuper),
        "l2": "flushed (512 MiB write) before every timed step",
    }


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["icr", "reference"], default="icr")
    ap.add_argument("--workload", choices=["tissue_c3", "batch_c2", "precision_c3", "serve_c4", "liver_c1", "press_c1"],
                    default="tissue_c3", help="tissue_c3 is the bench line; the others print their own line "
                                              "(liver_c1 and press_c1: the bench line's measurements on that scene)")
    ap.add_argument("--scenes", type=int, default=64, help="batch_c2: number of scenes")
    ap.add_argument("--batch-groups", default="1,2,4,8,16",
                    help="batch_c2: group counts to try (the fastest of a short timing is used)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve_c4: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=3.0, help="serve_c4: seconds of arrivals")
    ap.add_argument("--slots", type=int, default=32, help="serve_c4: concurrent streams")
    ap.add_argument("--oracle-columns", type=int, default=32, help="precision_c3: W_H columns checked by the oracle")
    ap.add_argument("--modes", default="simt,tf32x3,tf32,bf16", help="precision_c3: FP32 contraction modes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="leave out the liver_c1 and press_c1 keys")
    ap.add_argument("--no-parity", action="store_true", help="leave out the parity figures of the timed run")
    ap.add_argument("--tc-levels", default=None,
                    help="comma list, per etree level (leaves first) the forward-solve tile: 0 = 64-row "
                         "CUDA-core tiles, 1 = tcgen05, 2 = 32-row CUDA-core tiles; fixes the plan instead of "
                         "autotuning (a profiler distorts the autotuner's timings)")
    ap.add_argument("--nvtx-step", action="store_true",
                    help="after the timed steps, replay one more step inside an NVTX range named 'step' "
                         "(for a per-step kernel list: ncu --nvtx --nvtx-include step/)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# kernel -> the source file it is defined in (the ncu figures stay valid while that file is unchanged)
KERNEL_SOURCE = {"k_pgs": "icr_kernels.cu", "k_front_gemm": "icr_kernels.cu", "k_contract": "icr_kernels.cu",
                 "k_update_W": "icr_kernels.cu", "k_assemble": "icr_kernels.cu", "k_front_gemm_tc": "icr_tc.cu",
                 "k_contract_tc": "icr_tc.cu", "k_pack_tc": "icr_tc.cu"}


def source_sha(kernel: str) -> str | None:
    f = KERNEL_SOURCE.get(kernel)
    if f is None:
        return None
    try:
        data = open(os.path.join(ROOT, "paper_2306_06946_gb300", "csrc", f), "rb").read()
    except OSError:
        return None
    return hashlib.sha256(data).hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of ``kernel`` from the ncu summary
    profiles/traffic_<workload>.md (lines "kernel | bytes per launch | source
    sha"), or None when the kernel's source file has changed since."""
    sha = source_sha(kernel)
    try:
        for line in open(os.path.join(ROOT, "profiles", f"traffic_{workload}.md")):
            f = [x.strip() for x in line.strip().strip("|").split("|")]
            if len(f) >= 3 and f[0] == kernel and f[2] == sha:
                return int(float(f[1]))
    except (OSError, ValueError):
        pass
    return None


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------- oracle (CPU)
def oracle_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_columns_job(A, nodes, bary, cols):
    """Columns ``cols`` of W_H = H A^-1 H^T through the oracle's sparse LU
    (factored in the scene's own nested-dissection order); returns the
    columns, the factor time and the solve time.  Runs in a spawned process."""
    from oracle import delassus as dl
    t0 = time.perf_counter()
    solver = dl.SystemSolver(A, "NATURAL")
    t1 = time.perf_counter()
    H = dl.mapping_matrix(nodes, bary, A.shape[0])
    Z = solver.solve(H.T[:, cols].toarray())
    WHc = np.asarray(H @ Z)
    return WHc, t1 - t0, time.perf_counter() - t1


def start_oracle_sample(scene, ncols=ORACLE_SAMPLE_COLUMNS, seed=3):
    """Start the oracle's sampled W_H columns in a spawned process (before any
    GPU work, one BLAS thread); returns (pool, async result, columns)."""
    import multiprocessing as mp
    cols = np.sort(np.random.default_rng(seed).choice(3 * scene.m, size=min(ncols, 3 * scene.m), replace=False))
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        pool = mp.get_context("spawn").Pool(1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, pool.apply_async(oracle_columns_job, (scene.A, scene.nodes, scene.bary, cols)), cols


def oracle_sample_text(ncols, m3, t_fac):
    return (f"{ncols} of the {m3} W_H columns (= H A^-1 H^T e_j) through the oracle's sparse LU solve, scaled to "
            f"all {m3}: the W_H build of one step; the factorisation of A ({t_fac:.1f} s, per system, not per step) "
            "and the Newton iterations are left out, so the value is an upper bound of the oracle's steps/s")


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import scenegen
    from oracle import delassus as dl
    scene = scenegen.NAMED[WORKLOAD]()
    t0 = time.perf_counter()
    solver = dl.SystemSolver(scene.A, "NATURAL")
    t_fac = time.perf_counter() - t0
    H = dl.mapping_matrix(scene.nodes, scene.bary, scene.n)
    m3 = 3 * scene.m
    per = 16                   # W_H columns per sampled step
    rng = np.random.default_rng(7)

    busy = [0.0, 0.0]          # wall and process CPU seconds of the timed samples

    def sample():
        cols = np.sort(rng.choice(m3, size=per, replace=False))
        t, c = time.perf_counter(), time.process_time()
        np.asarray(H @ solver.solve(H.T[:, cols].toarray()))
        wall = time.perf_counter() - t
        busy[0] += wall
        busy[1] += time.process_time() - c
        return wall * m3 / per

    for _ in range(args.warmup):
        sample()
    busy[0] = busy[1] = 0.0
    times = [sample() for _ in range(args.steps)]
    total = sum(times)
    value = len(times) / total
    ms = [1e3 * t for t in times]
    # SuperLU's triangular solves of several right-hand sides call the
    # threaded BLAS: the cores kept busy, from CPU time over wall time
    cores = max(1, round(busy[1] / max(busy[0], 1e-12)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(scene),
        "latency_ms": {"p50": float(statistics.median(ms)), "p99": float(sorted(ms)[int(0.99 * (len(ms) - 1))])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: " + oracle_sample_text(per, m3, t_fac)
                                   + f"; the solves ran on the threaded BLAS, {busy[1] / max(busy[0], 1e-12):.1f} of "
                                     f"{oracle_threads()} host cores busy on average"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def load_scene(icr, driver, ctx, s, precision, contraction="auto", warm_start=False):
    sc = icr.Scene(ctx, precision=precision, n_sweeps=s.n_sweeps, contraction=contraction, warm_start=warm_start)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    return sc


def eager_step(sc, n_newton, stats=False):
    """One time step call by call: lambda~ of every Newton iteration, W of the
    first, the PGS statistics, dq and W_H."""
    sc.reset_proximity()
    sc.build_WH()
    lams, sts, W1 = [], [], None
    for k in range(n_newton):
        sc.linearize(k)
        sc.update_W()
        if k == 0:
            W1 = sc.get("W")
        sts.append(sc.solve_friction(stats=stats))
        lams.append(sc.get("LAMBDA"))
        sc.update_proximity()
    dq = sc.correct_motion(want_dq=True, reset=True)
    return {"WH": sc.get("WH"), "W1": W1, "lams": lams, "stats": sts, "dq": dq}


def timed_graph_steps(torch, sc, stream, flush, steps, warmup):
    for _ in range(warmup):
        sc.step_launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        sc.step_launch()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def phase_times(torch, sc, stream, flush, n_newton, reps=3):
    """Device ms of the paper's table columns, CUDA events on the scene stream."""
    phases = {"build_WH": [], "linearize": [], "update_W": [], "pgs": [], "update_proximity": [], "correct": []}

    def rec(name, fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        phases[name].append((a, b))
    for _ in range(reps):
        flush.fill_(1)
        sc.reset_proximity()
        rec("build_WH", sc.build_WH)
        for k in range(n_newton):
            rec("linearize", lambda: sc.linearize(k))
            rec("update_W", sc.update_W)
            rec("pgs", lambda: sc.solve_friction(warm_start=False))
            rec("update_proximity", sc.update_proximity)
        rec("correct", lambda: sc.correct_motion(want_dq=False, reset=True))
    torch.cuda.synchronize()
    per_launch = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in phases.items()}
    # PGS of each Newton iteration on its own (the first carries the loaded contacts)
    pgs_iter = [statistics.mean(a.elapsed_time(b) for a, b in phases["pgs"][k::n_newton]) for k in range(n_newton)]
    return per_launch, pgs_iter


def kernel_profile(sc, flush, n_newton, reps=3):
    """Per kernel: launches per step and device ms per launch, from CUDA
    events around every launch of `reps` eagerly launched steps."""
    sc.profile_begin()
    for _ in range(reps):
        flush.fill_(1)
        sc.step(n_newton)
    prof = sc.profile_end()
    return {k: {"launches_per_step": n / reps, "ms_per_launch": ms / n, "ms_per_step": ms / reps}
            for k, (n, ms) in prof.items()}


def rooflines(scene, name, prof, info, phase_ms, pgs_stats, peaks, sm_count):
    """Achieved against the bound of each kernel that carries the step's work.
    Algorithmic work per launch: flops from icr_build_info (forward solve
    3q (w^2 + 2 w r), contraction w c (c + 1) per front), bytes from the dense
    definition (W update: W_H read and W written once; PGS: W read once per
    sweep run)."""
    hbm = peaks.get("hbm_gbs") or 6800.0
    bf16 = peaks.get("bf16_tflops") or 1900.0
    src = "measured" if peaks.get("hbm_gbs") else "fallback"
    tf32x3 = bf16 * TF32_PER_BF16 / 3.0
    simt = sm_count * 128 * 2 * (peaks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    m3 = 3 * scene.m
    out = {}

    def ent(k, bound, work, unit, peak, note):
        if k not in prof or prof[k]["launches_per_step"] == 0:
            return
        per = work / prof[k]["launches_per_step"]
        t = prof[k]["ms_per_launch"] / 1e3
        ach = per / t / (1e9 if unit == "GB/s" else 1e12)
        out[k] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                  "traffic": profiled_traffic(k, name), "per_launch": per, "ms_per_launch": 1e3 * t,
                  "share_of_step": prof[k]["ms_per_step"] / sum(v["ms_per_step"] for v in prof.values()),
                  "peak_note": note}
    ent("k_front_gemm_tc", "tensor", info["flops_front_tc"], "TFLOP/s", tf32x3,
        f"3xTF32: the TF32 rate ({src} BF16 burst x {TF32_PER_BF16:.3f}, nominal ratio) / 3 products")
    ent("k_contract_tc", "tensor", info["flops_contract_tc"], "TFLOP/s", tf32x3,
        f"3xTF32: the TF32 rate ({src} BF16 burst x {TF32_PER_BF16:.3f}, nominal ratio) / 3 products")
    ent("k_front_gemm", "alu", info["flops_front_simt"], "TFLOP/s", simt,
        f"FP32 FMA: {sm_count} SMs x 128 lanes x 2 flops x max SM clock")
    ent("k_contract", "alu", info["flops_contract_simt"], "TFLOP/s", simt,
        f"FP32 FMA: {sm_count} SMs x 128 lanes x 2 flops x max SM clock")
    ent("k_update_W", "hbm", scene.n_newton * (2.0 * m3 * m3 * 4 + 9 * scene.m * 4), "GB/s", hbm,
        f"{src} copy bandwidth")
    sweeps = [int(s["sweeps"]) for s in pgs_stats]
    pgs_bytes = sum(sweeps) * m3 * m3 * 4.0 + scene.n_newton * m3 * 4 * 3
    ent("k_pgs", "hbm", pgs_bytes, "GB/s", hbm,
        f"{src} copy bandwidth, against the dense definition's W stream (one read of W per sweep)")
    if "k_pgs" in out:
        t = prof["k_pgs"]["ms_per_launch"] * 1e-3
        visits = sum(sweeps) * scene.m / scene.n_newton
        out["k_pgs"]["latency"] = {
            "sweeps_per_launch": sweeps, "s_only_sweeps_per_launch": [int(s["sweeps_s_only"]) for s in pgs_stats],
            "deferred_folds_per_launch": [int(s["deferred_folds"]) for s in pgs_stats],
            "rechecks_per_launch": [int(s["rechecks"]) for s in pgs_stats],
            "joins_per_launch": [int(s["joins"]) for s in pgs_stats],
            "loaded_contacts_per_launch": [int(s["n_stick"] + s["n_slip"]) for s in pgs_stats],
            "ns_per_contact_visit": t * 1e9 / max(visits, 1),
            "note": "one CTA runs the Gauss-Seidel chain; W stays in L2 when it fits (C3: 81 MB of 129 MB) "
                    "and a sweep reads only the rows of the blocks that may change, so the serial chain "
                    "(local rule, ballot, broadcast, 3x3 fold per applied contact) bounds it, not HBM"}
    flops = info["flops_front_tc"] + info["flops_front_simt"] + info["flops_contract_tc"] + \
        info["flops_contract_simt"]
    ach = flops / (phase_ms["build_WH"] * 1e-3) / 1e12
    out["w_h_build"] = {"bound": "tensor", "achieved": ach, "peak": tf32x3, "unit": "TFLOP/s", "frac": ach / tf32x3,
                        "traffic": None, "per_launch": flops, "ms_per_launch": phase_ms["build_WH"],
                        "peak_note": "the whole W_H build (reach, forward solve, scaling, packing, contraction) "
                                     "against the 3xTF32 rate of its two tensor-core kernels"}
    return out


def run_workload(torch, icr, driver, scene, name, ctx, stream, flush, args, tc_levels_arg=None, full=True):
    """Time one workload in the bench configuration; returns a dict of figures
    and the scene (left open)."""
    sc = load_scene(icr, driver, ctx, scene, icr.FP32)
    if tc_levels_arg:
        plan = [int(x) for x in tc_levels_arg.split(",")]
        sc.set_forward_plan(plan)
        tc_levels = sum(1 for x in plan if x == 1)
    else:
        tc_levels = sc.autotune()
    sc.step_capture(scene.n_newton)
    l0 = sc.launches()
    ms = timed_graph_steps(torch, sc, stream, flush, args.steps, args.warmup)
    graph_launches = (sc.launches() - l0) // max(1, args.steps + args.warmup)
    phase_ms, pgs_iter_ms = phase_times(torch, sc, stream, flush, scene.n_newton)
    prof = kernel_profile(sc, flush, scene.n_newton)
    # PGS statistics of every Newton iteration of one step (FP64 residual check included)
    st = eager_step(sc, scene.n_newton, stats=True)["stats"]
    info = sc.build_info()
    s_ms = sorted(ms)
    return sc, {"ms": ms, "tc_levels": tc_levels, "phase_ms": phase_ms, "pgs_ms_per_iteration": pgs_iter_ms,
                "kernels": prof, "pgs_stats": st, "build_info": info, "graph_kernels_per_step": graph_launches,
                "latency_ms": {"p50": float(statistics.median(ms)),
                               "p99": float(s_ms[int(round(0.99 * (len(ms) - 1)))])}}


def run_icr(args):
    import torch

    import scenegen
    from paper_2306_06946_gb300 import build, driver, icr

    world, rank, local = dist_env()
    scene = scenegen.NAMED[WORKLOAD]()
    # the oracle's sample runs in a spawned process, started before any GPU work
    pool = fut = cols = None
    if rank == 0 and not (args.no_cpu_baseline and args.no_parity):
        pool, fut, cols = start_oracle_sample(scene)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    # a stream of its own (a graph cannot be captured on the legacy default
    # stream), made current so that the L2 flush and the events share it
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = icr.Context(local, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- the timed region: the captured step graph replayed K times
    sc = load_scene(icr, driver, ctx, scene, icr.FP32)
    if args.tc_levels:
        plan = [int(x) for x in args.tc_levels.split(",")]
        sc.set_forward_plan(plan)
        tc_levels = sum(1 for x in plan if x == 1)
    else:
        tc_levels = sc.autotune()
    sc.step_capture(scene.n_newton)
    for _ in range(args.warmup):
        sc.step_launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = sc.launches()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            sc.step_launch()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sc.launches() - l0
    if args.nvtx_step:
        torch.cuda.nvtx.range_push("step")
        sc.step_launch()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # ---- per-phase and per-kernel device times, PGS statistics, rooflines
    phase_ms, pgs_iter_ms = phase_times(torch, sc, stream, flush, scene.n_newton)
    prof = kernel_profile(sc, flush, scene.n_newton)
    step32 = eager_step(sc, scene.n_newton, stats=True)
    info = sc.build_info()
    peaks = measured_peaks()
    roof = rooflines(scene, WORKLOAD, prof, info, phase_ms, step32["stats"], peaks, sm_count)
    dominant = max((k for k in roof if k.startswith("k_")), key=lambda k: prof[k]["ms_per_step"])
    top = {k: roof[dominant][k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    top["kernel"] = dominant
    top.update({k: v for k, v in roof[dominant].items() if k not in top})

    # ---- end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory().numpy()
        h_nodes = pin(scene.nodes, np.int32)
        h_bary = pin(scene.bary, np.float64)
        h_p0 = pin(scene.p0.reshape(-1), np.float64)
        h_anch = pin(scene.obstacle.anchors, np.float64)
        h_mu = pin(scene.mu, np.float64)
        h_dq = pin(np.zeros(scene.n), np.float64)
        h_spheres = pin(np.concatenate([scene.obstacle.centers, scene.obstacle.radii[:, None]], axis=1), np.float64)
        h_tool = pin(scene.obstacle.tool, np.int32)
        # one staged copy per step (icr_set_step_inputs): nodes, sphere ids, bary and mu
        # in FP32, p0, anchors and spheres in FP64, each part 16-byte aligned
        al = lambda x: (x + 15) // 16 * 16
        m_, ns_ = scene.m, h_spheres.shape[0]
        h2d = al(16 * m_) + al(4 * m_) + al(16 * m_) + al(4 * m_) + al(24 * m_) + al(24 * m_) + al(32 * ns_)
        d2h = h_dq.nbytes

        # each step: the step's inputs from pinned host buffers, the captured
        # step graph (it reads the scene's buffers), the corrective motion back
        def e2e_step():
            sc.set_step_inputs(h_nodes, h_bary, h_p0, h_mu, h_spheres, h_tool, h_anch)
            sc.step_launch()
            sc.get("DQ", out=h_dq)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        times = []
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        e2e = {"value": world * len(times) / sum(times), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # ---- extra workloads: the C1-size liver and the contact-dense press scene
    extras = {}
    if rank == 0 and not args.no_extras:
        for name in EXTRA_WORKLOADS:
            if name == WORKLOAD:
                continue
            s2 = scenegen.NAMED[name]()
            sc2, r = run_workload(torch, icr, driver, s2, name, ctx, stream, flush, args)
            ro = rooflines(s2, name, r["kernels"], r["build_info"], r["phase_ms"], r["pgs_stats"], peaks, sm_count)
            extras[name] = {
                "workload": describe(name, s2), "value": 1e3 * args.steps / sum(r["ms"]), "unit": UNIT,
                "ms_per_step": sum(r["ms"]) / args.steps, "latency_ms": r["latency_ms"], "phase_ms": r["phase_ms"],
                "pgs_ms_per_newton_iteration": r["pgs_ms_per_iteration"],
                "tc_levels": r["tc_levels"],
                "kernel_share": {k: v["ms_per_step"] for k, v in r["kernels"].items() if v["ms_per_step"] > 0.01},
                "roofline": {k: {x: ro[k][x] for x in ("bound", "achieved", "unit", "frac")} for k in ro},
                "pgs_latency": ro.get("k_pgs", {}).get("latency"),
            }
            sc2.close()

    # ---- parity of the timed configuration (FP32) on the same scene
    parity = cpu = None
    if rank == 0:
        if not args.no_parity:
            sc64 = load_scene(icr, driver, ctx, scene, icr.FP64)
            step64 = eager_step(sc64, scene.n_newton)
            sc64.close()
            rf = lambda a, b: float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))
            d2 = sum(float(np.linalg.norm(a - b) ** 2) for a, b in zip(step32["lams"], step64["lams"]))
            n2 = sum(float(np.linalg.norm(b) ** 2) for b in step64["lams"])
            parity = {"vs_fp64_gpu_path": {"W_H_rel_fro": rf(step32["WH"], step64["WH"]),
                                           "W_rel_fro": rf(step32["W1"], step64["W1"]),
                                           "lambda_rel_all_iters": (d2 / max(n2, 1e-300)) ** 0.5,
                                           "dq_rel": rf(step32["dq"], step64["dq"])},
                      "note": "the GPU FP64 path matches the oracle at this size to 1e-12 (W_H, W) and 1e-9 "
                              "(lambda~, dq) in tests/test_gpu_fullsize.py; W_H columns are also checked against "
                              "the oracle here"}
        if fut is not None:
            WHc, t_fac, t_sol = fut.get()
            pool.close()
            pool.join()
            if parity is not None:
                rf = lambda a, b: float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))
                parity["W_H_columns_vs_oracle"] = {"columns": int(cols.size),
                                                   "fp32_rel_fro": rf(step32["WH"][:, cols], WHc),
                                                   "fp64_rel_fro": rf(step64["WH"][:, cols], WHc)}
            if world == 1 and not args.no_cpu_baseline:
                m3 = 3 * scene.m
                cpu = {"value": 1.0 / (t_sol / cols.size * m3), "unit": UNIT, "cores": 1, "kind": "oracle",
                       "sample": oracle_sample_text(int(cols.size), m3, t_fac)}

    if rank == 0:
        ms_sorted = sorted(ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**workload_config(scene), "parallelism": f"replicas x{world}",
                       "execution": f"captured step graph replayed per step; forward solve on tcgen05 in "
                                    f"{tc_levels} etree levels, 32-row CUDA-core tiles in "
                                    f"{info['short_tile_levels']}, 64-row tiles elsewhere "
                                    f"({'fixed' if args.tc_levels else 'autotuned'}); 3xTF32 contraction"},
            "latency_ms": {"p50": float(statistics.median(ms)),
                           "p99": float(ms_sorted[int(round(0.99 * (len(ms) - 1)))])},
            "phase_ms": phase_ms,
            "pgs_ms_per_newton_iteration": pgs_iter_ms,
            "roofline": top,
            "roofline_kernels": roof,
            "kernel_ms_per_step": {k: v["ms_per_step"] for k, v in prof.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "parity_vs_fp64": parity,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- batched scenes
def _load_scene(icr, driver, ctx, s, precision=None, warm_start=False):
    sc = icr.Scene(ctx, precision=icr.FP32 if precision is None else precision, n_sweeps=s.n_sweeps,
                   warm_start=warm_start)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    return sc


def _pcts(x):
    x = sorted(x)
    return {"p50": float(x[len(x) // 2]), "p99": float(x[min(len(x) - 1, int(round(0.99 * (len(x) - 1))))])}


def run_batch(args):
    """batch_c2: independent scenes of uneven DOF and contact counts stepped
    together.  The timed line is the batched step (icr_batch: one captured
    graph whose every kernel launch covers all the scenes), K launches between
    CUDA events on the scenes' stream; the same scenes stepped as one captured
    graph per scene on concurrent streams (request loop, every request at
    once) and one after another are reported beside it.  Under torchrun the
    scenes are partitioned across the ranks (no collective on the data path)."""
    import numpy as np
    import torch

    import scenegen
    from paper_2306_06946_gb300 import build, driver, icr, sharding
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    scenes = scenegen.batch_scenes(args.scenes, seed=2)
    mine = sharding.shard([sharding.scene_cost(x.n, x.m) for x in scenes], world, rank)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = icr.Context(local, stream.cuda_stream)
    scs = [_load_scene(icr, driver, ctx, scenes[i]) for i in mine]
    n_newton = scenes[0].n_newton
    for sc, i in zip(scs, mine):
        sc.step_capture(scenes[i].n_newton)
    n = len(scs)
    ids = np.arange(n)
    # ---- the batched step (timed line): the group count (parallel branches of
    # the graph, scenes of similar cost per group) picked by a short timing of
    # each candidate
    def time_batch(bt, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for x, y in evs:
            x.record(stream)
            bt.launch()
            y.record(stream)
        torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in evs]

    group_ms = {}
    cands = [int(g) for g in args.batch_groups.split(",")]
    for g in cands:
        if len(cands) == 1:
            break
        bt = icr.Batch(scs, n_newton, g)
        time_batch(bt, 2)
        group_ms[g] = float(np.median(time_batch(bt, 5)))
        bt.close()
    n_groups = min(group_ms, key=group_ms.get) if group_ms else cands[0]
    b = icr.Batch(scs, n_newton, n_groups)
    resident = ctx.bytes_in_use()
    for _ in range(args.warmup):
        b.launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            b.launch()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = [x.elapsed_time(y) for x, y in ev]
    info = b.info()
    total_s, total_steps = sharding.reduce_timing(sum(ms) / 1e3, n * len(ms), device=f"cuda:{local}")
    # ---- the same scenes: one graph per scene on concurrent streams, and one after another
    b.close()
    for _ in range(max(1, args.warmup)):
        icr.serve(scs, ids, np.zeros(n), n_slots=n)
    torch.cuda.synchronize()
    spans = [icr.serve(scs, ids, np.zeros(n), n_slots=n)[1] for _ in range(args.steps)]
    seq = [icr.serve(scs, ids, np.zeros(n), n_slots=1)[1] for _ in range(2)]
    if rank != 0:
        return
    value = total_steps / total_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / total_steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch_c2: {len(scenes)} independent scenes, nodes log-uniform 500-8000 (ellipsoids "
                               f"and beams), 20-600 contacts, mu U(0.1, 0.6), {sum(x.n for x in scenes)} DOF and "
                               f"{sum(x.m for x in scenes)} contacts in total, 5 Newton x <=50 PGS sweeps",
                   "execution": f"batched step: one captured CUDA graph of {n_groups} parallel branches (cost-balanced groups of "
                                f"scenes), every kernel launch covering all scenes of its group "
                                f"({info['kernel_launches_per_step']} kernel launches per step for the "
                                f"{info['scene_launches_per_step']} of the scenes' own steps)",
                   "l2": f"not flushed: the scenes hold {resident / 2**20:.0f} MiB on the device, above the 129 MB L2",
                   "parallelism": f"scenes partitioned over {world} GPU(s) by cost, rank 0 shown"},
        "batch_makespan_ms": {k: v for k, v in _pcts(ms).items()},
        "groups": n_groups,
        "makespan_ms_by_groups": group_ms,
        "launches_per_step": info["launches_per_step"],
        "kernel_launches_per_step": info["kernel_launches_per_step"],
        "scene_kernel_launches_per_step": info["scene_launches_per_step"],
        "graphs_on_streams": {"makespan_ms": 1e3 * sum(spans) / len(spans),
                              "steps_per_s": n * len(spans) / sum(spans),
                              "execution": f"one captured step graph per scene, all released together on {n} streams"},
        "sequential": {"makespan_ms": 1e3 * min(seq), "steps_per_s": n / min(seq)},
        "speedup_vs_sequential": min(seq) / (total_s / len(ms)),
        "speedup_vs_graphs_on_streams": (sum(spans) / len(spans)) / (total_s / len(ms)),
        "gpu_launches": int(info["launches_per_step"] * len(ms)),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_serve(args):
    """serve_c4: Poisson arrivals of time-step requests over resident scenes of
    the C0, C1 and batched sizes, admitted under a 150 GB HBM budget, served by
    the request loop with concurrent slots; FP64 single-slot serving of the
    same schedule is the plain baseline."""
    import numpy as np
    import torch

    import scenegen
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    pool = [scenegen.NAMED["beam_c0"](), scenegen.NAMED["liver_c1"](), scenegen.NAMED["tissue_c3"]()] + \
        scenegen.batch_scenes(14, seed=4)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    budget = 150 << 30

    def admit(precision):
        ctx = icr.Context(0, stream.cuda_stream, hbm_budget=budget)
        scs, names, rejected = [], [], 0
        for s in pool:
            try:
                sc = _load_scene(icr, driver, ctx, s, precision, warm_start=True)
                sc.step_capture(s.n_newton)
                scs.append(sc)
                names.append(s.name)
            except icr.IcrError as e:
                if e.code != icr.ENOMEM:
                    raise
                rejected += 1
        return ctx, scs, names, rejected

    rng = np.random.default_rng(4)
    nreq = max(1, int(args.rate * args.duration))
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=nreq))
    ctx, scs, names, rejected = admit(icr.FP32)
    which = rng.integers(0, len(scs), size=nreq)
    icr.serve(scs, which[:64], arrivals[:64] - arrivals[0], n_slots=args.slots)   # warm-up
    with ClockSampler(0) as clk:
        lat, span, adm = icr.serve(scs, which, arrivals, n_slots=args.slots, timeout_s=120.0, stats=True)
    frame = 1.0 / 60.0
    ctx64, scs64, _, _ = admit(icr.FP64)
    n64 = max(1, nreq // 10)
    lat64, span64 = icr.serve(scs64, which[:n64], arrivals[:n64], n_slots=1, timeout_s=300.0)
    line = {
        "metric": METRIC, "value": nreq / span, "unit": UNIT, "n_gpus": 1, "steps": nreq, "warmup": 64,
        "ms_per_step": 1e3 * span / nreq, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve_c4: Poisson arrivals, mean {args.rate:g} steps/s for {args.duration:g} s, "
                               f"over {len(scs)} scenes (beam_c0, liver_c1, tissue_c3, 14 batched sizes), "
                               f"requests uniform over the scenes; HBM budget 150 GB ({rejected} rejected at load); "
                               "Newton iteration 1 warm-started from the scene's previous step",
                   "slots": args.slots},
        "admission": adm,
        "latency_ms": {k: 1e3 * v for k, v in _pcts(lat).items()},
        "within_frame_16.7ms": float(np.mean(lat <= frame)),
        "hbm_resident_gb": ctx.bytes_in_use() / 1e9,
        "fp64_single_slot_baseline": {"requests": n64, "steps_per_s": n64 / span64,
                                      "latency_ms": {k: 1e3 * v for k, v in _pcts(lat64).items()}},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- precision table
def _oracle_columns(A, nodes, bary, n, cols):
    """cpu_baseline leg of the precision table: columns ``cols`` of
    W_H = H A^-1 H^T through the oracle's sparse LU (run in a spawned process)."""
    from oracle import delassus as dl
    t0 = time.perf_counter()
    solver = dl.SystemSolver(A, "NATURAL")   # the scene's own nested-dissection order
    t1 = time.perf_counter()
    H = dl.mapping_matrix(nodes, bary, n)
    Z = solver.solve(H.T[:, cols].toarray())
    return np.asarray(H @ Z), t1 - t0, time.perf_counter() - t1


def _states(lam, mu):
    """0 separated, 1 stick, 2 slip (on the cone within 1e-9 relative)."""
    L = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    nt = np.linalg.norm(L[:, 1:], axis=1)
    out = np.where(nt >= mu * L[:, 0] * (1 - 1e-9), 2, 1)
    return np.where(L[:, 0] <= 0, 0, out)


def run_precision(args):
    """precision_c3: one time step of the 60k-DOF two-tool scene in FP64 and in
    FP32 with each contraction dtype; errors of W_H, W, lambda~ and dq against
    the FP64 path (W and the state classification at Newton iteration 1, the
    lambda~ increments of every iteration), the FP64 path's dq residual
    A dq - H^T u, and sampled W_H columns against the oracle."""
    import multiprocessing as mp

    import torch

    import scenegen
    from paper_2306_06946_gb300 import build, driver, icr
    scene = scenegen.NAMED["tissue_c3"]()
    pool = fut = None
    cols = np.sort(np.random.default_rng(3).choice(3 * scene.m, size=min(args.oracle_columns, 3 * scene.m),
                                                   replace=False))
    if cols.size:
        pool = mp.get_context("spawn").Pool(1)
        fut = pool.apply_async(_oracle_columns, (scene.A, scene.nodes, scene.bary, scene.n, cols))
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = icr.Context(0, stream.cuda_stream)

    def hT(u):
        r = np.zeros(scene.n)
        U = u.reshape(-1, 3)
        for i in range(4):
            for ax in range(3):
                np.add.at(r, 3 * scene.nodes[:, i] + ax, scene.bary[:, i] * U[:, ax])
        return r

    def run(prec, mode, w_update="fp32"):
        sc = icr.Scene(ctx, precision=prec, n_sweeps=scene.n_sweeps, contraction=mode, w_update=w_update)
        driver.load_system(sc, scene.factor)
        driver.load_contacts(sc, scene.nodes, scene.bary, scene.p0)
        driver.load_obstacle(sc, scene.obstacle)
        sc.set_field("MU", scene.mu)
        sc.autotune()
        sc.build_WH()
        lams = []
        for k in range(scene.n_newton):
            sc.linearize(k)
            sc.update_W()
            if k == 0:
                W1 = sc.get("W")
            sc.solve_friction()
            lams.append(sc.get("LAMBDA"))
            sc.update_proximity()
        out = {"WH": sc.get("WH"), "W": W1, "lams": lams, "u": sc.get("U")}
        out["dq"] = sc.correct_motion(want_dq=True, reset=True)
        # timing: whole steps and the W_H build alone, CUDA events on the scene stream
        for _ in range(args.warmup):
            sc.step(scene.n_newton)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(args.steps):
            sc.step(scene.n_newton)
        e[1].record(stream)
        e[2].record(stream)
        for _ in range(args.steps):
            sc.build_WH()
        e[3].record(stream)
        torch.cuda.synchronize()
        out["ms_step"] = e[0].elapsed_time(e[1]) / args.steps
        out["ms_build_WH"] = e[2].elapsed_time(e[3]) / args.steps
        sc.close()
        return out

    rf = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    with ClockSampler(0) as clk:
        ref = run(icr.FP64, "simt")
        rows = {}
        jobs = [(mode, mode, "fp32") for mode in args.modes.split(",")]
        # the W update with TF32 / BF16 operands (FP32 accumulation), 3xTF32 contraction
        jobs += [(f"tf32x3+W_{w}", "tf32x3", w) for w in ("tf32", "bf16")]
        for label, mode, wu in jobs:
            r = run(icr.FP32, mode, wu)
            st_ref, st = _states(ref["lams"][0], scene.mu), _states(r["lams"][0], scene.mu)
            d2 = sum(float(np.linalg.norm(a - b) ** 2) for a, b in zip(r["lams"], ref["lams"]))
            n2 = sum(float(np.linalg.norm(b) ** 2) for b in ref["lams"])
            rows[label] = {"W_H_rel_fro": rf(r["WH"], ref["WH"]), "W_rel_fro": rf(r["W"], ref["W"]),
                          "lambda_rel_iter1": rf(r["lams"][0], ref["lams"][0]),
                          "lambda_rel_all_iters": (d2 / max(n2, 1e-300)) ** 0.5, "dq_rel": rf(r["dq"], ref["dq"]),
                          "state_mismatches_iter1": int(np.sum(st != st_ref)),
                          "ms_per_step": r["ms_step"], "ms_build_WH": r["ms_build_WH"]}
    b = hT(ref["u"])
    res = float(np.linalg.norm(scene.A @ ref["dq"] - b) / max(np.linalg.norm(b), 1e-300))
    fp64 = {"ms_per_step": ref["ms_step"], "ms_build_WH": ref["ms_build_WH"], "dq_residual_rel": res,
            "states_iter1": {k: int(v) for k, v in zip(("separated", "stick", "slip"),
                                                       np.bincount(_states(ref["lams"][0], scene.mu), minlength=3))},
            "lambda_norm_per_iter": [float(np.linalg.norm(x)) for x in ref["lams"]]}
    cpu = None
    if fut is not None:
        WHc, t_fac, t_sol = fut.get()
        pool.close()
        pool.join()
        fp64["W_H_columns_vs_oracle_rel"] = rf(ref["WH"][:, cols], WHc)
        fp64["oracle_columns"] = int(cols.size)
        cpu = {"value": cols.size / (t_fac + t_sol), "unit": "W_H columns/s", "cores": 1, "kind": "oracle",
               "sample": f"{cols.size} columns of W_H through the oracle's sparse LU (factor {t_fac:.1f} s, "
                         f"solve {t_sol:.1f} s)"}
    head = "tf32x3" if "tf32x3" in rows else next(iter(rows))
    line = {
        "metric": METRIC, "value": 1e3 / rows[head]["ms_per_step"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[head]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"precision_c3: ellipsoid {scene.n} DOF, {scene.m} contacts split between 2 "
                               f"sphere tools, {scene.n_newton} Newton x {scene.n_sweeps} PGS sweeps, seed 3; "
                               f"value = FP32 path with the {head} contraction",
                   "supernodes": int(scene.factor.sym.nsuper)},
        "errors_vs_fp64": rows, "fp64": fp64, "cpu_baseline": cpu, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    global WORKLOAD
    args = parse()
    if args.workload in ("tissue_c3", "liver_c1", "press_c1"):
        WORKLOAD = args.workload
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_c2":
        run_batch(args)
    elif args.workload == "serve_c4":
        run_serve(args)
    elif args.workload == "precision_c3":
        run_precision(args)
    else:
        run_icr(args)


if __name__ == "__main__":
    main()
