#!/usr/bin/env python3
"""Constraint steps/s of the fast implicit constraint-resolution scheme.

One step = one time step of Alg. 3 on the liver workload (ellipsoid of
0.15 x 0.1 x 0.08 m with 3,000 nodes / 9,000 DOF, 300 contacts against a
sphere tool, 5 Newton iterations x 50 PGS sweeps, FP32):
build W_H (reach, supernodal forward solve, FP64 pivot scaling,
contraction), then 5 x (device linearisation of the directions, W = C W_H C^T,
PGS, proximity update), then the corrective motion dq = A^-1 H^T u.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl icr|reference]

--impl icr (default) times libicr on the GPU; under torchrun every rank runs
its own replica of the workload on its own GPU (no collective on the data
path) and rank 0 prints one JSON line.  --impl reference times the FP64 CPU
oracle on the host cores on the same workload.
"""
from __future__ import annotations

import argparse
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
WORKLOAD = "liver_c1"
L2_FLUSH_BYTES = 512 << 20


def workload_config(scene) -> dict:
    return {
        "workload": f"{WORKLOAD}: ellipsoid 0.15x0.1x0.08 m, {scene.X.shape[0]} nodes / {scene.n} DOF, "
                    f"{scene.m} contacts vs 0.02 m sphere tool, {scene.n_newton} Newton x {scene.n_sweeps} PGS "
                    f"sweeps, seed 1",
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
    ap.add_argument("--workload", choices=["liver_c1", "batch_c2", "precision_c3", "serve_c4"], default="liver_c1",
                    help="liver_c1 is the bench line; the others print their own line")
    ap.add_argument("--scenes", type=int, default=64, help="batch_c2: number of scenes")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve_c4: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=3.0, help="serve_c4: seconds of arrivals")
    ap.add_argument("--slots", type=int, default=32, help="serve_c4: concurrent streams")
    ap.add_argument("--oracle-columns", type=int, default=32, help="precision_c3: W_H columns checked by the oracle")
    ap.add_argument("--modes", default="simt,tf32x3,tf32,bf16", help="precision_c3: FP32 contraction modes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tc-levels", default=None,
                    help="liver_c1: comma list, per etree level (leaves first) 1 = forward solve on tcgen05; "
                         "fixes the plan instead of autotuning (a profiler distorts the autotuner's timings)")
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


def profiled_traffic(kernel_marker: str, end_marker: str, profile: str):
    """DRAM bytes per launch recorded by the ncu capture in ``profiles/``, or
    None when the kernel's source has changed since that capture."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_2306_06946_gb300", "csrc", "icr_kernels.cu")).read()
        a, b = src.index(kernel_marker), src.index(end_marker)
        h = hashlib.sha256(src[a:b].encode()).hexdigest()
        rec = {}
        for line in open(os.path.join(ROOT, "profiles", profile)):
            if ":" in line and line.split(":")[0] in ("dram_bytes_per_launch", "kernel_source_sha256"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("kernel_source_sha256") == h:
            return int(rec["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
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


def oracle_step(scene, solver, newton_iters=None):
    """One FP64 oracle time step (fast scheme, Alg. 3); ``newton_iters`` limits
    the Newton iterations for a bounded sample."""
    from oracle import newton as nw
    k = scene.n_newton if newton_iters is None else newton_iters
    return nw.fast_scheme(scene.A, scene.nodes, scene.bary, scene.mu, scene.p0, scene.linearize, k,
                          scene.n_sweeps, solver=solver)


def time_oracle(scene, steps: int, warmup: int, budget_s: float):
    """Time the oracle; when the full steps would not fit ``budget_s`` each
    timed step runs the W_H build plus one Newton iteration and the step time
    is extrapolated to all iterations (the iterations do identical work: a
    fixed sweep count).  Returns (per-step seconds list, sample description)."""
    from oracle import delassus as dl
    from oracle import newton as nw
    solver = dl.SystemSolver(scene.A)
    t0 = time.perf_counter()
    oracle_step(scene, solver)
    t_full = time.perf_counter() - t0
    full = (steps + max(0, warmup - 1)) * t_full <= budget_s
    for _ in range(max(0, warmup - 1)):
        if full:
            oracle_step(scene, solver)
    times = []
    for _ in range(steps):
        if full:
            t0 = time.perf_counter()
            oracle_step(scene, solver)
            times.append(time.perf_counter() - t0)
        else:
            t0 = time.perf_counter()
            H = nw.dl.mapping_matrix(scene.nodes, scene.bary, scene.n)
            WH = nw.dl.compliance_mapping(solver, H)
            t_wh = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle_step_iter(scene, WH)
            t_it = time.perf_counter() - t0
            times.append(t_wh + scene.n_newton * t_it)
    if full:
        sample = "full time steps of the FP64 oracle (fast scheme: W_H = H A^-1 H^T by sparse LU, " \
                 "W = C W_H C^T, PGS, proximity update, dq) on the same scene"
    else:
        sample = "per step: the oracle's W_H build plus one Newton iteration (W update, 50 PGS sweeps, " \
                 "proximity update), step time = W_H + n_newton x iteration (identical iterations)"
    return times, sample


def oracle_step_iter(scene, WH):
    from oracle import delassus as dl
    from oracle import pgs as pg
    C, delta = scene.linearize(scene.p0, 0)
    W = dl.delassus_fast(C, WH)
    lam, _, _ = pg.pgs(W, delta, scene.mu, None, scene.n_sweeps)
    uk = (C.transpose(0, 2, 1) @ lam.reshape(-1, 3, 1)).reshape(-1)
    return WH @ uk


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import scenegen
    scene = scenegen.NAMED[WORKLOAD]()
    times, sample = time_oracle(scene, args.steps, args.warmup, budget_s=150.0)
    total = sum(times)
    value = len(times) / total
    ms = [1e3 * t for t in times]
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(scene),
        "latency_ms": {"p50": float(statistics.median(ms)), "p99": float(sorted(ms)[int(0.99 * (len(ms) - 1))])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def run_icr(args):
    import numpy as np
    import torch

    import scenegen
    from paper_2306_06946_gb300 import build, driver, icr

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    scene = scenegen.NAMED[WORKLOAD]()
    # a stream of its own (a graph cannot be captured on the legacy default
    # stream), made current so that the L2 flush and the events share it
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = icr.Context(local, stream.cuda_stream)
    sc = icr.Scene(ctx, precision=icr.FP32, n_sweeps=scene.n_sweeps)
    driver.load_system(sc, scene.factor)
    driver.load_contacts(sc, scene.nodes, scene.bary, scene.p0)
    driver.load_obstacle(sc, scene.obstacle)
    sc.set_field("MU", scene.mu)

    # one time step (reset p and u, W_H build, n_newton x (linearise, W update,
    # PGS from zero, proximity update), corrective motion), captured once as a
    # CUDA graph after the per-level engine choice and replayed each step
    if args.tc_levels:
        plan = [int(x) for x in args.tc_levels.split(",")]
        sc.set_forward_plan(plan)
        tc_levels = int(sum(plan))
    else:
        tc_levels = sc.autotune()
    sc.step_capture(scene.n_newton)

    def step():
        sc.step_launch()

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    for _ in range(args.warmup):
        step()
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
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sc.launches() - l0
    if args.nvtx_step:
        torch.cuda.nvtx.range_push("step")
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # ---- per-phase device times (the paper's table columns), same stream
    phases = {"build_WH": [], "linearize": [], "update_W": [], "pgs": [], "update_proximity": [], "correct": []}
    for _ in range(3):
        flush.fill_(1)
        sc.reset_proximity()
        for name, fn in [("build_WH", sc.build_WH)]:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream); fn(); b.record(stream)
            phases[name].append((a, b))
        for k in range(scene.n_newton):
            for name, fn in [("linearize", lambda: sc.linearize(k)), ("update_W", sc.update_W),
                             ("pgs", lambda: sc.solve_friction(warm_start=False)),
                             ("update_proximity", sc.update_proximity)]:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream); fn(); b.record(stream)
                phases[name].append((a, b))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream); sc.correct_motion(want_dq=False, reset=True); b.record(stream)
        phases["correct"].append((a, b))
    torch.cuda.synchronize()
    phase_ms = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in phases.items()}

    # ---- sweeps each PGS launch of the step runs (the solve stops at a fixed point)
    sc.reset_proximity()
    sc.build_WH()
    sweeps, s_only, folds = [], [], []
    for k in range(scene.n_newton):
        sc.linearize(k)
        sc.update_W()
        st = sc.solve_friction(warm_start=False, stats=True)
        sweeps.append(int(st["sweeps"]))
        s_only.append(int(st["sweeps_s_only"]))
        folds.append(int(st["deferred_folds"]))
        sc.update_proximity()
    sc.correct_motion(want_dq=False, reset=True)

    # ---- roofline of the dominant kernel (PGS: one k_pgs launch per Newton iteration)
    peaks = measured_peaks()
    m3 = 3 * scene.m
    mean_sweeps = sum(sweeps) / len(sweeps)
    # per launch: W streamed once per sweep run, plus delta, mu and lambda
    pgs_bytes = mean_sweeps * m3 * m3 * 4 + m3 * 4 * 3
    pgs_s = phase_ms["pgs"] / 1e3
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    achieved = pgs_bytes / pgs_s / 1e9
    traffic = profiled_traffic("static constexpr int PGS_MAX_BLOCKS",
                               "template <class T, int BC>\nstatic size_t pgs_smem_bytes", "k_pgs_liver_c1.md")
    roofline = {"kernel": "k_pgs", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "algorithmic_bytes": pgs_bytes, "sweeps_per_launch": sweeps,
                "s_only_sweeps_per_launch": s_only, "deferred_folds_per_launch": folds,
                "ns_per_contact_visit": pgs_s * 1e9 / (mean_sweeps * scene.m),
                "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"}

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

    # ---- parity of the timed configuration (FP32) against the FP64 oracle
    parity = None
    cpu = None
    if rank == 0:
        from oracle import delassus as dl
        solver = dl.SystemSolver(scene.A)
        ref = oracle_step(scene, solver)
        sc.reset_proximity()
        sc.build_WH()
        lams = []
        for k in range(scene.n_newton):
            sc.linearize(k)
            sc.update_W()
            if k == 0:
                W1 = sc.get("W")
            sc.solve_friction(warm_start=False)
            lams.append(sc.get("LAMBDA"))
            sc.update_proximity()
        dq = sc.correct_motion(want_dq=True, reset=True)
        WH_gpu = sc.get("WH")
        W1_ref = ref["iters"][0]["W"]
        d2 = sum(float(np.linalg.norm(a - it["lam"]) ** 2) for a, it in zip(lams, ref["iters"]))
        n2 = sum(float(np.linalg.norm(it["lam"]) ** 2) for it in ref["iters"])
        parity = {"W_H_rel_fro": float(np.linalg.norm(WH_gpu - ref["WH"]) / np.linalg.norm(ref["WH"])),
                  "W_rel_fro": float(np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)),
                  "lambda_rel_all_iters": (d2 / max(n2, 1e-300)) ** 0.5,
                  "dq_rel": float(np.linalg.norm(dq - ref["dq"]) / np.linalg.norm(ref["dq"]))}
        if world == 1 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            oracle_step(scene, solver)
            t = time.perf_counter() - t0
            cpu = {"value": 1.0 / t, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                   "sample": "one full time step of the FP64 oracle (fast scheme, sparse-LU W_H, Python PGS) "
                             "on the same liver_c1 scene"}

    if rank == 0:
        ms_sorted = sorted(ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**workload_config(scene), "parallelism": f"replicas x{world}",
                       "execution": f"captured step graph replayed per step; forward solve on tcgen05 in "
                                    f"{tc_levels} etree levels ({'fixed' if args.tc_levels else 'autotuned'}), CUDA cores elsewhere"},
            "latency_ms": {"p50": float(statistics.median(ms)),
                           "p99": float(ms_sorted[int(round(0.99 * (len(ms) - 1)))])},
            "phase_ms": phase_ms,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "parity_vs_fp64_oracle": parity,
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
    """batch_c2: independent scenes stepped concurrently (one captured step graph
    per scene, replayed through the request loop with every request arriving at
    once) against the same scenes stepped one after another.  Under torchrun the
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
    ctx = icr.Context(local, stream.cuda_stream)
    scs = [_load_scene(icr, driver, ctx, scenes[i]) for i in mine]
    for sc, i in zip(scs, mine):
        sc.step_capture(scenes[i].n_newton)
    n = len(scs)
    ids = np.arange(n)
    for _ in range(args.warmup):
        icr.serve(scs, ids, np.zeros(n), n_slots=n)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = sum(sc.launches() for sc in scs)
    spans, lats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            lat, span = icr.serve(scs, ids, np.zeros(n), n_slots=n)
            spans.append(span)
            lats.extend(lat.tolist())
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sum(sc.launches() for sc in scs) - l0
    total_s, total_steps = sharding.reduce_timing(sum(spans), n * len(spans), device=f"cuda:{local}")
    seq = [icr.serve(scs, ids, np.zeros(n), n_slots=1)[1] for _ in range(2)]
    if rank != 0:
        return
    value = total_steps / total_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / len(spans) / (total_steps / len(spans)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch_c2: {len(scenes)} independent scenes, nodes log-uniform 500-8000 (ellipsoids "
                               f"and beams), 20-600 contacts, mu U(0.1, 0.6), {sum(x.n for x in scenes)} DOF and "
                               f"{sum(x.m for x in scenes)} contacts in total, 5 Newton x <=50 PGS sweeps",
                   "execution": "one captured step graph per scene, all scenes released together on "
                                f"{n} streams (request loop)",
                   "parallelism": f"scenes partitioned over {world} GPU(s) by cost, rank 0 shown"},
        "latency_ms": {k: 1e3 * v for k, v in _pcts(lats).items()},
        "batch_makespan_ms": 1e3 * sum(spans) / len(spans),
        "sequential_makespan_ms": 1e3 * min(seq),
        "speedup_vs_sequential": min(seq) / (sum(spans) / len(spans)),
        "gpu_launches": int(launches),
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
    pool = [scenegen.NAMED["beam_c0"](), scenegen.NAMED["liver_c1"]()] + scenegen.batch_scenes(14, seed=4)
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
        lat, span = icr.serve(scs, which, arrivals, n_slots=args.slots, timeout_s=120.0)
    frame = 1.0 / 60.0
    ctx64, scs64, _, _ = admit(icr.FP64)
    n64 = max(1, nreq // 10)
    lat64, span64 = icr.serve(scs64, which[:n64], arrivals[:n64], n_slots=1, timeout_s=300.0)
    line = {
        "metric": METRIC, "value": nreq / span, "unit": UNIT, "n_gpus": 1, "steps": nreq, "warmup": 64,
        "ms_per_step": 1e3 * span / nreq, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve_c4: Poisson arrivals, mean {args.rate:g} steps/s for {args.duration:g} s, "
                               f"over {len(scs)} resident scenes (beam_c0, liver_c1, 14 batched sizes); "
                               f"HBM budget 150 GB ({rejected} rejected); Newton iteration 1 warm-started from the "
                               "scene's previous step",
                   "slots": args.slots},
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
    solver = dl.SystemSolver(A)
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

    def run(prec, mode):
        sc = icr.Scene(ctx, precision=prec, n_sweeps=scene.n_sweeps, contraction=mode)
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
        for mode in args.modes.split(","):
            r = run(icr.FP32, mode)
            st_ref, st = _states(ref["lams"][0], scene.mu), _states(r["lams"][0], scene.mu)
            d2 = sum(float(np.linalg.norm(a - b) ** 2) for a, b in zip(r["lams"], ref["lams"]))
            n2 = sum(float(np.linalg.norm(b) ** 2) for b in ref["lams"])
            rows[mode] = {"W_H_rel_fro": rf(r["WH"], ref["WH"]), "W_rel_fro": rf(r["W"], ref["W"]),
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
    args = parse()
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
