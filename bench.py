"""Benchmark: batched multiresolution contact detection on one GB300.

Workload (one "step" = one pass of the whole hot path over the batch):
4096 particle pairs of bumped icospheres (subdivision 1..5, 80..20480
triangles, radius log-uniform in [0.1, 1], eps = 0.01 min radius, slab gap
U[-0.5 eps, 3 eps]); hierarchies built once on the host (untimed
preprocessing); per step: pair setup + root test, the per-level surrogate
unfolding, the finest-level tile sweep, exact refinement (FP32 bulk with FP64
final values), penalty forces and energy, and the adjoint (vertex and pose
gradients plus the 12x12 Gauss-Newton blocks).

Metric: particle-pair detections per second (whole job), with the device
timed by CUDA events around CUDA-graph replays of the step.  L2 is flushed
between timed steps (a 256 MiB write).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Floating-point operations per unit of work, counted from the kernels' source
# as FADD + FMUL + 2 FFMA + MUFU (min/max and compares not counted):
FLOPS_PER_SWEEP = 429           # one penalty sweep: 4 iterations, convergence check, certificate
FLOPS_PER_XFORM = 54            # moving B's triangle into A's frame (27 FFMA)
FLOPS_PER_AXIS = 108            # separating-axis test along both face normals
FLOPS_PER_NODE_SWEEP = 398 + 54  # the surrogate sweep has no convergence check
FLOPS_PER_SPHERE_TEST = 11      # bounding-sphere test of a fine pair
FLOPS_PER_FINE_VS_SURR = 18     # fine triangle's sphere vs a surrogate's plane and node sphere
FLOPS_PER_TILE = 40             # per leaf pair: B's surrogate plane and sphere into A's frame
FLOPS_PER_EXPAND_TEST = 29      # child-pair sphere test incl. moving B's centre (9 FFMA)
FLOPS_PER_BOX_TEST = 360        # oriented-box test: B's box into A's frame (63) + six axes (297)
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-merge", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of tuning them first")
    ap.add_argument("--merge-calls", type=int, default=50)
    ap.add_argument("--workload", default="batched", choices=["batched", "packing", "scale"],
                    help="batched: the batched particle-pair step (default); packing: the "
                         "implicit Euler step of a many-particle packing; scale: detection and "
                         "forces of the 136 M-triangle scale workload")
    ap.add_argument("--chunk", type=int, default=65536,
                    help="scale workload: particle pairs per detection call")
    ap.add_argument("--particles", type=int, default=10000)
    ap.add_argument("--packing", choices=("compress", "rsa"), default="compress",
                    help="packing workload: compression by soft-sphere energy minimisation "
                         "or random sequential addition")
    ap.add_argument("--host-trees", action="store_true",
                    help="scale workload: build the surrogate trees on the host instead of the GPU")
    ap.add_argument("--shapes", default=None,
                    help="launch shapes instead of autotuning, e.g. level_warps=4,expand_items=8,"
                         "node_threads=256,tile_warps=8,sweep_warps=2,exact_threads=64")
    return ap.parse_args()


def _dist_init(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _whole_job_rate(steps, units_per_rank, world, ms_max):
    """Units all ranks processed in the timed steps per second of the slowest
    rank (replicas: every rank runs the same workload)."""
    return steps * units_per_rank * world / (ms_max * 1e-3)


def _max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region: the sampler (10 ms period)
    is running, confirmed by its first sample, before the region starts."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t_start = None

    def _read(self):
        import time
        for ln in self.proc.stdout:
            if ln.strip():
                self.raw.append((time.perf_counter(), ln))

    def __enter__(self):
        import threading
        import time
        self.raw = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.raw and time.perf_counter() - t0 < 10.0:
            time.sleep(0.005)
        self.t_start = time.perf_counter()
        return self

    def __exit__(self, *a):
        import time
        t_end = time.perf_counter()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.thread.join(timeout=5)
            # samples taken while the timed region ran
            self.lines = [ln for t, ln in self.raw if self.t_start <= t <= t_end]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources the detection kernels are built from (the traffic table's
# kernels live in mrdem_detect.cu)
TRAFFIC_SOURCES = ("mrdem_detect.cu", "mrdem_device.cuh", "mrdem_geometry.cuh", "mrdem_internal.h",
                   "mrdem_dd.cuh")


def _source_hash():
    """Hash of the detection kernels' sources without their comments and
    blank lines (a traffic figure is valid only for the code it was measured
    on; comment edits do not change it)."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2105_12415_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in TRAFFIC_SOURCES:
            with open(os.path.join(d, f), encoding="utf-8") as fh:
                src = fh.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
            lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
            h.update(f.encode() + b"\0" + "\n".join(lines).encode())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes per launch of each kernel, from the table in the committed
    ncu summary (rows `| kernel | bytes per full launch | source hash |`),
    for rows measured on the current source; {} if none."""
    p = os.path.join(ROOT, "profiles", "dram_traffic_c2_batched.md")
    out = {}
    try:
        with open(p) as f:
            lines = f.read().splitlines()
    except OSError:
        return out
    cur = _source_hash()
    for ln in lines:
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) == 3 and cells[2] == cur:
            try:
                out[cells[0]] = float(cells[1])
            except ValueError:
                pass
    return out


# ---------------------------------------------------------------------------
def _cpu_model():
    """The host CPU's model name (lscpu, then /proc/cpuinfo, then the
    architecture)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine() or "unknown"


def cpu_oracle_baseline(scene, budget_s, n_threads=0):
    """The FP64 oracle (brute force over all fine triangle pairs) on a bounded
    sample of the same workload: from the fixed subset of pair ids = 0 mod 8,
    the largest pairs that fit in about budget_s seconds at a rate calibrated
    on the subset's smallest pair; reported per particle pair of the whole
    workload (its triangle-pair rate over the workload's mean triangle pairs
    per particle pair)."""
    import numpy as np

    import oracle
    oracle.build()
    ntri = np.diff(scene.tri_off)
    ids = np.arange(0, scene.n_pairs, 8)
    work = ntri[scene.pairs[ids, 0]].astype(np.int64) * ntri[scene.pairs[ids, 1]]
    calib = int(ids[int(np.argmin(work))])
    t0 = time.perf_counter()
    oracle.detect(scene.subset([calib]), n_threads=n_threads)
    rate = float(work.min()) / max(time.perf_counter() - t0, 1e-6)
    # the largest pairs that fit: they carry most of the workload's tests
    take, est = [], 0.0
    for k in np.argsort(-work, kind="stable"):
        i, w = int(ids[k]), float(work[k])
        if i != calib and est + w / rate <= budget_s:
            take.append(i)
            est += w / rate
    sub = scene.subset(sorted(take) or [calib])
    t0 = time.perf_counter()
    oracle.detect(sub, n_threads=n_threads)
    dt = time.perf_counter() - t0
    cores = n_threads if n_threads > 0 else (os.cpu_count() or 1)
    nt = np.diff(sub.tri_off)
    tri_pairs = int((nt[sub.pairs[:, 0]].astype(np.int64) * nt[sub.pairs[:, 1]]).sum())
    # the brute force costs one test per triangle pair: its rate in triangle
    # pairs/s, divided by the workload's mean triangle pairs per particle
    # pair, is the workload's rate (a sample's own pairs/s would depend on
    # which sizes it happened to hold)
    mean_work = float((ntri[scene.pairs[:, 0]].astype(np.int64) * ntri[scene.pairs[:, 1]]).mean())
    tri_rate = tri_pairs / dt
    return {"value": tri_rate / mean_work, "unit": "particle-pair detections/s", "cores": cores,
            "kind": "oracle", "triangle_pairs_per_s": tri_rate, "seconds": dt,
            "sample": f"{sub.n_pairs} pairs of the pair-id = 0 mod 8 subset ({tri_pairs} "
                      f"triangle pairs), FP64 brute force, {dt:.1f} s; value = triangle pairs/s "
                      f"/ the workload's mean {mean_work:.4g} triangle pairs per particle pair"}


def merge_oracle_baseline(contacts, eps, gpu_members):
    """The oracle's merge (numpy, one host thread) on the same contact list
    as the GPU call, timed once; its partition must equal the GPU's (the
    merged count and the members of each merged contact, in output order)."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    ref = oracle.merge_contacts(contacts, eps)
    dt = time.perf_counter() - t0
    same = (len(ref["members"]) == len(gpu_members)
            and bool(np.array_equal(ref["members"], np.asarray(gpu_members))))
    return {"ms_per_call": dt * 1e3, "contacts_out": int(len(ref["members"])), "cores": 1,
            "kind": "oracle", "partition_equal": same}


def run_reference(args):
    """The oracle, as it stands, on the host cores (the reference arm)."""
    rank, world, _ = _dist_init(args.gpus)
    if rank != 0:
        return
    from gen import scene_c2
    scene = scene_c2(args.pairs)
    per_step, sample_s = [], []
    last = None
    for k in range(args.warmup + args.steps):
        # the whole run stays within about two minutes of oracle time
        budget = max(0.3, min(args.cpu_budget_s, 120.0 / max(1, args.steps + args.warmup)))
        r = cpu_oracle_baseline(scene, budget)
        if k >= args.warmup:
            per_step.append(r["value"])
            sample_s.append(r["seconds"])
        last = r
    v = sum(per_step) / len(per_step)
    line = {"impl": "reference", "metric": "particle-pair detections/s", "value": v,
            "unit": "particle-pair detections/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup,
            # a projection, not a measured time: the oracle's time for one full
            # step of the workload at the measured rate (a full step would take
            # hours); each timed step ran the bounded sample below
            "ms_per_step": scene.n_pairs / v * 1e3,
            "ms_per_step_projected": True,
            "ms_per_sample_step": 1e3 * sum(sample_s) / len(sample_s),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c2-batched-{args.pairs}-pairs (bounded sample per step)",
                       "pairs": args.pairs},
            "cpu_baseline": {"value": v, "unit": "particle-pair detections/s",
                             "cores": last["cores"], "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": v, "unit": "particle-pair detections/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_packing(args):
    """The implicit Euler step (Algorithm 3) of a random packing of
    bumped icospheres (subdivision 2-4, radius log-uniform in [1, 10], 55 %
    requested, dt = 1e-4, gravity): broad phase once, then Picard iterations
    (pose update, detection, forces, velocity update) and Newton iterations
    (contact Hessian blocks, conjugate-gradient solve, one residual
    evaluation) and multiresolution Picard iterations on settled active sets
    (Algorithm 6), each timed with CUDA events over enqueued iterations, and
    the three solvers run to convergence through the API.  One JSON line."""
    import numpy as np
    import torch

    import paper_2105_12415_gb300 as m
    from gen import scene_packing
    from paper_2105_12415_gb300.api import _p, _stream

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    m.build()
    lib = m.load()
    t0 = time.perf_counter()
    s, achieved, _ = scene_packing(args.particles, 0.55, levels=(2, 3, 4), r_min=1.0, r_max=10.0,
                                   seed=21, method=args.packing)
    packing_s = time.perf_counter() - t0
    n = s.n_particles
    bound = np.array([np.sqrt((s.particle(i)[0].astype(np.float64) ** 2).sum(1)).max()
                      for i in range(n)])
    ctx = m.Context(0)
    hier = m.Hierarchy.from_scene(ctx, s)
    prep_s = time.perf_counter() - t0
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    poses0, mass = t(s.poses), t(s.mass)
    inertia = t(0.4 * s.mass * s.radius ** 2)
    vel0 = t(np.random.default_rng(5).normal(scale=0.05, size=(n, 6)))
    dt = 1e-4
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # broad phase
    tb, tr = t(bound), t(s.radius)
    pairs, eps = m.broad_phase(ctx, poses0, tb, tr)
    P = pairs.shape[0]
    # launch shapes for this batch's size class (untimed preparation)
    tuning = None
    if not args.no_autotune:
        t_tune = time.perf_counter()
        tuning = m.autotune(ctx, hier, pairs, eps, poses0, args.precision, reps=10)
        tuning["s"] = round(time.perf_counter() - t_tune, 2)
        tuning["gain"] = tuning["ms_default"] / tuning["ms_tuned"]
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    a, b = ev(), ev()
    reps = 20
    a.record()
    for _ in range(reps):
        m._lib.check(lib.mrdem_broad_phase(ctx.handle, n, _p(poses0), _p(tb), _p(tr), 0.01,
                                           _p(pairs), _p(eps), P, _p(count), _stream(None)),
                     "broad phase")
    b.record()
    torch.cuda.synchronize()
    bp_ms = a.elapsed_time(b) / reps

    # both solvers to convergence through the API (checked, synchronising)
    t1 = time.perf_counter()
    _, Vp, it_p, _ = m.implicit_euler_step(ctx, hier, poses0, vel0, mass, inertia, pairs, eps, dt,
                                           precision=args.precision, tol=1e-6, max_iter=500)
    picard_s = time.perf_counter() - t1
    t1 = time.perf_counter()
    _, Vn, it_n, nst = m.implicit_euler_step_newton(ctx, hier, poses0, vel0, mass, inertia, pairs,
                                                    eps, dt, precision=args.precision, tol=1e-6,
                                                    max_iter=50)
    newton_s = time.perf_counter() - t1

    # enqueued Picard iterations (no host synchronisation inside)
    V = vel0.clone()
    poses = torch.empty_like(poses0)
    com = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    ft = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    m.move_poses(ctx, poses0, V, dt, out=poses)
    contacts, _ = m.detect(ctx, hier, pairs, eps, poses, args.precision)   # sizes the lists
    stats = torch.zeros(m._lib.MRDEM_STAT_COUNT, dtype=torch.int64, device=dev)

    def picard_iter():
        m.move_poses(ctx, poses0, V, dt, out=poses)
        ft.zero_()
        m.detect(ctx, hier, pairs, eps, poses, args.precision, contacts=contacts, stats=stats,
                 check=False)
        m.contact_forces(ctx, hier, pairs, eps, poses, contacts, mass, com, 1000.0,
                         force_torque=ft, energy=energy)
        m.picard_update(ctx, vel0, ft, mass, inertia, dt, V, norms)

    K = max(args.steps, 10)
    for _ in range(args.warmup):
        picard_iter()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        a.record()
        for _ in range(K):
            picard_iter()
        b.record()
        torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "Picard iterations")
    picard_ms = a.elapsed_time(b) / K

    # enqueued Picard iterations with the candidates kept across the step
    # (detected once at eps + w, refined by exact FP64 distances)
    w = 0.25 * float(eps.min().item())
    cand, _ = m.detect(ctx, hier, pairs, eps + w, poses, args.precision)
    kept = m.refine_contacts(ctx, hier, pairs, eps, poses, cand)
    import ctypes as C

    def cached_iter():
        m.move_poses(ctx, poses0, V, dt, out=poses)
        ft.zero_()
        ci, co = cand.struct(), kept.struct()
        m._lib.check(lib.mrdem_refine_contacts(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                               _p(poses), C.byref(ci), C.byref(co),
                                               _stream(None)), "refine")
        m.contact_forces(ctx, hier, pairs, eps, poses, kept, mass, com, 1000.0,
                         force_torque=ft, energy=energy)
        m.picard_update(ctx, vel0, ft, mass, inertia, dt, V, norms)

    for _ in range(args.warmup):
        cached_iter()
    torch.cuda.synchronize()
    a.record()
    for _ in range(K):
        cached_iter()
    b.record()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "cached Picard iterations")
    cached_ms = a.elapsed_time(b) / K

    # the multiresolution Picard iteration (Algorithm 6): to convergence
    # through the API, then enqueued iterations on settled active sets
    t1 = time.perf_counter()
    _, Vm, it_m, _, rec_m = m.implicit_euler_step_multires(ctx, hier, poses0, vel0, mass, inertia,
                                                           pairs, eps, dt,
                                                           precision=args.precision, tol=1e-6,
                                                           max_iter=500)
    multires_s = time.perf_counter() - t1
    m.move_poses(ctx, poses0, V, dt, out=poses)
    sets = m.active_sets_init(ctx, hier, pairs)
    spare = con_m = sur_m = cnt_m = None
    for _ in range(30):
        spare, con_m, sur_m, cnt_m = m.active_sets_step(ctx, hier, pairs, eps, poses, sets, spare,
                                                        args.precision, con_m, sur_m, cnt_m)
        sets, spare = spare, sets
        if cnt_m[0].item() == 0 and cnt_m[1].item() == 0:
            break
    act = [sets, spare]

    def multires_iter():
        m.move_poses(ctx, poses0, V, dt, out=poses)
        ft.zero_()
        m.active_sets_step(ctx, hier, pairs, eps, poses, act[0], act[1], args.precision, con_m,
                           sur_m, cnt_m, check=False)
        m.contact_forces(ctx, hier, pairs, eps, poses, con_m, mass, com, 1000.0,
                         force_torque=ft, energy=energy)
        m.surrogate_forces(ctx, hier, pairs, eps, poses, sur_m, mass, com, 1000.0, 0.25,
                           force_torque=ft, energy=energy)
        m.picard_update(ctx, vel0, ft, mass, inertia, dt, V, norms)
        act.reverse()

    for _ in range(args.warmup):
        multires_iter()
    torch.cuda.synchronize()
    a.record()
    for _ in range(K):
        multires_iter()
    b.record()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "multiresolution iterations")
    multires_ms = a.elapsed_time(b) / K
    ctx.profile(True)
    for _ in range(K):
        multires_iter()
    torch.cuda.synchronize()
    ctx.profile(False)
    multires_parts = {k: round(v[0] / K, 4) for k, v in ctx.profile_read().items()}
    flat_stats = stats.cpu().numpy()
    multires = {"ms_per_iteration": round(multires_ms, 4), "iterations_to_1e-6": it_m,
                "wall_s": round(multires_s, 3), "active_items": act[0].n(),
                "pairs_of_leaves": int(cnt_m[2].item()),
                "widening_iterations": sum(r["widened"] > 0 for r in rec_m),
                "surrogate_contacts_first": [r["surrogate"] for r in rec_m[:6]],
                "agree_with_picard": float((Vp - Vm).abs().max().item() / Vp.abs().max().item()),
                "ms_parts": multires_parts,
                "flat_node_pair_tests": int(flat_stats[m._lib.MRDEM_STAT_TESTS:
                                                       m._lib.MRDEM_STAT_TESTS + 8].sum()),
                "flat_leaf_tiles": int(flat_stats[m._lib.MRDEM_STAT_TILES])}

    # enqueued Newton iterations: Hessian blocks, CG solve, one residual evaluation
    blocks = torch.zeros((P, 12, 12), dtype=torch.float64, device=dev)
    res = torch.empty((n, 6), dtype=torch.float64, device=dev)
    x = torch.empty((n, 6), dtype=torch.float64, device=dev)
    info = torch.empty(4, dtype=torch.float64, device=dev)
    Vt = torch.empty_like(V)

    def newton_iter():
        blocks.zero_()
        m.contact_hessian(ctx, hier, pairs, eps, poses, contacts, mass, 1000.0, blocks=blocks)
        m.newton_solve(ctx, pairs, blocks, mass, inertia, dt, res, x, 100, 1e-10, info)
        m._lib.check(lib.mrdem_vel_axpy(ctx.handle, 6 * n, -1.0, _p(x), _p(V), _p(Vt), None), "axpy")
        m.move_poses(ctx, poses0, Vt, dt, out=poses)
        ft.zero_()
        m.detect(ctx, hier, pairs, eps, poses, args.precision, contacts=contacts, stats=stats,
                 check=False)
        m.contact_forces(ctx, hier, pairs, eps, poses, contacts, mass, com, 1000.0,
                         force_torque=ft, energy=energy)
        m.newton_residual(ctx, vel0, Vt, ft, mass, inertia, dt, res, norms)

    m.newton_residual(ctx, vel0, V, ft, mass, inertia, dt, res, norms)
    for _ in range(args.warmup):
        newton_iter()
    torch.cuda.synchronize()
    Kn = max(K // 10, 3)
    a.record()
    for _ in range(Kn):
        newton_iter()
    b.record()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "Newton iterations")
    newton_ms = a.elapsed_time(b) / Kn
    # the same iteration captured once into a CUDA graph and replayed
    gN = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(gN, stream=side):
        newton_iter()
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(args.warmup):
        gN.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(Kn):
        gN.replay()
    b.record()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "Newton iterations (graph)")
    newton_graph_ms = a.elapsed_time(b) / Kn
    cg_it = float(info[0].item())
    # where a Newton iteration's time goes (CUDA events around each call)
    ctx.profile(True)
    for _ in range(Kn):
        newton_iter()
    torch.cuda.synchronize()
    ctx.profile(False)
    newton_parts = {k: round(v[0] / Kn, 4) for k, v in ctx.profile_read().items()}

    print(json.dumps({
        "metric": "implicit Euler step, packing: time per Picard iteration (pose update, "
                  "detection, forces, velocity update)",
        "value": round(picard_ms, 4), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": K, "warmup": args.warmup, "dtype": "f32+f64" if args.precision == "fp32" else "f64",
        "data": "synthetic", "workload": "packing",
        "config": {"workload": f"random packing of {n} bumped icospheres (subdivision 2-4, "
                               f"radius log-uniform [1, 10]), packed by "
                               + ("compression (soft-sphere energy minimisation)"
                                  if args.packing == "compress" else
                                  "random sequential addition")
                               + f", {achieved:.3f} volume fraction reached of 0.55 requested, "
                               f"dt = 1e-4",
                   "volume_fraction": round(achieved, 4),
                   "particles": n, "triangles": int(np.diff(s.tri_off).sum()), "pairs": P,
                   "contacts": contacts.n(), "precision": args.precision,
                   "launch_shapes": tuning},
        "broad_phase_ms": round(bp_ms, 4),
        "picard": {"ms_per_iteration": round(picard_ms, 4), "iterations_to_1e-6": it_p,
                   "wall_s": round(picard_s, 3),
                   "ms_per_iteration_kept_candidates": round(cached_ms, 4),
                   "kept_candidates": cand.n(), "margin_w": w},
        "multires": multires,
        "newton": {"ms_per_iteration": round(newton_ms, 4),
                   "ms_per_iteration_graph": round(newton_graph_ms, 4), "ms_parts": newton_parts,
                   "cg_iterations_last": cg_it,
                   "iterations_to_1e-6": it_n, "wall_s": round(newton_s, 3),
                   "line_search_halvings": [st["halvings"] for st in nst]},
        "agree": float((Vp - Vn).abs().max().item() / Vp.abs().max().item()),
        "prep_s": round(prep_s, 1), "packing_s": round(packing_s, 1), "clocks": clk.summary(),
    }), flush=True)
    return 0


def run_scale(args):
    """The scale workload (100 000 particles of 1 280 triangles and 100 of
    81 920 at 20 times the radius, 136 M triangles): broad phase, then per
    step the detection and forces of every candidate pair, in chunks of
    --chunk pairs per call (the work lists stay near their default size),
    enqueued without host synchronisation and timed with CUDA events.  One
    JSON line."""
    import numpy as np
    import torch

    import paper_2105_12415_gb300 as m
    from gen.icosphere import scene_scale
    from paper_2105_12415_gb300.api import _p, _stream

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    m.build()
    lib = m.load()
    t0 = time.perf_counter()
    s, achieved = scene_scale()
    n = s.n_particles
    bound = np.array([np.sqrt((s.particle(i)[0].astype(np.float64) ** 2).sum(1)).max()
                      for i in range(n)])
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx = m.Context(0)
    if args.host_trees:
        hier = m.Hierarchy.from_scene(ctx, s)
    else:
        hier = m.Hierarchy.from_scene_device(ctx, s)
    build_s = time.perf_counter() - t0
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    poses, mass, com = t(s.poses), t(s.mass), t(np.zeros((n, 3)))
    pairs, eps = m.broad_phase(ctx, poses, t(bound), t(s.radius))
    P = pairs.shape[0]
    chunks = [(a, min(a + args.chunk, P)) for a in range(0, P, args.chunk)]
    contacts = None
    stats = torch.zeros(m._lib.MRDEM_STAT_COUNT, dtype=torch.int64, device=dev)
    ft = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    n_contacts = 0
    for a, b in chunks:   # checked pass: sizes the lists and the contact buffer
        contacts, _ = m.detect(ctx, hier, pairs[a:b], eps[a:b], poses, args.precision,
                               contacts=contacts, stats=stats)
        n_contacts += contacts.n()
    import ctypes as C

    def step():
        ft.zero_()
        energy.zero_()
        for a, b in chunks:
            cs = contacts.struct()
            m._lib.check(lib.mrdem_detect(ctx.handle, hier.handle, b - a, _p(pairs[a:b]),
                                          _p(eps[a:b]), _p(poses),
                                          m.api.PRECISION[args.precision], C.byref(cs),
                                          _p(stats), _stream(None)), "detect")
            m._lib.check(lib.mrdem_contact_forces(ctx.handle, hier.handle, b - a, _p(pairs[a:b]),
                                                  _p(eps[a:b]), _p(poses), C.byref(cs), _p(mass),
                                                  _p(com), 1000.0, _p(ft), _p(energy),
                                                  _stream(None)), "forces")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "warm-up check")
    K = max(1, min(args.steps, 20))
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        a_ev.record()
        for _ in range(K):
            step()
        b_ev.record()
        torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "timed steps")
    ms = a_ev.elapsed_time(b_ev) / K
    print(json.dumps({
        "metric": "particle-pair detections/s, scale workload (detection and forces per step)",
        "value": round(P / (ms * 1e-3), 1), "unit": "pairs/s", "higher_is_better": True,
        "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
        "workload": "scale",
        "config": {"workload": f"{n - 100} particles of 1280 triangles and 100 of 81920 at 20x "
                               f"the radius, {achieved:.3f} volume fraction",
                   "particles": n, "triangles": int(np.diff(s.tri_off).sum()), "pairs": P,
                   "contacts": n_contacts, "chunk": args.chunk, "precision": args.precision},
        "prep_s": {"generate": round(gen_s, 1), "trees": round(build_s, 1),
                   "trees_where": "host" if args.host_trees else "device",
                   "trees_device_ms": None if args.host_trees else round(hier.build_ms, 1)},
        "clocks": clk.summary(),
    }), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "packing":
        return run_packing(args)
    if args.workload == "scale":
        return run_scale(args)
    import numpy as np
    import torch

    rank, world, local = _dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2105_12415_gb300 as m
    from gen import scene_c2

    if rank == 0:
        m.build()
    _barrier(world)
    m.load()

    t_prep = time.perf_counter()
    scene = scene_c2(args.pairs)
    ctx = m.Context(local)
    hier = m.Hierarchy.from_scene(ctx, scene)
    info = hier.info()
    prob = m.ContactProblem.from_scene(ctx, hier, scene, dev, precision=args.precision)
    prep_s = time.perf_counter() - t_prep

    stats = torch.zeros(m._lib.MRDEM_STAT_COUNT, dtype=torch.int64, device=dev)
    ft = torch.zeros((scene.n_particles, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    P = scene.n_pairs
    gv = torch.zeros((info["n_verts"], 3), dtype=torch.float32, device=dev)
    gp = torch.zeros((scene.n_particles, 6), dtype=torch.float64, device=dev)
    jac = torch.zeros((P, 12, 12), dtype=torch.float64, device=dev)
    lib = m.load()
    import ctypes as C
    from paper_2105_12415_gb300.api import _p, _stream

    # warm-up through the checked path (grows the work lists once if needed)
    for _ in range(max(1, args.warmup)):
        prob.detect(stats=stats)
    contacts = prob.contacts
    # launch shapes for this GPU and batch size (untimed preparation)
    tuning = None
    if args.shapes:
        kw = {k: int(v) for k, v in (kv.split("=") for kv in args.shapes.split(","))}
        ctx.set_params(**kw)
        tuning = {"chosen": kw, "given": True}
    elif not args.no_autotune:
        t_tune = time.perf_counter()
        tuning = m.autotune(ctx, hier, prob.pairs, prob.eps, prob.poses, args.precision,
                            contacts=contacts, reps=10)
        tuning["s"] = round(time.perf_counter() - t_tune, 2)
        tuning["gain"] = tuning["ms_default"] / tuning["ms_tuned"]

    side = torch.cuda.Stream()

    def step():
        s = _stream(None)
        cs = contacts.struct()
        # the accumulated outputs are zeroed first, so that detect, forces and
        # the adjoint follow each other directly in the stream
        ft.zero_()
        energy.zero_()
        gv.zero_()
        gp.zero_()
        jac.zero_()
        m._lib.check(lib.mrdem_detect(ctx.handle, hier.handle, P, _p(prob.pairs), _p(prob.eps),
                                      _p(prob.poses), m.api.PRECISION[args.precision],
                                      C.byref(cs), _p(stats), s), "detect")
        # forces and the adjoint both read the contacts: the adjoint runs on a
        # second stream beside the forces
        side.wait_stream(torch.cuda.current_stream())
        m._lib.check(lib.mrdem_contact_forces(ctx.handle, hier.handle, P, _p(prob.pairs),
                                              _p(prob.eps), _p(prob.poses), C.byref(cs),
                                              _p(prob.mass), _p(prob.com), 1000.0, _p(ft),
                                              _p(energy), s), "forces")
        m._lib.check(lib.mrdem_contact_grad(ctx.handle, hier.handle, P, _p(prob.pairs),
                                            _p(prob.eps), _p(prob.poses), C.byref(cs),
                                            _p(prob.mass), 1000.0, 1.0, _p(gv), _p(gp), _p(jac),
                                            C.c_void_p(side.cuda_stream)), "grad")
        torch.cuda.current_stream().wait_stream(side)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "warm-up check")

    # capture one step in a CUDA graph
    g = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap_stream):
        step()
    torch.cuda.current_stream().wait_stream(cap_stream)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.fill_(1)
        g.replay()
    torch.cuda.synchronize()

    # ---- timed region: graph replays, events per step, L2 flushed between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record()
            g.replay()
            ev[k][1].record()
        torch.cuda.synchronize()
    _barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms)
    m._lib.check(lib.mrdem_check(ctx.handle, None, None), "timed-region check")
    ms_max = _max_over_ranks(ms, world, dev)
    value = _whole_job_rate(args.steps, P, world, ms_max)
    st = stats.cpu().numpy()
    n_contacts = int(contacts.count.item())
    # our kernels per step: k_setup, the surrogate levels below the roots
    # (per level k_expand + k_sweep_nodes, or one k_level; or one k_levels
    # for all), k_tile, k_sweep_fine, the exact pass (FP32 form: k_cp_float,
    # 3 x k_cp_items, k_select_exact; FP64 form: k_exact64), the ordering by
    # pair (k_sort_scan, k_sort_scatter), then k_frames + k_forces and
    # k_frames + k_grad
    exact_launches = 5 if args.precision == "fp32" else 1
    levels = max(0, info["max_depth"] - 1)
    lk = int(tuning["chosen"].get("level_kernel", ctx.params.level_kernel) if tuning
             else ctx.params.level_kernel)
    level_launches = {0: 2 * levels, 1: min(levels, 1), 2: levels}[int(lk)]
    launches_per_step = 1 + level_launches + 2 + exact_launches + 2 + 4

    # ---- per-kernel timing (same steps, outside the graph, events per kernel)
    ctx.profile(True)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        step()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    fine_tests = int(st[m._lib.MRDEM_STAT_FINE_TESTS])
    fine_sweeps = int(st[m._lib.MRDEM_STAT_FINE_SWEEPS])
    sphere_tests = int(st[m._lib.MRDEM_STAT_SPHERE_TESTS])
    level_sweeps = int(st[m._lib.MRDEM_STAT_LEVEL_SWEEPS])
    tiles = int(st[m._lib.MRDEM_STAT_TILES])
    fvs = int(st[m._lib.MRDEM_STAT_FINE_SURROGATE])
    expand_tests = int(st[1:m._lib.MRDEM_STAT_LEVELS].sum())
    # every child pair that passed the sphere test got the box test: those
    # it pruned and those that went on to the sweep
    box_tests = int(st[m._lib.MRDEM_STAT_BOX_PRUNED]) + level_sweeps
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    total_prof = sum(v[0] for v in prof.values())
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                   "share": v[0] / total_prof} for k, v in prof.items()}
    # algorithmic FP32 flops per step of the culling and sweep kernels
    flops = {"k_sweep_fine": fine_tests * (FLOPS_PER_XFORM + FLOPS_PER_AXIS)
             + fine_sweeps * FLOPS_PER_SWEEP,
             "k_sweep_nodes": level_sweeps * FLOPS_PER_NODE_SWEEP,
             "k_tile": tiles * FLOPS_PER_TILE + fvs * FLOPS_PER_FINE_VS_SURR
             + sphere_tests * FLOPS_PER_SPHERE_TEST,
             "k_expand": expand_tests * FLOPS_PER_EXPAND_TEST + box_tests * FLOPS_PER_BOX_TEST}
    rl = {}
    for k, f in flops.items():
        if k in prof:
            avg_s = prof[k][0] / prof[k][1] * 1e-3
            per_launch = f / (prof[k][1] / args.steps)
            ach = per_launch / avg_s / 1e12
            rl[k] = {"achieved": ach, "frac": ach / fp32_peak, "flops_per_launch": per_launch,
                     "avg_ms": avg_s * 1e3, "ms_per_step": prof[k][0] / args.steps}
    # the headline is the finest level (Algorithm 4's tests of fine triangle
    # pairs): k_tile and k_sweep_fine, one launch each per step, taken
    # together; every modelled kernel is listed under roofline.all
    top = "k_tile+k_sweep_fine"
    fine_k = [k for k in ("k_tile", "k_sweep_fine") if k in rl]
    if fine_k:
        f_step = sum(rl[k]["flops_per_launch"] * prof[k][1] / args.steps for k in fine_k)
        ms_step = sum(rl[k]["ms_per_step"] for k in fine_k)
        ach = f_step / (ms_step * 1e-3) / 1e12
        rl[top] = {"achieved": ach, "frac": ach / fp32_peak, "flops_per_launch": f_step,
                   "avg_ms": ms_step, "ms_per_step": ms_step}
    traffic = _traffic_per_launch()
    fin = rl.get(top, {"achieved": float("nan"), "frac": float("nan"), "avg_ms": float("nan"),
                       "flops_per_launch": float("nan")})

    # ---- redundant-contact merge (Sec. 2) of the step's contact list, timed
    # on its own (not part of the step): CUDA events around each call, L2
    # flushed between calls
    merge = None
    if not args.no_merge:
        merged, members = m.merge_contacts(ctx, prob.eps, contacts)  # sizes the output
        for k in range(args.warmup):
            flush.fill_(k & 0xFF)
            m.merge_contacts(ctx, prob.eps, contacts, out=merged, members=members, check=False)
        torch.cuda.synchronize()
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.merge_calls)]
        for k in range(args.merge_calls):
            flush.fill_(k & 0xFF)
            mev[k][0].record()
            m.merge_contacts(ctx, prob.eps, contacts, out=merged, members=members, check=False)
            mev[k][1].record()
        torch.cuda.synchronize()
        m._lib.check(lib.mrdem_check(ctx.handle, None, None), "merge check")
        mms = sum(a.elapsed_time(b) for a, b in mev) / args.merge_calls
        n_out = int(merged.count.item())
        # compulsory bytes: read each contact once (pair, tri_a, tri_b, pa, pb:
        # 60 B), write each merged contact once (68 B + member count 4 B),
        # eps and two per-pair counts (16 B)
        mbytes = 60 * n_contacts + 72 * n_out + 16 * P
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        merge = {"ms_per_call": mms, "contacts_in": n_contacts, "contacts_out": n_out,
                 "launches_per_call": 7, "calls": args.merge_calls,
                 "roofline": {"bound": "hbm", "achieved": mbytes / (mms * 1e-3) / 1e9,
                              "peak": hbm, "unit": "GB/s",
                              "frac": mbytes / (mms * 1e-3) / 1e9 / hbm,
                              "bytes_per_call": mbytes, "traffic": None}}
        if rank == 0 and not args.no_baselines:
            merge["oracle"] = merge_oracle_baseline(contacts.to_numpy(sort=False),
                                                    scene.eps, members[:n_out].cpu().numpy())

    # ---- end to end through the public API (host inputs, host results)
    e2e = None
    if not args.no_e2e:
        h_poses = torch.as_tensor(scene.poses, dtype=torch.float64).pin_memory()
        h_pairs = torch.as_tensor(scene.pairs, dtype=torch.int32).pin_memory()
        h_eps = torch.as_tensor(scene.eps, dtype=torch.float64).pin_memory()
        h_ft = torch.empty((scene.n_particles, 6), dtype=torch.float64).pin_memory()
        h_gp = torch.empty((scene.n_particles, 6), dtype=torch.float64).pin_memory()
        h_e = torch.empty(1, dtype=torch.float64).pin_memory()
        h_n = torch.empty(1, dtype=torch.int64).pin_memory()
        host_in = {"poses": h_poses, "pairs": h_pairs, "eps": h_eps}
        host_out = {"ft": h_ft, "gp": h_gp, "energy": h_e, "count": h_n}
        e_ms = 0.0
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            # one public call: the inputs copied from pinned host memory,
            # detect + forces + adjoint, the results copied back, the status
            # checked with one synchronisation
            prob.step(want_jac=True, host_in=host_in, host_out=host_out)
            b.record()
            b.synchronize()
            e_ms += a.elapsed_time(b)
        e_ms = _max_over_ranks(e_ms, world, dev)
        h2d = h_poses.numel() * 8 + h_pairs.numel() * 4 + h_eps.numel() * 8
        d2h = h_ft.numel() * 8 + h_gp.numel() * 8 + 8 + 8
        e2e = {"value": _whole_job_rate(args.steps, P, world, e_ms), "unit": "particle-pair detections/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    plain = cpu = None
    if rank == 0 and not args.no_baselines:
        # plain GPU form on a sample: every 256th pair, one launch per pair
        ids = np.arange(0, P, 256)
        pairs_s = prob.pairs[torch.as_tensor(ids, device=dev)].contiguous()
        eps_s = prob.eps[torch.as_tensor(ids, device=dev)].contiguous()
        m.detect_plain_fp64(ctx, hier, pairs_s, eps_s, prob.poses)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        m.detect_plain_fp64(ctx, hier, pairs_s, eps_s, prob.poses)
        b.record()
        b.synchronize()
        pms = a.elapsed_time(b)
        plain = {"value": len(ids) / (pms * 1e-3), "unit": "particle-pair detections/s",
                 "sample": f"{len(ids)} pairs (ids = 0 mod 256), FP64 comparison-based over all "
                           f"fine triangle pairs, one launch per pair",
                 "ms": pms, "speedup_of_ours": value / world / (len(ids) / (pms * 1e-3))}
        cpu = cpu_oracle_baseline(scene, args.cpu_budget_s)
        cpu["single_thread"] = cpu_oracle_baseline(scene, min(5.0, args.cpu_budget_s / 3),
                                                   n_threads=1)
        cpu["cpu_model"] = _cpu_model()

    if rank != 0:
        return
    line = {
        "metric": "particle-pair detections/s", "value": value,
        "unit": "particle-pair detections/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "ms_per_step_median": float(statistics.median(step_ms)),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"c2-batched-{P}-pairs", "pairs": P,
                   "particles": scene.n_particles, "fine_triangles": int(info["n_tri"]),
                   "max_depth": info["max_depth"], "precision": args.precision,
                   "replicas": world, "l2": "flushed between steps (256 MiB write)",
                   "step": "detect + forces + adjoint (verts, poses, 12x12 blocks)",
                   "graph": "one CUDA graph per step", "prep_s": round(prep_s, 1),
                   "launch_shapes": tuning},
        "roofline": {"bound": "alu", "kernel": top, "achieved": fin["achieved"],
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": fin["frac"],
                     "traffic": (sum(traffic[k] for k in ("k_tile", "k_sweep_fine"))
                                 if all(k in traffic for k in ("k_tile", "k_sweep_fine"))
                                 else None),
                     "per_launch": {"flops": fin["flops_per_launch"], "avg_ms": fin["avg_ms"]},
                     "peak_note": "152 SMs x 128 FP32 lanes x 2 x max SM clock (nominal)",
                     "all": rl},
        "clocks": clk.summary(),
        "gpu_launches": launches_per_step * args.steps,
        "kernels": kernels,
        "stats": {"tests_per_level": [int(x) for x in st[0:6]],
                  "survivors_per_level": [int(x) for x in st[8:14]],
                  "leaf_tiles": int(st[16]), "sphere_tests": sphere_tests,
                  "level_sweeps": level_sweeps, "box_pruned": int(st[m._lib.MRDEM_STAT_BOX_PRUNED]),
                  "fine_vs_surrogate": int(st[23]),
                  "fine_tests": fine_tests, "fine_sweeps": fine_sweeps, "candidates": int(st[18]),
                  "unconverged": int(st[19]), "contacts": n_contacts, "fp64_refinements": int(st[21]),
                  "fp64_items": [int(st[m._lib.MRDEM_STAT_ITEMS_PT]), int(st[m._lib.MRDEM_STAT_ITEMS_EE])],
                  "fine_tests_per_s": fine_tests * args.steps * world / (ms_max * 1e-3),
                  "level_tests_per_s": [float(x) * args.steps * world / (ms_max * 1e-3)
                                        for x in st[0:6]],
                  "brute_force_pairs_per_s": float(
                      (np.diff(scene.tri_off)[scene.pairs[:, 0]] *
                       np.diff(scene.tri_off)[scene.pairs[:, 1]]).sum()) * args.steps * world / (ms_max * 1e-3)},
        "e2e": e2e,
        "merge": merge,
        "plain_fp64_gpu": plain,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
