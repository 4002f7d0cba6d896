"""Throughput of the fused cascaded D2Q9 update on one GB300 (and N replicas).

Workload: decaying Taylor-Green vortex, 4096 x 4096 periodic nodes, diffusive
scaling U0 = 0.04*64/4096, shear omega = 1.6, other rates 1 (the largest
single-GPU Taylor-Green case).  One step = one lattice update of every node =
one launch of the fused stream-and-collide kernel.  The populations (4096^2 x
9 x 4 B = 604 MB in FP32) are far larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, one single-threaded process per host core, each on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 cascaded MLUPS & % HBM roofline, FP16-store vs FP32 at stated error"
N_DEFAULT = 4096
OMEGA = 1.6
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_cascaded_tg4096.md")


def parse():
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--store", choices=["f32", "f16", "bf16", "f64"], default="f32")
    p.add_argument("--no-extras", action="store_true", help="skip the sibling / precision comparison runs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--part", choices=["all", "adjoint", "batch", "cost", "steps"], default="all",
                   help="adjoint / batch: run only that measurement and print it; cost: four single-launch "
                        "steps of each collision model in FP32 and FP64 storage on --n^2; steps: --steps "
                        "steps of the --store lattice in kernel --variant (for profiling)")
    p.add_argument("--variant", type=int, default=-1, help="kernel variant for --part steps (-1: the default)")
    p.add_argument("--adjoint-n", type=int, default=512)
    p.add_argument("--adjoint-steps", type=int, default=2000)
    p.add_argument("--batch-steps", type=int, default=200)
    p.add_argument("--batch-domains", type=int, default=96, help="first N domains of the ensemble (--part batch)")
    return p.parse_args()


def omegas():
    return (1.0, OMEGA, OMEGA, 1.0, 1.0, 1.0)


STEP_KERNEL_SOURCES = ("include/lbm.h", "paper_1202_6351_gb300/csrc/lbm_device.cuh",
                       "paper_1202_6351_gb300/csrc/lbm_fused.cuh", "paper_1202_6351_gb300/csrc/lbm_async.cuh",
                       "paper_1202_6351_gb300/csrc/lbm_internal.h", "paper_1202_6351_gb300/csrc/lbm_pair.cuh",
                       "paper_1202_6351_gb300/csrc/lbm_vec.cuh",
                       "paper_1202_6351_gb300/csrc/lbm_step_impl.cuh", "paper_1202_6351_gb300/csrc/lbm_step_f64.cu",
                       "paper_1202_6351_gb300/csrc/lbm_step_f32.cu", "paper_1202_6351_gb300/csrc/lbm_step_bf16.cu",
                       "paper_1202_6351_gb300/csrc/lbm_step_f16.cu")


KERNEL_NAMES = {2: "step_kernel_vec (one step per launch, four nodes per thread)",
                3: "fused2_kernel (two steps per launch)"}


def strip_comments(text: str) -> str:
    """C/C++/CUDA source without its comments and with runs of white space
    collapsed, so that an edit of comments or layout alone leaves the digest
    unchanged (the sources hold no string literal containing a comment marker)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_digest():
    """Digest of the code (comments stripped) of the sources that define the
    step kernel, used to tell whether a committed ncu summary still describes
    the kernel being timed."""
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            h.update(f.encode() + b"\0" + strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(store_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current sources; else None."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"source digest:\s*`?([0-9a-f]+)", text)
    if not m or m.group(1) != source_digest():
        return None
    m = re.search(rf"traffic_bytes_per_launch\[{store_name}\]:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks sampler

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.samples = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def wait_first(self, timeout=5.0):
        t0 = time.time()
        while self.proc and not self.samples and time.time() - t0 < timeout:
            time.sleep(0.05)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [p for (t, p) in self.samples if t0 <= t <= t1]
        use = inside or [p for (_, p) in self.samples]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(p[1]) for p in use if num(p[1]) is not None]
        smax = [num(p[2]) for p in use if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in use for k in range(4) if p[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside), "power_w_max": max(num(p[3]) or 0 for p in use)}


# ---------------------------------------------------------------- oracle timing (CPU)

def _oracle_lattice(kind, side):
    """An oracle lattice of one of the timed sample workloads: the Taylor-Green
    start of the bench workload (diffusive scaling) or the lid-driven cavity at
    Re 1000 from rest (U = 0.1, nu = U (side - 1) / Re)."""
    import oracle as O
    from paper_1202_6351_gb300 import workloads

    if kind == "cavity":
        U = 0.1
        om = 1.0 / (3.0 * U * (side - 1) / 1000.0 + 0.5)
        return O.Lattice(side, side, (1.0, om, om, 1.0, 1.0, 1.0), edges=(1, 1, 1, 2), wall_u=(0, 0, 0, U)).init()
    rho, u = workloads.taylor_green_init(side, workloads.diffusive_u0(side))
    return O.Lattice(side, side, omegas()).init(rho, u)


def time_oracle(n_side, steps, max_seconds=None, kind="taylor_green"):
    """Run the FP64 oracle on an n_side^2 sample (kind: "taylor_green" or
    "cavity"); returns (lattice updates per second, steps done, seconds)."""
    L = _oracle_lattice(kind, n_side)
    done, t0 = 0, time.perf_counter()
    chunk = max(1, min(steps, 10, int(2e6 // (n_side * n_side)) or 1))
    while done < steps:
        k = min(chunk, steps - done)
        L.run(k)
        done += k
        if max_seconds is not None and time.perf_counter() - t0 >= max_seconds:
            break
    dt = time.perf_counter() - t0
    return n_side * n_side * done / dt, done, dt


def host_cores():
    """Host cores this process may run on."""
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _oracle_worker(job):
    """One host process: the oracle on its own sample (warm-up steps untimed,
    then `steps` steps or `seconds`, whichever ends first)."""
    side, warmup, steps, seconds, kind = job
    if warmup:
        time_oracle(side, warmup, kind=kind)
    return time_oracle(side, steps, max_seconds=seconds, kind=kind)


def time_oracle_all_cores(side, warmup, steps, seconds=None, kind="taylor_green", pool=None):
    """The oracle as it stands, one single-threaded process per host core, each on
    its own side^2 sample at the same time (processes started with spawn: this
    process may already hold a CUDA context).  Returns (cores, [(ups, done, dt)])."""
    import multiprocessing as mp

    cores = host_cores()
    jobs = [(side, warmup, steps, seconds, kind)] * cores
    if pool is not None:
        return cores, pool.map(_oracle_worker, jobs)
    with mp.get_context("spawn").Pool(cores) as p:
        res = p.map(_oracle_worker, jobs)
    return cores, res


# The oracle's sample workloads beside the GPU numbers: Taylor-Green at the
# sides of the Taylor-Green configuration it can run, and the 257^2 cavity.
CPU_SAMPLES = (("taylor_green", 64), ("taylor_green", 128), ("taylor_green", 256), ("taylor_green", 1024),
               ("cavity", 257))


def cpu_baseline_line(seconds_per_sample=2.0):
    """The oracle as it stands on the host cores: each sample workload timed on
    one core alone and as one process per core at once (the summed rate).
    `value` is the all-core Taylor-Green 256^2 rate."""
    import multiprocessing as mp

    by_size = []
    single = {}
    for kind, side in CPU_SAMPLES:
        ups, done, dt = time_oracle(side, 10 ** 9, max_seconds=seconds_per_sample, kind=kind)
        single[kind, side] = (ups, done)
    cores = host_cores()
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(16, 1, 1, None, "taylor_green")] * cores)  # start every worker first
        for kind, side in CPU_SAMPLES:
            _, res = time_oracle_all_cores(side, 0, 10 ** 9, seconds_per_sample, kind=kind, pool=pool)
            ups1, done1 = single[kind, side]
            by_size.append({"workload": f"{kind}_{side}x{side}", "single_core_mlups": round(ups1 / 1e6, 3),
                            "all_cores_mlups": round(sum(r[0] for r in res) / 1e6, 3),
                            "steps_single": done1, "steps_per_process_min": min(r[1] for r in res)})
    main = next(b for b in by_size if b["workload"] == "taylor_green_256x256")
    return {"value": main["all_cores_mlups"], "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, Taylor-Green 256x256 cascaded, one single-threaded process per host core "
                      f"({cores}), each for about {seconds_per_sample:.0f} s; by_size lists every sample workload "
                      f"on one core alone and on all cores",
            "by_size": by_size}


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, dist=None, device="cuda") -> float:
    """The largest of one float per rank (the timed interval of the slowest rank)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launch_count(t0, steps, two_step):
    """Kernel launches of `steps` steps from step t0 (lbm_step without graphs):
    with two fused steps per launch, a pair from every even step with two
    steps left, single launches otherwise."""
    n, t, end = 0, t0, t0 + steps
    while t < end:
        t += 2 if (two_step and t % 2 == 0 and end - t >= 2) else 1
        n += 1
    return n


MIN_PASSES = 5
MIN_TIMED_SECONDS = 2.0


def passes_for(first_pass_seconds: float, dist=None) -> int:
    """Timed passes of K steps: at least MIN_PASSES and enough to span
    MIN_TIMED_SECONDS, agreed over ranks (the largest count) so that every
    rank runs the same number of barriers."""
    p = max(MIN_PASSES, int(math.ceil(MIN_TIMED_SECONDS / max(first_pass_seconds, 1e-6))))
    p = min(p, 100000)
    if dist is None:
        return p
    import torch

    t = torch.tensor([p], dtype=torch.int64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return int(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, seconds: float, world: int) -> float:
    """Lattice updates of all ranks (weak scaling: each rank its own replica) per second / 1e6."""
    return world * nodes_per_rank * steps / seconds / 1e6


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # each step: one oracle lattice update of a bounded Taylor-Green sample, sized
    # so that warmup + steps take about a minute at ~10 MLUPS
    budget_updates = 60.0 * 10e6
    side = int(math.sqrt(budget_updates / max(1, args.steps + args.warmup)))
    side = max(16, min(256, side // 16 * 16))
    cores, res = time_oracle_all_cores(side, args.warmup, args.steps)
    dt = max(r[2] for r in res)  # every process runs all its steps; the slowest one ends the run
    v = cores * side * side * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / max(args.steps, 1), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.n, args.store),
        "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 C oracle, one single-threaded process per host core, each on its own "
                                   f"Taylor-Green {side}x{side} sample ({cores} x {side}x{side} nodes per step), "
                                   f"{args.steps} steps after {args.warmup} warm-up"},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(n, store_name, world=1):
    """The `config` object of the bench line (both arms)."""
    bpu = {"f64": 144, "f32": 72, "bf16": 36, "f16": 36}[store_name]
    return {"workload": f"taylor_green_{n}x{n}_cascaded_{store_name}_store", "nodes": n * n,
            "omega_shear": OMEGA, "u0": 0.04 * 64 / n, "model": "cascaded", "store": store_name,
            "l2_flush": f"none: populations {bpu // 2 * n * n / 1e6:.0f} MB > 129 MB L2",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_1202_6351_gb300 import lbm, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stores = {"f32": lbm.F32, "f16": lbm.F16DEV, "bf16": lbm.BF16DEV, "f64": lbm.F64}
    store = stores[args.store]
    n = args.n
    nodes = n * n
    u0 = workloads.diffusive_u0(n)
    rho_h, u_h = workloads.taylor_green_init(n, u0)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def make(model=lbm.CASCADED, st=store):
        L = lbm.Lattice(n, n, omegas(), model=model, store=st, stream=sp)
        L.init(rho_h, u_h)
        return L

    def timed(L, steps, sampler=None):
        """Warm-up already done; returns (seconds, t_wall0, t_wall1)."""
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(stream)
        L.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        barrier()
        return e0.elapsed_time(e1) / 1e3, w0, w1

    peak, peak_kind = measured_peaks()
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None

    # ---- the timed region: passes of exactly K steps of the cascaded kernel,
    # repeated (the same count on every rank) until they span at least
    # MIN_TIMED_SECONDS so that the clock sampler sees the load; the median pass counts
    L = make()
    # the library's per-lattice autotuner picks the kernel variant and CTA shape
    # (on this workload: two fused steps per launch, variant 3, when it is fastest)
    tuned_ms = L.tune(50)
    variant = L.info()["variant"]
    sampler = ClockSampler(uuid) if rank == 0 else None
    if sampler:
        sampler.wait_first()
    # W warm-up steps, one more if W is odd and the kernel takes steps in pairs:
    # a pair of steps starts at an even step, so a pass that started at an odd
    # step would time two single-step launches at its ends
    warmup_run = args.warmup + (1 if variant == 3 and args.warmup % 2 else 0)
    L.step(warmup_run)
    first, w0, _ = timed(L, args.steps)
    passes = passes_for(first, dist)
    pass_secs = [first] + [timed(L, args.steps)[0] for _ in range(passes - 1)]
    w1 = time.time()
    if sampler:
        time.sleep(0.3)
        sampler.stop()
    secs = statistics.median(pass_secs)
    secs_max = max_over_ranks(secs, dist, "cuda")
    value = whole_job_mlups(nodes, args.steps, secs_max, world)
    bpu = lbm.lbm_bytes_per_update(store)
    two_step = variant == 3
    step_s = secs / args.steps
    achieved = bpu * nodes / step_s / 1e9  # algorithmic bytes per update x updates per second
    store_name = lbm.STORE_NAMES[store]
    traffic = profiled_traffic(store_name + ("_two_step" if two_step else ""))
    updates_per_launch = 2 if two_step else 1
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth", "bytes_per_update": bpu,
                "algorithmic_bytes_per_launch": bpu * nodes * updates_per_launch,
                "kernel": KERNEL_NAMES.get(variant, "step_kernel (one step per launch)")}
    if two_step:
        # one read and one write of the state per two steps: the design's own
        # DRAM bytes per update are half of the per-step algorithmic bytes
        roofline["design_bytes_per_update"] = bpu // 2
        roofline["frac_of_design_bytes"] = round(achieved / 2 / peak, 4)
    launches = launch_count(warmup_run, args.steps, two_step)
    L.close()

    # ---- end to end through the C ABI with pinned host buffers (every rank, right
    # after the timed region so that it runs under the same conditions each time)
    esampler = ClockSampler(uuid) if rank == 0 else None
    if esampler:
        esampler.wait_first()
    e0w = time.time()
    e2e = run_e2e(args, lbm, torch, np, n, rho_h, u_h, sp, nodes, barrier,
                  lambda v: max_over_ranks(v, dist, "cuda"), world)
    e1w = time.time()
    if esampler:
        time.sleep(0.3)
        esampler.stop()
        e2e["clocks"] = esampler.summary(e0w, e1w)  # SM clocks while the end-to-end sequences ran

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(args, make, timed, lbm, nodes, peak, np)
        extras["one_decay_time_1024"] = run_decay_extras(lbm, np, sp, headline=extras)
        extras["batch"] = run_batch_extras(lbm, torch, np, peak, sp)
        extras["cavity_16384_f16_re5000"] = run_cavity_extras(lbm, torch, peak, sp)
        extras["d3q27"] = run_d3q27_extras(lbm, torch, peak, sp)
        extras["adjoint"] = run_adjoint_extras(lbm, torch, np, sp, peak=peak)
        extras["adjoint_2048"] = run_adjoint_extras(lbm, torch, np, sp, n=2048, steps=2000, peak=peak)

    if rank == 0:
        clocks = sampler.summary(w0, w1) if sampler else None
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * secs_max / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32" if store != lbm.F64 else "f64",
            "data": "synthetic",
            "config": workload_config(n, store_name, world),
            "roofline": roofline,
            "gpu_launches": launches,
            "timing": {"passes": len(pass_secs), "steps_per_pass": args.steps,
                       "pass_ms": {"min": round(1e3 * min(pass_secs), 4), "median": round(1e3 * secs, 4),
                                   "max": round(1e3 * max(pass_secs), 4)},
                       "reported": "median pass of K steps (max over ranks); every pass is K steps bracketed by "
                                   "barrier + synchronize, timed with CUDA events on the launching stream",
                       "timed_window_s": round(w1 - w0, 3), "gpu_launches_all_passes": launches * len(pass_secs),
                       "kernel_variant": variant, "tuned_ms_per_step": round(tuned_ms[variant], 5),
                       "warmup_steps_run": warmup_run},
            "clocks": clocks,
            "e2e": e2e,
            "extras": extras,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_line()
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_extras(args, make, timed, lbm, nodes, peak, np):
    """Same workload with the other storage kinds and the sibling collisions
    (separate timed regions, not part of `value`), plus the stated velocity
    error of each storage kind against the FP64 run of the same steps."""
    steps = max(200, min(args.steps, 2000))
    out = {"steps": steps}
    ref = make(lbm.CASCADED, lbm.F64)
    ref.step(10)
    s64, _, _ = timed(ref, steps)
    _, u64 = ref.macros()
    ref.close()
    out["cascaded_f64"] = {"mlups": round(nodes * steps / s64 / 1e6, 1),
                           "frac": round(lbm.lbm_bytes_per_update(lbm.F64) * nodes * steps / s64 / 1e9 / peak, 4)}
    runs = (("f32", lbm.F32, lbm.ROUND_NEAREST), ("f16", lbm.F16DEV, lbm.ROUND_NEAREST),
            ("bf16", lbm.BF16DEV, lbm.ROUND_NEAREST), ("f16_stochastic", lbm.F16DEV, lbm.ROUND_STOCHASTIC),
            ("bf16_stochastic", lbm.BF16DEV, lbm.ROUND_STOCHASTIC))
    for name, st, rounding in runs:
        L = make(lbm.CASCADED, st)
        if rounding == lbm.ROUND_STOCHASTIC:
            L.set_rounding(rounding, 2026)
        L.tune(50)  # each storage kind on the kernel variant the tuner picks for it
        variant = L.info()["variant"]
        L.step(10)
        s, _, _ = timed(L, steps)
        _, u = L.macros()
        L.close()
        err = float(np.sqrt(((u - u64) ** 2).sum() / (u64 ** 2).sum()))
        out[f"cascaded_{name}"] = {
            "mlups": round(nodes * steps / s / 1e6, 1),
            "frac": round(lbm.lbm_bytes_per_update(st) * nodes * steps / s / 1e9 / peak, 4),
            "rel_l2_velocity_error_vs_f64": err, "after_steps": steps + 10, "variant": variant}
    # the per-lattice tuner's timings of the kernel variants on this workload
    names = ("one_node_per_thread_mlups", "two_rows_packed_fp32x2_mlups", "four_nodes_64bit_mlups",
             "two_steps_per_launch_tma_mlups")
    tuned = {}
    for name, st in (("f32", lbm.F32), ("f16", lbm.F16DEV), ("bf16", lbm.BF16DEV)):
        L = make(lbm.CASCADED, st)
        ms = L.tune(100)
        L.close()
        tuned[name] = {k: round(nodes / m / 1e3, 1) for k, m in zip(names, ms) if m > 0}
    out["kernel_variants"] = tuned
    # the three collisions in the same kernel (one node per thread, one step per launch)
    for name, model in (("cascaded", lbm.CASCADED), ("bgk", lbm.BGK), ("rawmrt", lbm.RAWMRT)):
        L = make(model, lbm.F32)
        L.set_variant(0)
        L.step(10)
        s, _, _ = timed(L, steps)
        L.close()
        out[f"{name}_f32_one_step"] = {"mlups": round(nodes * steps / s / 1e6, 1)}
    out["cost_cascaded_over_rawmrt_f32"] = round(
        out["rawmrt_f32_one_step"]["mlups"] / out["cascaded_f32_one_step"]["mlups"] - 1, 4)
    # FP64 storage and arithmetic: GB300's FP64 pipe is narrow, so these runs are
    # bound by arithmetic and show the cascaded collision's extra work
    f64_steps = max(20, steps // 10)
    for name, model in (("bgk", lbm.BGK), ("rawmrt", lbm.RAWMRT)):
        L = make(model, lbm.F64)
        L.step(4)
        s, _, _ = timed(L, f64_steps)
        L.close()
        out[f"{name}_f64"] = {"mlups": round(nodes * f64_steps / s / 1e6, 1)}
    out["cost_cascaded_over_rawmrt_f64"] = round(out["rawmrt_f64"]["mlups"] / out["cascaded_f64"]["mlups"] - 1, 4)
    out["cost_cascaded_over_bgk_f64"] = round(out["bgk_f64"]["mlups"] / out["cascaded_f64"]["mlups"] - 1, 4)
    out["cost_note"] = ("paper (Sec. V): cascaded about 11.6 % slower than raw MRT, CPU, hardware not stated; "
                        "FP32 storage is HBM-bound (the extra arithmetic hides behind memory), FP64 is FP64-ALU-bound")
    return out


def run_decay_extras(lbm, np, sp, n=1024, headline=None):
    """The stated error of each storage kind over the configuration's own
    horizon: Taylor-Green on n^2 (diffusive scaling) run to one decay time
    T = 1 / (2 nu k^2) (Sec. III-B; 318,729 steps at n = 1024) and compared with
    the analytic decay (relative L2 velocity error and fitted amplitude), for
    FP32 storage and for the 16-bit stores with round to nearest and with
    stochastic rounding.  `headline` holds the 4096^2 MLUPS of each storage kind
    and rounding mode (run_extras), so that the FP16 / FP32 comparison is made at
    matched accuracy."""
    from paper_1202_6351_gb300 import workloads

    nu = (1.0 / OMEGA - 0.5) / 3.0
    u0 = workloads.diffusive_u0(n)
    T = workloads.taylor_green_decay_steps(n, nu)
    rho, u = workloads.taylor_green_init(n, u0)
    ua = workloads.taylor_green_velocity(n, u0, nu, T)
    out = {"n": n, "steps": T, "reference": "analytic Taylor-Green decay (Sec. III-B)"}
    runs = (("f32", lbm.F32, lbm.ROUND_NEAREST), ("f16_nearest", lbm.F16DEV, lbm.ROUND_NEAREST),
            ("f16_stochastic", lbm.F16DEV, lbm.ROUND_STOCHASTIC), ("bf16_nearest", lbm.BF16DEV, lbm.ROUND_NEAREST),
            ("bf16_stochastic", lbm.BF16DEV, lbm.ROUND_STOCHASTIC))
    for name, st, rounding in runs:
        t0 = time.perf_counter()
        with lbm.Lattice(n, n, omegas(), store=st, stream=sp) as L:
            if rounding == lbm.ROUND_STOCHASTIC:
                L.set_rounding(rounding, 2026)
            L.init(rho, u).step(T)
            _, ug = L.macros()
        dt = time.perf_counter() - t0
        err = float(np.sqrt(((ug - ua) ** 2).sum() / (ua ** 2).sum()))
        amp = float((ug * ua).sum() / (ua * ua).sum())
        out[name] = {"rel_l2_velocity_error": err, "amplitude": round(amp, 6), "seconds": round(dt, 2)}
    if headline:
        f32 = headline["cascaded_f32"]["mlups"]
        f16 = headline["cascaded_f16_stochastic"]["mlups"]
        out["fp16_vs_fp32"] = {
            "rounding": "stochastic (the mode whose error holds to one decay time; round to nearest drifts)",
            "f16_mlups_4096": f16, "f32_mlups_4096": f32, "speedup": round(f16 / f32, 3),
            "f16_error_at_one_decay_time": out["f16_stochastic"]["rel_l2_velocity_error"],
            "f32_error_at_one_decay_time": out["f32"]["rel_l2_velocity_error"],
            "f16_nearest_mlups_4096": headline["cascaded_f16"]["mlups"],
            "f16_nearest_error_at_one_decay_time": out["f16_nearest"]["rel_l2_velocity_error"]}
    return out


def run_d3q27_extras(lbm, torch, peak, sp, n=256, steps=100):
    """The D3Q27 central-moment lattice (the method carried to 3-D): the 3-D
    Taylor-Green vortex on n^3 periodic nodes in FP32 storage, one launch per
    step; MLUPS and the fraction of the copy bandwidth at 216 B per update
    (27 loads and 27 stores of 4 bytes); the same in FP16 storage (108 B)."""
    from paper_1202_6351_gb300 import workloads

    rho, u = workloads.taylor_green_3d_init(n, 0.04 * 64 / n)
    stream = torch.cuda.current_stream()
    out = {}
    for name, st in (("f32", lbm.F32), ("f16", lbm.F16DEV)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with lbm.Lattice3(n, n, n, (1.0, OMEGA, 1.0, 1.0, 1.0, 1.0), store=st, stream=sp) as L:
            L.init(rho, u).step(4)
            torch.cuda.synchronize()
            e0.record(stream)
            L.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
        bpu = lbm.load_library().lbm3_bytes_per_update(st)
        entry = {"workload": f"taylor_green_3d_{n}^3_d3q27_{name}", "steps": steps,
                 "mlups": round(n ** 3 * steps / t / 1e6, 1), "frac": round(bpu * n ** 3 * steps / t / 1e9 / peak, 4),
                 "bytes_per_update": bpu, "state_gb": round(bpu / 2 * n ** 3 / 1e9, 2)}
        if name == "f32":
            out.update(entry)
        else:
            out["f16"] = entry
    return out


def run_batch_extras(lbm, torch, np, peak, sp, steps=200, count=96):
    """Batched ensemble: 96 domains (sides log-uniform in [64, 2048], half
    lid-driven cavities at Re in [100, 5000], half Taylor-Green, FP32 / FP16
    storage), advanced together in the configuration the batch tuner keeps (one
    launch per step over all tiles, or one launch per two steps with a kernel
    per class of lattice) under CUDA graphs of 100 steps, against one lbm_step
    launch per domain per step."""
    from paper_1202_6351_gb300 import workloads

    doms = workloads.batch_domains()[:count]  # fewer domains only for profiling captures
    Ls, nodes, nbytes = [], 0, 0
    for i, d in enumerate(doms):
        n = d["side"]
        st = lbm.F32 if d["store"] == "f32" else lbm.F16DEV
        if d["kind"] == "cavity":
            U = 0.1
            om = 1.0 / (3.0 * U * (n - 1) / d["re"] + 0.5)
            L = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=(1, 1, 1, 2), wall_u=(0, 0, 0, U),
                            store=st, stream=sp)
            L.init()
        else:
            L = lbm.Lattice(n, n, omegas(), store=st, stream=sp)
            rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
            L.init(rho, u)
        Ls.append(L)
        nodes += n * n
        nbytes += n * n * lbm.lbm_bytes_per_update(st)
    stream = torch.cuda.current_stream()
    # per-domain launches, each lattice in its own tuned kernel variant and CTA shape
    for L in Ls:
        L.tune(10)
        L.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for L in Ls:
            L.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sep = e0.elapsed_time(e1) / 1e3
    # all lattices in one batch, graphs of 100 steps, autotuned
    B = lbm.Batch(Ls)
    tuned_ms = B.tune(5)
    info = B.info()
    bstream = torch.cuda.ExternalStream(info["stream"])
    B.step(100)
    B.sync()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(bstream)
    B.step(steps)
    f1.record(bstream)
    B.sync()
    torch.cuda.synchronize()
    t_bat = f0.elapsed_time(f1) / 1e3
    B.close()
    for L in Ls:
        L.close()
    out = {
        "domains": len(doms), "nodes": nodes, "steps": steps,
        "per_domain_launches": {"mlups": round(nodes * steps / t_sep / 1e6, 1),
                                "frac": round(nbytes * steps / t_sep / 1e9 / peak, 4), "launches": steps * len(doms)},
        "batched": {"mlups": round(nodes * steps / t_bat / 1e6, 1),
                    "frac": round(nbytes * steps / t_bat / 1e9 / peak, 4), "launches": steps,
                    "graph_steps": 100, "tuned": {k: v for k, v in info.items() if k != "stream"},
                    "tuned_ms_per_step": round(tuned_ms, 4)},
        "speedup_batched_over_per_domain": round(t_sep / t_bat, 3),
    }
    return out


def run_cavity_extras(lbm, torch, peak, sp):
    """The single-domain roofline point: one 16384^2 FP16-storage cavity at Re 5000."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 16384
    U, re = 0.1, 5000.0
    om = 1.0 / (3.0 * U * (n - 1) / re + 0.5)
    L = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=(1, 1, 1, 2), wall_u=(0, 0, 0, U),
                    store=lbm.F16DEV, stream=sp)
    L.init()
    L.step(4)
    torch.cuda.synchronize()
    k = 50
    e0.record(stream)
    L.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    L.close()
    return {"mlups": round(n * n * k / t / 1e6, 1), "frac": round(36 * n * n * k / t / 1e9 / peak, 4), "steps": k,
            "state_gb": round(9 * 2 * n * n / 1e9, 2)}


def adjoint_bytes_per_run(n, steps, every):
    """Algorithmic DRAM bytes of one lbm_adjoint_run on an n^2 FP32 lattice with
    a per-node force field: the forward pass (steps launches of 72 B + 8 B of
    force per node), the recomputation of each checkpoint segment (every step of
    a segment but its first, same bytes) and the reverse steps (9 lambda read,
    9 lambda written, 9 f read: 108 B, the segment force gradient read and
    written in FP32: 16 B, the force: 8 B; 132 B per node)."""
    nck = (steps + every - 1) // every
    return n * n * (80 * steps + 80 * (steps - nck) + 132 * steps)


def run_adjoint_extras(lbm, torch, np, sp, n=512, steps=2000, peak=None):
    """The adjoint configuration: periodic n^2 (512^2 in the configuration), 16
    random divergence-free Fourier modes (amplitude 0.02), `steps` FP32 steps,
    checkpoints every 100, loss against the analytic Taylor-Green field at
    t = steps.  The whole run (forward, recomputation, reverse) is timed with
    CUDA events on the lattice's stream; `frac` puts its algorithmic bytes
    (adjoint_bytes_per_run) against the peak copy bandwidth."""
    import math

    from paper_1202_6351_gb300 import workloads

    every = min(100, steps)
    u0 = torch.from_numpy(workloads.fourier_modes_field(20261202, n, modes=16, amp=0.02, kmax=8)).cuda()
    nu = (1.0 / OMEGA - 0.5) / 3.0
    k = 2 * math.pi / n
    x = torch.arange(n, dtype=torch.float64, device="cuda")
    Y, X = torch.meshgrid(x, x, indexing="ij")
    dec = math.exp(-2 * k * k * nu * steps)
    U0 = 0.04 * 64 / n
    target = torch.stack([-U0 * torch.cos(k * X) * torch.sin(k * Y) * dec, U0 * torch.sin(k * X) * torch.cos(k * Y) * dec])
    stream = torch.cuda.ExternalStream(sp)
    with lbm.Lattice(n, n, omegas(), store=lbm.F32, stream=sp) as L:
        L.set_force_field(torch.zeros((2, n, n), dtype=torch.float64, device="cuda"))
        L.adjoint_run(50, 10, u0, target)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss, gu, gf, gom = L.adjoint_run(steps, every, u0, target)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
    out = {"config": f"periodic {n}x{n}, {steps} FP32 steps, checkpoint every {every}", "seconds": round(dt, 4),
           "loss": loss, "d_loss_d_omega_shear": float(gom[1] + gom[2]),
           "gradient_mlups": round(n * n * steps / dt / 1e6, 1),
           "gradient_mlups_note": "node-steps of the differentiated run per second (forward + recompute + reverse)"}
    if peak:
        b = adjoint_bytes_per_run(n, steps, every)
        out["roofline"] = {"bound": "hbm", "algorithmic_bytes": b, "achieved_gbs": round(b / dt / 1e9, 1),
                           "peak": peak, "frac": round(b / dt / 1e9 / peak, 4),
                           "state_mb": round(36 * n * n / 1e6, 1)}
    return out


def run_e2e(args, lbm, torch, np, n, rho_h, u_h, sp, nodes, barrier, max_ranks, world):
    """End to end through the public API with host buffers: each cycle uploads
    (rho, u) from pinned host memory, initialises, runs 100 steps and reads
    (rho, u) back into pinned host memory.

    blocking:  lbm_init(host) + lbm_step(100) + lbm_macros(host), each call
               synchronous (mapped pinned buffers are read and written by the
               kernels in place).
    pipelined (the reported value): the same work with the device-side calls
               (lbm_init_device, lbm_step, lbm_macros_device) on the lattice's
               stream and the host copies on two copy streams, double-buffered,
               so that the upload of cycle k+1 and the download of cycle k-1
               overlap the steps of cycle k.  Every copy is inside the timed
               region."""
    inner = 100
    iters = 12  # about 0.25 s of steps: long enough that the pipeline's fill and drain do not dominate
    rho_p = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    u_p = torch.empty((2, n, n), dtype=torch.float64, pin_memory=True)
    rho_p.numpy()[...] = rho_h
    u_p.numpy()[...] = u_h
    out_r = [torch.empty((n, n), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    out_u = [torch.empty((2, n, n), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    lib = lbm.load_library()

    # ---- blocking sequence
    L = lbm.Lattice(n, n, omegas(), store=lbm.F32, stream=sp)
    L.tune(20)

    def job():
        lbm._check(lib.lbm_init(L.h, rho_p.data_ptr(), u_p.data_ptr()))
        lbm.lbm_step(L.h, inner)
        lbm._check(lib.lbm_macros(L.h, out_r[0].data_ptr(), out_u[0].data_ptr()))

    job()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(iters):
        job()
    torch.cuda.synchronize()
    dt_block = max_ranks(time.perf_counter() - t0)
    L.close()
    ref_u = out_u[0].numpy().copy()
    assert np.isfinite(ref_u).all()

    # ---- pipelined sequence
    comp, cin, cout = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    L = lbm.Lattice(n, n, omegas(), store=lbm.F32, stream=comp.cuda_stream)
    L.tune(20)
    d_in = [(torch.empty((n, n), dtype=torch.float64, device="cuda"),
             torch.empty((2, n, n), dtype=torch.float64, device="cuda")) for _ in range(2)]
    d_out = [(torch.empty((n, n), dtype=torch.float64, device="cuda"),
              torch.empty((2, n, n), dtype=torch.float64, device="cuda")) for _ in range(2)]
    in_ready = [torch.cuda.Event() for _ in range(2)]
    in_free = [torch.cuda.Event() for _ in range(2)]
    out_ready = [torch.cuda.Event() for _ in range(2)]
    out_free = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    for b in range(2):
        for ev, st in ((in_free[b], comp), (out_free[b], cout)):
            ev.record(st)

    def cycle(k):
        b = k & 1
        with torch.cuda.stream(cin):
            cin.wait_event(in_free[b])
            d_in[b][0].copy_(rho_p, non_blocking=True)
            d_in[b][1].copy_(u_p, non_blocking=True)
            in_ready[b].record(cin)
        comp.wait_event(in_ready[b])
        L.init_device(d_in[b][0], d_in[b][1])
        in_free[b].record(comp)
        L.step(inner)
        comp.wait_event(out_free[b])
        L.macros_device(d_out[b][0], d_out[b][1])
        out_ready[b].record(comp)
        with torch.cuda.stream(cout):
            cout.wait_event(out_ready[b])
            out_r[b].copy_(d_out[b][0], non_blocking=True)
            out_u[b].copy_(d_out[b][1], non_blocking=True)
            out_free[b].record(cout)

    for k in range(2):  # warm-up: graph capture, copy engines, caching allocator
        cycle(k)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(iters):
        cycle(k)
    torch.cuda.synchronize()
    dt_pipe = max_ranks(time.perf_counter() - t0)
    L.close()
    # every cycle computes the same fields: the pipelined result must equal the blocking one
    assert np.array_equal(out_u[(iters - 1) & 1].numpy(), ref_u)
    return {"value": round(world * nodes * inner * iters / dt_pipe / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": 3 * 8 * nodes // inner, "d2h_bytes_per_step": 3 * 8 * nodes // inner,
            "steps_per_transfer": inner, "cycles": iters,
            "sequence": "pipelined: H2D of (rho,u) from pinned host on a copy stream, lbm_init_device + "
                        "lbm_step(100) + lbm_macros_device on the lattice stream, D2H of (rho,u) to pinned host "
                        "on a second copy stream; double-buffered, all copies inside the timed region",
            "blocking_value": round(world * nodes * inner * iters / dt_block / 1e6, 1),
            "blocking_sequence": "lbm_init(pinned host rho,u) + lbm_step(100) + lbm_macros(pinned host rho,u)"}


def run_part(args):
    """One extra measurement alone (used for profiling captures)."""
    import numpy as np
    import torch

    from paper_1202_6351_gb300 import lbm

    torch.cuda.set_device(0)
    sp = torch.cuda.current_stream().cuda_stream
    peak, _ = measured_peaks()
    if args.part == "adjoint":
        out = run_adjoint_extras(lbm, torch, np, sp, n=args.adjoint_n, steps=args.adjoint_steps, peak=peak)
    elif args.part == "batch":
        out = run_batch_extras(lbm, torch, np, peak, sp, steps=args.batch_steps, count=args.batch_domains)
    else:
        from paper_1202_6351_gb300 import workloads

        n = args.n
        rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
        stores = {"f32": lbm.F32, "f16": lbm.F16DEV, "bf16": lbm.BF16DEV, "f64": lbm.F64}
        runs = ([(m, st, -1, 4) for st in (lbm.F32, lbm.F64) for m in (lbm.CASCADED, lbm.BGK, lbm.RAWMRT)]
                if args.part == "cost" else [(lbm.CASCADED, stores[args.store], args.variant, args.steps)])
        for model, st, variant, steps in runs:
            with lbm.Lattice(n, n, omegas(), model=model, store=st, stream=sp) as L:
                if variant >= 0:
                    L.set_variant(variant)
                L.set_graph_steps(0).init(rho, u).step(steps)
                torch.cuda.synchronize()
        out = {"runs": len(runs), "n": n}
    print(json.dumps({"part": args.part, **out}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.part != "all":
        return run_part(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
