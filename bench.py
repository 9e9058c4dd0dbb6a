#!/usr/bin/env python
"""Throughput benchmark of the GB300 FHP lattice-gas path.

Metric: site updates per second (GSUPS = 1e9 node updates / s) of the fused
FHP step (motion, FHP-II scattering, bounce-back, forcing; arXiv:1208.2428
Section 2), and its fraction of the HBM roofline.

Workload (default ``cylinder``): 16384 x 4096 lattice, solid disc of radius
256 at (4096, 2048), walls on the first and last rows, periodic x, forcing
p = 5e-4, density 0.25, seed 3.  One benchmark step = the run's 1,000 time
steps followed by 32 x 32 coarse-graining, on inputs already resident on the
GPU.  The L2 cache is flushed (a 512 MB write) before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun (N > 1) every rank advances its own replica of the workload
(weak scaling, no collective on the data path); rank 0 prints the JSON line.
``--impl reference`` times the CPU oracle (test infrastructure, plain C) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-updates/s (GSUPS) and % of HBM roofline, 1 GB300"
UNIT = "GSUPS"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40, help="timed benchmark steps")
    ap.add_argument("--warmup", type=int, default=3, help="untimed warm-up benchmark steps")
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["cylinder", "channel", "periodic", "paper", "cylinder2x", "ensemble",
                                           "serving"],
                    default="cylinder")
    ap.add_argument("--ensemble-size", type=int, default=512, help="lattices of the ensemble workload")
    ap.add_argument("--batch-step-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="batch step kernel of the ensemble workload (0: tuned online)")
    ap.add_argument("--batch-temporal-block", type=int, default=0, choices=[0, 1, 2, 4],
                    help="batch temporal block of the ensemble workload (0: tuned online)")
    ap.add_argument("--serving-jobs", type=int, default=2000, help="requests of the serving trace")
    ap.add_argument("--serving-budget-gb", type=float, default=80.0, help="HBM budget of the serving arena")
    ap.add_argument("--no-serving-compare", action="store_true",
                    help="skip the one-lattice-at-a-time replay of the serving trace")
    ap.add_argument("--no-batch-compare", action="store_true",
                    help="skip the reduced batched-vs-per-lattice comparison of the default run")
    ap.add_argument("--lattice-steps", type=int, default=None,
                    help="time steps per benchmark step (default: the workload's run length)")
    ap.add_argument("--temporal-block", type=int, default=1)
    ap.add_argument("--temporal-block-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="blocked kernel for --temporal-block > 1: 0 automatic, 1 row wavefronts, 2 2-D tiles")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the automatic kernel choice instead of timing the configurations first")
    ap.add_argument("--step-kernel", type=int, default=0,
                    help="0 auto, 1 direct, 2 bulk-copy ring, 3 multi-step ring")
    ap.add_argument("--rules", type=int, default=2, choices=[1, 2, 3],
                    help="collision rule set: 2 FHP-II (default), 1 FHP-I, 3 FHP-III")
    ap.add_argument("--no-rules-compare", action="store_true",
                    help="skip the FHP-I / FHP-III throughput comparison of the cylinder line")
    ap.add_argument("--cg-block", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k-sweep", action="store_true",
                    help="skip the temporal-block comparison (k = 1, 2, 4, 8) of the cylinder line")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(name: str):
    """The single lattice a workload is timed on (for the batched workloads,
    the CPU oracle's sample: the ensemble's first lattice, or the first
    cylinder request of the serving trace)."""
    import workloads
    return {"cylinder": workloads.cylinder_16384x4096, "channel": workloads.channel_4096x1024,
            "periodic": workloads.periodic_256, "paper": workloads.cylinder_paper_size,
            "cylinder2x": lambda: workloads.cylinder_scaled(16384, 8192),
            "ensemble": lambda: workloads.ensemble_512()[0],
            "serving": lambda: next(j for j in workloads.serving_jobs(50) if j.obstacle == "cylinder"),
            }[name]()


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


def source_hash(files=("fhp_step.cu", "fhp_device.cuh", "fhp_quad.cuh")) -> str:
    """Hash of the kernel sources a recorded ncu figure was taken on."""
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_1208_2428_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str, steps_per_launch: float):
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    (recorded per lattice step of the workload), if it was taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", f"fhp_step_{workload_name}.txt")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("source_hash") != source_hash():
            return None
        return float(fields["dram_bytes_per_lattice_step_full_size"]) * steps_per_launch
    except Exception:
        return None


def recorded_block_traffic(count: int):
    """DRAM bytes per pass of the blocked batch kernel (k = 4) over the ensemble
    of `count` lattices from the committed ncu summary, if it was taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", f"fhp_batch_block_ensemble_{count}.txt")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("source_hash") != source_hash(("fhp_batch_block.cu", "fhp_device.cuh", "fhp_quad.cuh")):
            return None
        return float(fields["dram_bytes_per_pass_full_size"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="fhp_clocks_", suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        indices = sorted({r[0] for r in rows})
        idx = str(self.gpu_index) if str(self.gpu_index) in indices else indices[0]
        rows = [r for r in rows if r[0] == idx]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "gpu_index": int(idx)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model() -> str:
    """Host CPU model (lscpu's "Model name", else /proc/cpuinfo) and thread count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return f"{name or 'unknown'} ({os.cpu_count()} logical CPUs, {os.uname().machine})"


def cpu_baseline(job, s0, target_seconds: float):
    """Time the CPU oracle (as it stands) on bounded samples of the benchmark's
    workload: whole-lattice steps, as many as fit ~target_seconds, on all host
    cores (OpenMP row strips, the paper's threaded "Pth" analogue) and on one
    thread (its "seq" analogue)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.run(s0, job.seed, 0, 1, job.p)
    one = time.perf_counter() - t0
    n = max(1, min(50, int(target_seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(s0, job.seed, 1, n, job.p)
    dt = time.perf_counter() - t0
    single = None
    try:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.run(s0, job.seed, 1, 1, job.p)
        dt1 = time.perf_counter() - t0
        single = {"value": job.W * job.H / dt1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                  "sample": f"1 whole-lattice time step of the {job.W}x{job.H} workload "
                            f"({job.W * job.H:.3g} site updates, {dt1:.1f} s, one thread)"}
    finally:
        oracle.set_threads(cores)
    return {"value": job.W * job.H * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} whole-lattice time steps of the {job.W}x{job.H} workload "
                      f"({job.W * job.H * n:.3g} site updates, {dt:.1f} s, OpenMP row strips)",
            "one_thread": single, "cpu_model": cpu_model()}


def batched_vs_per_lattice(dev, stream, count: int, steps: int, per_steps: int, repeats: int = 1,
                           step_kernel: int = 0, temporal_block: int = 0):
    """Aggregate GSUPS of `count` ensemble lattices (sides 128..2048, 1 %
    point obstacles, per-lattice seeds and densities) advanced (a) as one
    batch -- one launch per step over all lattices, CUDA-graph replays -- and
    (b) lattice by lattice, each with its own launches."""
    import torch
    import workloads
    from paper_1208_2428_gb300 import Batch, Lattice
    jobs = workloads.ensemble_512(count)
    states = [j.initial_state() for j in jobs]
    nodes = sum(j.nodes for j in jobs)
    arena = sum(Batch.lattice_bytes(j.W, j.H) for j in jobs) + (256 << 20)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Batch(arena, device=dev, stream=stream) as b:
        b.set_graph_steps(64)
        b.set_step_kernel(step_kernel)
        b.set_temporal_block(temporal_block)
        for j, s0 in zip(jobs, states):
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
        # warm-up; the automatic choice times its six candidates here (64 steps each): both kernels at two
        # tile sizes, and blocked passes of 2 and 4 steps
        b.step(384)
        b.synchronize()
        b.step(1)   # reads that measurement
        b.synchronize()
        tuned = b.tuned_kernel() if step_kernel == 0 else step_kernel
        tuned_quads = b.tile_quads
        tuned_block = temporal_block if temporal_block else (b.tuned_temporal_block() if step_kernel == 0 else 1)
        best = None
        for _ in range(repeats):
            l0 = b.kernel_launches
            ev0.record(stream)
            b.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1)
            best = ms if best is None else min(best, ms)
            launches_batched = b.kernel_launches - l0
    batched = nodes * steps / (best / 1e3) / 1e9
    lats = []
    for j, s0 in zip(jobs, states):
        lat = Lattice(j.W, j.H, seed=j.seed, forcing_p=j.p, device=dev, stream=stream)
        lat.set_state(s0)
        lats.append(lat)
    for lat in lats:
        lat.step(2)
    torch.cuda.synchronize(dev)
    l0 = sum(lat.kernel_launches for lat in lats)
    ev0.record(stream)
    for lat in lats:
        lat.step(per_steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_per = ev0.elapsed_time(ev1)
    launches_per = sum(lat.kernel_launches for lat in lats) - l0
    for lat in lats:
        lat.close()
    per = nodes * per_steps / (ms_per / 1e3) / 1e9
    return {"lattices": count, "nodes": nodes, "batched_gsups": batched, "batched_steps": steps,
            "batched_kernel": ("fhp_batch_block_kernel" if tuned_block > 1 else
                               "fhp_batch_run_kernel" if tuned == 2 else "fhp_batch_kernel"),
            "batched_tile_quads": tuned_quads,
            "tuned": {"kernel": tuned, "tile_quads": tuned_quads, "temporal_block": tuned_block, "graph_steps": 64,
                      "set_by_flags": bool(step_kernel or temporal_block),
                      "candidates": "single-step graphs / multi-step cooperative x 256 / 128 quads per tile, "
                                    "and blocked passes of 2 / 4 steps"},
            "batched_launches": launches_batched, "per_lattice_gsups": per, "per_lattice_steps": per_steps,
            "per_lattice_launches": launches_per, "speedup": batched / per,
            "batched_ms": best, "per_lattice_ms": ms_per}


def run_ensemble(args):
    """The 512-lattice ensemble: the batched path is the timed metric."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    steps = args.lattice_steps or 2000
    sampler = ClockSampler(local)
    sampler.start()
    r = batched_vs_per_lattice(dev, stream, args.ensemble_size, steps, min(steps, 200), repeats=max(1, args.steps),
                               step_kernel=args.batch_step_kernel, temporal_block=args.batch_temporal_block)
    clocks = sampler.stop()
    peak, peak_src = measured_hbm_peak()
    # Algorithmic bytes per site update: 1.875 B for a single-step kernel; a
    # blocked pass of k steps reads and writes the state once, 1.875 / k B
    # per site update.  The single-step figure is kept for comparison.
    k_used = max(1, int(r["tuned"]["temporal_block"] or 1))
    bytes_per_node = 15 / 8.0 / k_used
    achieved = r["batched_gsups"] * 1e9 * bytes_per_node / 1e9
    traffic = recorded_block_traffic(args.ensemble_size) if k_used == 4 else None
    line = {
        "metric": METRIC, "value": r["batched_gsups"], "unit": UNIT, "n_gpus": 1, "steps": max(1, args.steps),
        "warmup": args.warmup, "ms_per_step": r["batched_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 (bit-planes, boolean/integer)",
        "data": "synthetic (512 seeded lattices, sides uniform in 128..2048 step 64, 1 % point obstacles)",
        "config": {"workload": f"ensemble_{args.ensemble_size}", "lattice_steps_per_step": steps,
                   "graph_steps": 64, "tuned": r["tuned"], "l2": "inputs (1.1 GB) larger than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": r["batched_kernel"],
                     "algorithmic_bytes_per_node_step": bytes_per_node, "temporal_block": k_used,
                     "single_step_equivalent_frac": r["batched_gsups"] * 15 / 8.0 / peak,
                     "peak_source": peak_src,
                     **({"note": "blocked passes move the state once per k steps, so DRAM is far from its roof; "
                                 "the pass is bound by instruction issue (ALU pipe ~52 %, "
                                 "profiles/fhp_batch_block_ensemble_512.txt); traffic: DRAM bytes per pass of "
                                 "the 512 lattices from that capture"} if k_used > 1 else {})},
        "batched_vs_per_lattice": r, "cpu_baseline": None, "e2e": None,
        "gpu_launches": r["batched_launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_requests(count: int, time_scale: float = 1.0):
    """The serving trace: Poisson arrivals (200/s), log-uniform sides and step
    counts, half of the requests with the cylinder geometry and forcing."""
    import workloads
    from paper_1208_2428_gb300.serving import Request
    reqs = []
    for j in workloads.serving_jobs(count):
        shapes = workloads.cylinder_shapes(j.W, j.H) if j.obstacle == "cylinder" else None
        reqs.append(Request(j.W, j.H, j.steps, seed=j.seed, density=j.density, forcing_p=j.p,
                            obstacle_shapes=shapes, cg_block=64, arrival=j.arrival * time_scale, name=j.name))
    return reqs


def serve_trace(dev, stream, reqs, budget_bytes: int, compare: bool):
    """Serve a trace by continuous batching (and, optionally, one lattice at a
    time); returns the summaries and the server's counters."""
    from paper_1208_2428_gb300 import serving
    with serving.Server(budget_bytes, quantum_max=64, quantum_min=8, graph_steps=16, device=dev, stream=stream,
                        time_device=True) as srv:
        done = srv.serve(reqs, realtime=True)
        st = srv.stats
    out = {"served": serving.summarize(done), "ticks": st.ticks, "peak_resident": st.peak_resident,
           "peak_resident_gb": st.peak_resident_bytes / 1e9, "admissions_deferred": st.admissions_deferred,
           "device_ms": st.device_ms, "device_launches": st.device_launches,
           "issued_site_updates": st.issued_site_updates,
           "issued_solid_site_updates": st.issued_solid_site_updates}
    if compare:
        out["one_lattice_at_a_time"] = serving.summarize(serving.serve_sequential(reqs, realtime=True, device=dev))
    return out


def run_serving(args):
    """Serving: requests arrive (Poisson, 200/s) and are served by continuous
    batching within an HBM budget; the metric is aggregate GSUPS over the
    trace, with p50/p99 request latency."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    budget = int(args.serving_budget_gb * 1e9)
    for _ in range(args.warmup):   # short traces: graph capture, allocator, clocks
        serve_trace(dev, stream, serving_requests(40, 0.2), min(budget, 8 << 30), compare=False)
    torch.cuda.synchronize(dev)
    reqs = serving_requests(args.serving_jobs)
    sampler = ClockSampler(local)
    sampler.start()
    r = serve_trace(dev, stream, reqs, budget, compare=not args.no_serving_compare)
    clocks = sampler.stop()
    peak, peak_src = measured_hbm_peak()
    # Algorithmic bytes: 7 state bits read and written per node update, plus
    # the solid bit where the lattice carries obstacles.
    alg_bytes = r["issued_site_updates"] * 1.75 + r["issued_solid_site_updates"] * 0.125
    achieved = alg_bytes / (r["device_ms"] / 1e3) / 1e9 if r["device_ms"] > 0 else 0.0
    served = r["served"]
    h2d = sum(16 * len(q.obstacle_shapes or []) + 64 for q in reqs)   # shapes and request parameters
    d2h = sum((q.width // q.cg_block) * (q.height // q.cg_block) * 48 for q in reqs)
    value = served["gsups"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": served["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 (bit-planes, boolean/integer)",
        "data": f"synthetic serving trace ({len(reqs)} requests, Poisson 200/s, sides log-uniform 256..8192, "
                "steps log-uniform 100..10000, half with a cylinder and forcing 5e-4)",
        "config": {"workload": f"serving_{len(reqs)}", "hbm_budget_gb": args.serving_budget_gb,
                   "quantum_steps": "8..64", "graph_steps": 16, "coarse_grain_block": 64,
                   "l2": "inputs (resident lattices, GBs) larger than L2"},
        "latency_ms": {"p50": served.get("p50_ms"), "p99": served.get("p99_ms"), "mean": served.get("mean_ms"),
                       "max": served.get("max_ms")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "fhp_batch_kernel",
                     "algorithmic_bytes": alg_bytes, "kernel_ms": r["device_ms"], "peak_source": peak_src},
        "serving": r, "cpu_baseline": None,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "the serving metric is itself end to end: wall clock from arrival to result on the host"},
        "gpu_launches": r["device_launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    job = workload(args.workload)
    s0 = job.initial_state()
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    # each step: a bounded whole-lattice sample sized so the run ends in minutes
    t0 = time.perf_counter()
    oracle.run(s0, job.seed, 0, 1, job.p)
    one = time.perf_counter() - t0
    per_step = max(1, min(job.steps, int(3.0 / max(one, 1e-3))))
    t = 1
    for _ in range(args.warmup):
        oracle.run(s0, job.seed, t, 1, job.p)
        t += 1
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(s0, job.seed, t, per_step, job.p)
        times.append(time.perf_counter() - t0)
        t += per_step
    total = sum(times)
    value = job.W * job.H * per_step * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded Bernoulli lattice, index-coordinate cylinder)",
        "config": {"workload": job.name, "W": job.W, "H": job.H, "lattice_steps_per_step": per_step,
                   "forcing_p": job.p, "density": job.density, "seed": job.seed,
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {per_step} whole-lattice time steps of {job.W}x{job.H}",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world != args.gpus:
        if world > 1 or args.gpus > 1:
            raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}: launch with torchrun for N > 1")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_1208_2428_gb300 import Lattice

    job = workload(args.workload)
    nsteps = args.lattice_steps or job.steps
    B = args.cg_block if (job.W % args.cg_block == 0 and job.H % args.cg_block == 0) else 0
    s0 = job.initial_state()
    seed = job.seed + 1_000_003 * rank   # independent replicas per rank
    has_solid = bool((s0 & 0x80).any())

    stream = torch.cuda.current_stream(dev)
    lat = Lattice(job.W, job.H, seed=seed, forcing_p=job.p, device=dev, stream=stream)
    lat.set_state(s0)
    lat.set_rules(args.rules)
    lat.set_temporal_block(args.temporal_block)
    if args.temporal_block_kernel:
        lat.set_temporal_block_kernel(args.temporal_block_kernel)
    lat.set_step_kernel(args.step_kernel)
    tuned = None
    if not args.no_autotune and args.step_kernel == 0 and args.temporal_block == 1:
        tuned = lat.autotune(128)  # untimed: the kernel / temporal block used below
    k_block = lat.temporal_block
    nby, nbx = (job.H // B, job.W // B) if B else (1, 1)
    counts = torch.empty((nby, nbx, 9), dtype=torch.int32, device=dev)
    rho = torch.empty((nby, nbx), dtype=torch.float32, device=dev)
    ux = torch.empty_like(rho)
    uy = torch.empty_like(rho)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def coarse():
        if B:
            lat.coarse_grain_into(B, counts, rho, ux, uy)

    # Coarse-grained fields every `every` lattice steps where the workload asks
    # for them (the channel: every 1,000 of its 10,000 steps), else once at the
    # end of the benchmark step.
    cg_every = getattr(job, "cg_every", None)
    every = cg_every if (B and cg_every and nsteps % cg_every == 0) else nsteps
    chunks = nsteps // every

    def bench_step():
        for _ in range(chunks):
            lat.step(every)
            coarse()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # around each fhp_step call of the timed region (one per chunk)
    step_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(chunks)] for _ in range(args.steps)]
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = lat.kernel_launches
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                       # L2 flush between timed steps
        starts[i].record(stream)
        for c in range(chunks):
            step_ev[i][c][0].record(stream)
            lat.step(every)
            step_ev[i][c][1].record(stream)
            coarse()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    launches = lat.kernel_launches - launches0
    clocks = sampler.stop()
    kernel_name = {1: "fhp_step_direct_kernel", 2: "fhp_step_tma_kernel", 3: "fhp_run_kernel",
                   4: "fhp_resident_kernel"}.get(lat.step_kernel, "?")
    # For the resident kernel the temporal block is the exchange interval
    # (steps between hand-offs of strip edge rows), not a blocked pass.
    resident = lat.step_kernel == 4
    if resident and k_block > 1:
        kernel_name = f"fhp_resident_ghost_kernel (exchange every {k_block} steps)"
    elif k_block > 1:
        kernel_name = f"{'fhp_wave_kernel' if lat.temporal_block_kernel == 1 else 'fhp_block_kernel'} (k={k_block})"
    k_pass = 1 if resident else k_block
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    step_kernel_ms = sum(a.elapsed_time(b) for evs in step_ev for a, b in evs)
    if dist:
        t = torch.tensor([total_ms, step_kernel_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, step_kernel_ms = float(t[0]), float(t[1])

    nodes = job.W * job.H
    value = world * nodes * nsteps * args.steps / (total_ms / 1e3) / 1e9
    bytes_per_node = (14 + (1 if has_solid else 0)) / 8.0
    # Step-kernel launches in the timed region: one per lattice step for the
    # single-step kernels, one per fhp_step call (chunks of 2^24 steps) for
    # the multi-step kernel.
    cg_launches = args.steps * chunks if B else 0
    step_launches = max(1, launches - cg_launches)
    steps_per_launch = nsteps * args.steps / step_launches
    launch_s = step_kernel_ms / 1e3 / step_launches
    # A temporally blocked pass reads and writes the state once for k steps.
    bytes_per_launch = bytes_per_node * nodes * steps_per_launch / k_pass
    achieved = bytes_per_launch / launch_s / 1e9
    peak, peak_src = measured_hbm_peak()
    # The committed capture is of the multi-step kernel.
    traffic = recorded_traffic(job.name, steps_per_launch) if (lat.step_kernel == 3 and k_block == 1) else None

    # End to end through the C ABI with host buffers: pinned initial state in,
    # coarse-grained fields out, host<->device copies inside the timed region.
    e2e = None
    if not args.no_e2e:
        host_state = torch.from_numpy(s0).pin_memory().numpy()
        h_counts = np.empty((nby, nbx, 9), dtype=np.int32)
        h_rho = np.empty((nby, nbx), dtype=np.float32)
        h_ux = np.empty_like(h_rho)
        h_uy = np.empty_like(h_rho)
        e2e_steps = max(3, min(args.steps, 10))
        def e2e_step():
            lat.set_state(host_state)
            for _ in range(chunks):
                lat.step(every)
                if B:
                    lat.coarse_grain_host_into(B, h_counts, h_rho, h_ux, h_uy)
            if not B:
                lat.synchronize()
        e2e_step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        if dist:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t[0])
        e2e = {"value": world * nodes * nsteps * e2e_steps / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(s0.nbytes),
               "d2h_bytes_per_step": chunks * int(h_counts.nbytes + h_rho.nbytes + h_ux.nbytes + h_uy.nbytes)
               if B else 0,
               "steps": e2e_steps}

    batch_cmp = None
    serving_cmp = None
    if rank == 0 and not args.no_batch_compare and args.workload == "cylinder":
        batch_cmp = batched_vs_per_lattice(dev, stream, 64, 200, 200)
        # A reduced serving trace (the first 300 requests, Poisson 200/s):
        # continuous batching against one lattice at a time.
        serving_cmp = serve_trace(dev, stream, serving_requests(300), int(args.serving_budget_gb * 1e9),
                                  compare=True)
        serving_cmp = {"requests": 300, "continuous_batching": serving_cmp["served"],
                       "one_lattice_at_a_time": serving_cmp["one_lattice_at_a_time"],
                       "peak_resident": serving_cmp["peak_resident"]}

    k_sweep = None
    if rank == 0 and not args.no_k_sweep and args.workload == "cylinder":
        k_sweep = temporal_block_sweep(job, s0, seed, dev, stream, nsteps, peak)
    rules_cmp = None
    if rank == 0 and not args.no_rules_compare and args.workload == "cylinder" and args.rules == 2:
        rules_cmp = rule_set_comparison(job, s0, seed, dev, stream, nsteps, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(job, s0, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 (bit-planes, boolean/integer)",
            "data": "synthetic (seeded Bernoulli lattice, index-coordinate cylinder)",
            "config": {"workload": job.name, "W": job.W, "H": job.H, "lattice_steps_per_step": nsteps,
                       "coarse_grain_block": B, "coarse_grain_every": every if B else None, "forcing_p": job.p, "density": job.density,
                       "seed": job.seed, "temporal_block": k_block, "rules": f"FHP-{'I' * args.rules}",
                       "autotuned": {"kernel": tuned[0], "temporal_block": tuned[1]} if tuned else None,
                       "step_kernel": kernel_name,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed (512 MB write) before every timed step; the 120 MB working "
                             "set is below the 126 MB L2 within a step"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kernel_name, "algorithmic_bytes_per_node_step": bytes_per_node,
                         "lattice_steps_per_launch": steps_per_launch,
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "launch_duration_us": launch_s * 1e6,
                         "peak_source": peak_src},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched_vs_per_lattice": batch_cmp,
            "serving_reduced": serving_cmp,
            "temporal_blocks": k_sweep,
            "rule_sets": rules_cmp,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.destroy_process_group()
    return 0


def temporal_block_sweep(job, s0, seed, dev, stream, nsteps, peak):
    """One call of `nsteps` lattice steps from the same state for temporal
    blocks k = 1, 2, 4, 8 (k = 1: the automatic single-step choice; k > 1:
    the automatic blocked kernel, 2-D tiles where they apply) and, as
    ``k<k>_wave``, the row-wavefront kernel for k = 2, 3, 4: GSUPS, the HBM
    fraction of the algorithmic bytes (a blocked pass reads and writes the
    state once per k steps) and whether the final states are identical."""
    import numpy as np
    import torch
    from paper_1208_2428_gb300 import Lattice
    bytes_per_node = (14 + (1 if (s0 & 0x80).any() else 0)) / 8.0
    names = {0: None, 1: "fhp_wave_kernel", 2: "fhp_block_kernel"}
    out, ref = {}, None
    for k, bk in ((1, 0), (2, 0), (4, 0), (8, 0), (2, 1), (3, 1), (4, 1)):
        with Lattice(job.W, job.H, seed=seed, forcing_p=job.p, device=dev, stream=stream) as lat:
            lat.set_step_kernel(0)
            lat.set_temporal_block(k)
            lat.set_temporal_block_kernel(bk)
            used_k, used_bk = lat.temporal_block, lat.temporal_block_kernel
            if bk and used_bk != bk:
                continue               # the requested kernel does not apply here
            lat.set_state(s0)
            lat.step(64)
            lat.set_state(s0)
            lat.set_time(0)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            final = lat.get_state()
        if ref is None:
            ref = final
        gsups = job.W * job.H * nsteps / (ms / 1e3) / 1e9
        key = f"k{k}" + ("_wave" if bk == 1 else "")
        if bk == 1 and out.get(f"k{k}", {}).get("kernel") == names[1]:
            continue                   # the automatic line already ran the wavefront kernel
        out[key] = {"temporal_block": used_k, "kernel": names.get(used_bk) or "single-step (automatic)",
                    "gsups": gsups, "ms": ms,
                    "hbm_frac": gsups * 1e9 * bytes_per_node / used_k / (peak * 1e9),
                    "same_final_state_as_k1": bool(np.array_equal(final, ref))}
    return out


def rule_set_comparison(job, s0, seed, dev, stream, nsteps, peak):
    """One autotuned call of `nsteps` lattice steps for each collision rule set
    (FHP-I, FHP-II, FHP-III) from the same state: GSUPS, the kernel the tuner
    chose and the HBM fraction of the algorithmic bytes."""
    import torch
    from paper_1208_2428_gb300 import Lattice
    bytes_per_node = (14 + (1 if (s0 & 0x80).any() else 0)) / 8.0
    names = {1: "fhp_step_direct_kernel", 2: "fhp_step_tma_kernel", 3: "fhp_run_kernel",
             4: "fhp_resident_kernel"}
    out = {}
    for rules in (1, 2, 3):
        with Lattice(job.W, job.H, seed=seed, forcing_p=job.p, device=dev, stream=stream) as lat:
            lat.set_rules(rules)
            lat.set_state(s0)
            kernel, k = lat.autotune(64)
            lat.set_state(s0)
            lat.set_time(0)
            lat.step(16)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(nsteps)
            e1.record(stream)
            lat.synchronize()
            ms = e0.elapsed_time(e1)
        gsups = job.W * job.H * nsteps / (ms / 1e3) / 1e9
        out[f"FHP-{'I' * rules}"] = {"gsups": gsups, "ms": ms, "kernel": names.get(kernel, str(kernel)),
                                     "temporal_block": k,
                                     "hbm_frac": gsups * 1e9 * bytes_per_node / k / (peak * 1e9)}
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
