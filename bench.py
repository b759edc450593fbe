"""Benchmark: Gerchberg-Saxton iterations/s on a 2048x2048 Fourier hologram (FP32, complex64).

Workload (one step = one full hot-path run over one synthetic input): hg_gs_run of 100 GS iterations,
continuous phase, on a 2048 x 2048 target (smoothed-noise amplitude, sigma 2 px, seed 0 + rank),
uniform starting phase (seed 1 + rank), NMSE of every iterate.  Inputs are resident in HBM when the
timed region starts; L2 is flushed (a 512 MiB write) before every timed step, outside the step's
events.  value = GS iterations/s over all ranks (weak scaling: every rank runs its own hologram).

Also reported:
  roofline      the dominant kernel's algorithmic bytes per launch / its mean launch time, against
                the measured HBM copy bandwidth.  The launch time is the kernel's share of device
                time (CUDA events the library records around every launch, in extra replays of a
                timed copy of the graph after the timed region) times the untimed step time, over
                its launches per step; the raw event-node time is reported beside it.
                iteration_frac: 36 B/px per GS iteration x px x it/s over the same peak.  traffic =
                DRAM bytes per launch from the committed ncu summary when it was taken on the
                current kernel sources (else null)
  e2e           the same metric through the public API with host buffers: every step copies the
                target and starting phase from pinned host memory and reads back the NMSE curve and
                the output phase inside the timed region, pipelined (the next step's inputs copied in
                and the last step's outputs read back while a step computes)
  cpu_baseline  the FP64 oracle (single thread) on a bounded sample of the same workload
  clocks        nvidia-smi SM clocks / throttle reasons sampled during the timed steps
  secondary     the rest of the metric, each timed over graph replays after warm-up and given
                with its fraction of the HBM peak: the 4-level variant of the headline, GS at
                4096^2 (the size whose working set leaves L2), OSPR 1080x1920 (16 targets x 24
                subframes), GS 256^2 and Fresnel GS 1024^2 8-level, gradient descent vs
                multi-plane GS at 2048^2 with 3 Fresnel planes (time to NMSE), and the 64-hologram
                mixed-size batch (holograms/s, p50 / p99 latency)

--impl reference times the oracle (the only reference this method has) on the same workload.
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
sys.path.insert(0, ROOT)
if "reference" in sys.argv:
    # the oracle leg runs on one host thread (set before numpy is imported)
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

H = W = 2048
N_ITER = 100
SIGMA = 2.0
METRIC = "GS iterations/s at 2048x2048 FP32 (Fourier, continuous phase, 100 iterations per run)"
UNIT = "it/s"
WORKLOAD = "Fourier GS 2048x2048 complex64, continuous phase, 100 iterations/run, per-iteration NMSE"
BYTES_PER_PX = {"col_gs": 20, "row_gs": 16, "row_init": 12, "col_nmse": 12}  # algorithmic HBM bytes
PROFILE_MD = os.path.join(ROOT, "profiles", "gs_2048_kernels.md")
KERNEL_SOURCES = ["paper_2006_10509_gb300/csrc/hg_fft.cuh", "paper_2006_10509_gb300/csrc/hg_kernels.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(kind: str):
    """DRAM bytes per launch of ``kind`` from the committed ncu summary, if it matches the sources."""
    if not os.path.exists(PROFILE_MD):
        return None
    src_hash, traffic = None, {}
    with open(PROFILE_MD) as f:
        for line in f:
            if line.startswith("source_hash:"):
                src_hash = line.split(":", 1)[1].strip()
            if line.startswith("traffic_bytes_per_launch:"):
                _, k, v = line.split()
                traffic[k] = int(v)
    if src_hash != kernel_source_hash():
        return None
    return traffic.get(kind)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if os.environ.get("HG_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def rank_seeds(rank: int) -> tuple[int, int]:
    """Seeds of the hologram a rank runs (target, starting phase): every rank has its own hologram."""
    return 0 + rank, 1 + rank


def max_over_ranks(x: float, ws: int, dev) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle legs


ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import synth
from oracle import gs as ogs
a = synth.blur_target({h}, {w}, {sigma}, seed=0).astype(np.float64)
phi = synth.uniform_phase({h}, {w}, seed=1).astype(np.float64)
h = np.exp(1j * phi)
h = ogs.gs_step(h, a, 0)["h"]  # warm-up (page in, allocator)
t = time.perf_counter()
for _ in range({n}):
    h = ogs.gs_step(h, a, 0)["h"]
dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt, "iterations": {n}}}))
"""


def host_cpu() -> dict:
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo, else platform)."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def oracle_gs_rate(n_iter: int) -> tuple[float, float]:
    """Runs n_iter FP64 oracle GS iterations (forward transform, amplitude replacement, inverse
    transform, projection) in a single-threaded subprocess; returns (iterations/s, seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, h=H, w=W, sigma=SIGMA, n=n_iter)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["iterations"] / d["seconds"], d["seconds"]


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric / unit / workload."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import synth
    from oracle import gs as ogs

    a = synth.blur_target(H, W, SIGMA, seed=0).astype(np.float64)
    phi = synth.uniform_phase(H, W, seed=1).astype(np.float64)
    h = np.exp(1j * phi)
    for _ in range(args.warmup):
        h = ogs.gs_step(h, a, 0)["h"]
    t = time.perf_counter()
    for _ in range(args.steps):
        h = ogs.gs_step(h, a, 0)["h"]  # one sample GS iteration per step
    dt = time.perf_counter() - t
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "1 GS iteration per step (the oracle's 100-iteration run "
                                                   "takes minutes; the per-iteration NMSE is not taken): the "
                                                   "per-iteration rate is comparable with the GPU arm's, whose "
                                                   "step is a 100-iteration run", "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} single GS iterations of the 2048x2048 workload, float64, "
                                   "one thread", **host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU leg


def run_ours(args):
    ws, rank, local = dist_setup()
    import numpy as np
    import torch

    import paper_2006_10509_gb300 as hg
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from __graft_entry__ import build

    if rank == 0 or ws == 1:
        build()
    barrier(ws)
    build()

    seed_t, seed_p = rank_seeds(rank)
    a_host = torch.from_numpy(synth.blur_target(H, W, SIGMA, seed=seed_t)).pin_memory()
    p_host = torch.from_numpy(synth.uniform_phase(H, W, seed=seed_p)).pin_memory()
    a = a_host.to(dev)
    p = p_host.to(dev)
    nm = torch.zeros((1, N_ITER + 1), dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # graph mode: each step replays one CUDA graph of the run's 200+ launches (captured in the
    # warm-up); the last warm-up step also captures the timed variant of the graph
    plan = hg.Plan([H], [W])
    if args.tuning:  # fixed choice (reproduces a tuned run without the autotuner's launches)
        w_, pr_, pc_ = (int(x) for x in args.tuning.split(","))
        plan.set_strip_width(0, w_)
        plan.set_radix_plan(0, pr_, pc_)
    else:
        plan.autotune()  # strip width and per-pass radix plans (library autotuner)
    tuned = {"strip_width": plan.strip_width(0), "radix_plan_row_col": list(plan.radix_plan(0)),
             "by": "given" if args.tuning else "hg_plan_autotune"}
    plan.set_graph(True)
    for i in range(args.warmup):
        plan.set_timing(i == args.warmup - 1)
        plan.gs([a], N_ITER, init_phase=[p], nmse_out=nm)
    plan.set_timing(False)
    torch.cuda.synchronize()

    # timed region: K steps of the untimed graph, L2 flushed before each (outside the step's events)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = plan.launch_count()
    with ClockSampler(local) as clocks:
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            plan.gs([a], N_ITER, init_phase=[p], nmse_out=nm)
            e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        wall = time.perf_counter() - t0
    launches = plan.launch_count() - launches0
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    dev_ms = max_over_ranks(dev_ms, ws, dev)
    ms_per_step = dev_ms / args.steps
    value = ws * N_ITER * args.steps / (dev_ms / 1e3)
    final_nmse = float(nm[0, -1].item())

    # per-kernel shares of device time: extra replays (after the timed region) of the graph copy
    # whose event nodes bracket every kernel; the totals take its latest replay.  The event nodes
    # slow a replay down, so they give shares; a kernel's launch time is its share of the untimed
    # step time over its launches per step.
    plan.reset_timing()
    plan.set_timing(True)
    timed_ms = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.gs([a], N_ITER, init_phase=[p], nmse_out=nm)
        e1.record(stream)
        e1.synchronize()
        timed_ms.append(e0.elapsed_time(e1))
    plan.set_timing(False)
    ktimes = plan.kernel_times()
    ktot = sum(v[0] for v in ktimes.values())
    share = {k: v[0] / ktot for k, v in ktimes.items()}

    # dominant kernel roofline
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    launch_us = share[dom] * ms_per_step / dom_n * 1e3
    alg_bytes = BYTES_PER_PX.get(dom, 16) * H * W
    achieved = alg_bytes / (launch_us / 1e6) / 1e9
    peak, peak_src = measured_peaks()
    it_gbs = 36 * H * W * value / ws / 1e9  # one rank's GS iterations: 36 B/px each
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": profiled_traffic(dom),
                "alg_bytes_per_launch": alg_bytes, "mean_launch_us": launch_us,
                "launch_time": "share of device time in the timed graph copy x untimed ms_per_step / launches per step",
                "event_node_launch_us": dom_ms / dom_n * 1e3,
                "timed_copy_ms_per_step": statistics.median(timed_ms),
                "iteration_bytes_per_px": 36, "iteration_achieved": it_gbs, "iteration_frac": it_gbs / peak,
                "kernel_share": share,
                "kernel_launch_us": {k: share[k] * ms_per_step / v[1] * 1e3 for k, v in ktimes.items()}}

    # end to end through the public API with host buffers, pipelined as a serving loop runs it: each
    # step's target and starting phase are copied from pinned host memory while the previous step
    # computes, and its NMSE curve and output phase are read back while the next step computes (two
    # device buffer sets on a copy stream, and two plans so that each replays its own graph).  The
    # timed region runs from the first input copy to the last read-back; the L2 flush before each
    # step (on the compute stream, not part of the work) is timed with its own events and taken out.
    plan2 = hg.Plan([H], [W])
    plan2.set_strip_width(0, plan.strip_width(0))
    plan2.set_radix_plan(0, *plan.radix_plan(0))
    plan2.set_graph(True)
    plans = [plan, plan2]
    cs = torch.cuda.Stream(dev)
    a_d = [torch.empty_like(a) for _ in range(2)]
    p_d = [torch.empty_like(p) for _ in range(2)]
    ph_d = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(2)]
    nm_d = [torch.empty_like(nm) for _ in range(2)]
    nm_h = [torch.empty((1, N_ITER + 1), dtype=torch.float32).pin_memory() for _ in range(2)]
    ph_h = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    d2h_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(k_steps):
        """k_steps pipelined steps; returns (wall ms, flush ms) from events."""
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        e_start.record(stream)
        cs.wait_event(e_start)
        with torch.cuda.stream(cs):
            a_d[0].copy_(a_host, non_blocking=True)
            p_d[0].copy_(p_host, non_blocking=True)
            h2d_done[0].record(cs)
        for k in range(k_steps):
            s = k % 2
            fl[k][0].record(stream)
            flush.zero_()
            fl[k][1].record(stream)
            if k >= 2:
                stream.wait_event(d2h_done[s])  # step k - 2's outputs have been read back
            stream.wait_event(h2d_done[s])
            plans[s].gs([a_d[s]], N_ITER, init_phase=[p_d[s]], phase_out=[ph_d[s]], nmse_out=nm_d[s])
            comp_done[s].record(stream)
            with torch.cuda.stream(cs):
                if k + 1 < k_steps:  # the next step's inputs, into the buffers step k - 1 read
                    if k >= 1:
                        cs.wait_event(comp_done[1 - s])
                    a_d[1 - s].copy_(a_host, non_blocking=True)
                    p_d[1 - s].copy_(p_host, non_blocking=True)
                    h2d_done[1 - s].record(cs)
                cs.wait_event(comp_done[s])
                nm_h[s].copy_(nm_d[s], non_blocking=True)
                ph_h[s].copy_(ph_d[s], non_blocking=True)
                d2h_done[s].record(cs)
        for s in range(min(2, k_steps)):
            stream.wait_event(d2h_done[s])
        e_end.record(stream)
        torch.cuda.synchronize()
        return e_start.elapsed_time(e_end), sum(f0.elapsed_time(f1) for f0, f1 in fl)

    e2e_run(max(3, args.warmup))  # warm-up: the second plan captures its graph
    barrier(ws)
    wall_ms, flush_ms = e2e_run(args.steps)
    e2e_ms = max_over_ranks(wall_ms - flush_ms, ws, dev)
    e2e = {"value": ws * N_ITER * args.steps / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": a_host.numel() * 4 + p_host.numel() * 4,
           "d2h_bytes_per_step": nm_h[0].numel() * 4 + ph_h[0].numel() * 4,
           "pipelined": "inputs of step k+1 copied in while step k computes, outputs of step k read back "
                        "while step k+1 computes; timed from the first input copy to the last read-back, "
                        "minus the L2 flushes between steps",
           "flush_ms_excluded": flush_ms,
           "same_nmse_curve_as_device_run": bool(torch.equal(nm_h[(args.steps - 1) % 2], nm.cpu()))}
    plan2.close()
    plan.close()

    if rank != 0:
        return
    # the rest of the metric (one GPU; rank 0 only under torchrun)
    secondary = None
    if not args.no_secondary:
        secondary = {}
        for w in ("gs2048q4", "gs4096", "ospr"):
            secondary[w] = time_workload(w, dev, 3, 10, tune=False)
        for w in ("gs256", "fresnel1024"):  # configurations 1 and 2, strip widths autotuned
            secondary[w] = time_workload(w, dev, 3, 10)
        g = gd_vs_gs(dev, 3)
        secondary["gd_vs_gs"] = {k: g[k] for k in ("workload", "metric", "time_to", "gd", "gs")}
        b = batch_workload(dev, 3, 5)
        secondary["batch"] = {k: v for k, v in b.items() if k not in ("by_size_last_run",)}
        torch.cuda.synchronize()
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        n = args.cpu_iters
        rate, secs = oracle_gs_rate(n)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} GS iterations of the same 2048x2048 workload, "
                         f"{secs:.1f} s, float64, one thread, NMSE not taken",
               **host_cpu()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "n_iter": N_ITER, "quant_levels": 0,
                   "target": f"smoothed noise sigma {SIGMA} px, seed 0+rank", "init_phase": "uniform, seed 1+rank",
                   "l2": "flushed (512 MiB write) before every timed step", "parallelism": f"replicas x{ws}",
                   "launch": "CUDA graph replay per step (library graph mode)", "autotuned": tuned,
                   "kernel_times": "shares from event nodes of a timed graph copy replayed after the timed "
                                   "region, times the untimed step time",
                   "final_nmse": final_nmse},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks.summary(), "wall_s": wall, "secondary": secondary,
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- other workloads (not the headline)


def run_batch(args):
    """Prints batch_workload (below) as one JSON line."""
    import torch

    from __graft_entry__ import build

    build()
    print(json.dumps(batch_workload(torch.device("cuda", 0), args.warmup, args.steps)))


def batch_workload(dev, warmup: int, steps: int) -> dict:
    """Mixed-size serving batch: 64 Fourier GS holograms, sizes drawn with seed 5000 from
    {512^2, 1024^2, 1536x864, 2048^2, 4096^2}, smoothed-noise targets (seeds 5001..5064), 4-level
    phase, 50 iterations, starting phase drawn on the device; strip widths autotuned per size class;
    the whole batch as one CUDA-graph launch (size classes smallest first).  Compared with the plain
    per-hologram loop (one-item plans, same kernels and widths, launched one after another), which
    reaches the same NMSE."""
    import numpy as np
    import torch

    import paper_2006_10509_gb300 as hg
    import synth

    sizes = synth.mixed_sizes(64, 5000)
    n_iter, levels = 50, 4
    targets = [torch.from_numpy(synth.blur_target(h, w, SIGMA, seed=5001 + i)).to(dev) for i, (h, w) in enumerate(sizes)]
    px = sum(h * w for h, w in sizes)
    nm = torch.zeros((64, n_iter + 1), dtype=torch.float32, device=dev)
    plan = hg.Plan([h for h, _ in sizes], [w for _, w in sizes], quant_levels=levels)
    # strip widths of the tiled field per size class, picked by the library's autotuner
    plan.autotune()
    widths = {sizes[i]: plan.strip_width(i) for i in range(len(sizes))}
    radix = {sizes[i]: plan.radix_plan(i) for i in range(len(sizes))}
    # starting phases: the device draw (seed 5000) projected to the levels, taken once so that the
    # per-hologram loop below starts every hologram from exactly the same field
    phases = [torch.empty((h, w), dtype=torch.float32, device=dev) for h, w in sizes]
    plan.gs(targets, 0, seed=5000, phase_out=phases)
    plan.set_graph(True)
    for _ in range(warmup):
        plan.gs(targets, n_iter, init_phase=phases, nmse_out=nm)
    torch.cuda.synchronize()
    lats, times = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.gs(targets, n_iter, init_phase=phases, nmse_out=nm)
        e1.record()
        lats.extend(plan.item_latency_ms())
        times.append(e0.elapsed_time(e1))
    final_batch = nm[:, -1].cpu().numpy()
    plan.close()
    # plain per-hologram loop: one-item plans, same kernels (same strip widths and radix plans),
    # launched one after another
    singles = [hg.Plan([h], [w], quant_levels=levels) for h, w in sizes]
    for pl, sz in zip(singles, sizes):
        pl.set_strip_width(0, widths[sz])
        pl.set_radix_plan(0, *radix[sz])
    nm1 = torch.zeros((64, n_iter + 1), dtype=torch.float32, device=dev)
    for k, pl in enumerate(singles):
        pl.gs([targets[k]], n_iter, init_phase=[phases[k]], nmse_out=nm1[k])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k, pl in enumerate(singles):
        pl.gs([targets[k]], n_iter, init_phase=[phases[k]], nmse_out=nm1[k])
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    final_loop = nm1[:, -1].cpu().numpy()
    for pl in singles:
        pl.close()
    ms = statistics.median(times)
    lat = np.array(lats)
    line = {"workload": "mixed-size GS batch: 64 holograms, 4-level, 50 iterations, one CUDA-graph launch",
            "metric": "holograms/s", "value": 64 / (ms / 1e3), "unit": "holograms/s", "ms_per_batch": ms,
            "px_iter_per_s": px * n_iter / (ms / 1e3), "total_px": px,
            "alg_gbytes_per_batch": 36 * px * n_iter / 1e9,
            "achieved_gb_s": 36 * px * n_iter / (ms / 1e3) / 1e9,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "by_size_last_run": {f"{h}x{w}": round(float(np.mean([l for l, sz in zip(lats[-64:], sizes)
                                                                               if sz == (h, w)])), 3)
                                                for h, w in sorted(set(sizes))}},
            "sequential_loop_ms": seq_ms, "speedup_vs_loop": seq_ms / ms,
            "final_nmse_median": float(np.median(final_batch)),
            "loop_same_final_nmse": bool(np.array_equal(final_batch, final_loop)),
            "steps": steps, "warmup": warmup,
            "sizes": {f"{h}x{w}": sum(1 for s in sizes if s == (h, w)) for h, w in sorted(set(sizes))},
            "autotuned_strip_widths": {f"{h}x{w}": widths[(h, w)] for h, w in sorted(set(sizes))},
            "autotuned_radix_plans_row_col": {f"{h}x{w}": list(radix[(h, w)]) for h, w in sorted(set(sizes))}}
    return line


CONFIG_WORKLOADS = ("gs256", "fresnel1024", "ospr", "mraf2048", "hio2048", "dbs128", "gs2048q4", "gs4096")


def config_workload(w: str, dev):
    """One of the single-GPU configurations: returns (plan, run, units, unit, bytes per unit, nmse
    buffer, tunable).  Inputs are built on the host from the seeded generators and copied once.
    gs256:       Fourier GS 256^2, continuous, 20 iterations, smoothed-noise target (seed 1001), start
                 phase seed 1002 (latency-bound: the whole field is 512 KB).
    fresnel1024: Fresnel GS 1024^2 (532 nm, 8 um, z = 0.1 m), 8-level, 100 iterations, 50-spot target
                 (seed 2001), start phase seed 2002.
    ospr:        OSPR 1920x1080 (W x H), 16 point-symmetric smoothed-noise targets (seeds 3001..3016),
                 24 binary subframes each, Philox seed 3000, the whole batch as one graph launch.
    mraf2048:    MRAF 2048^2, continuous, signal window rows and columns [1/8, 3/8) of the FFT-order
                 plane, m = 0.5, 100 iterations, 50-spot target (seed 6001), start phase seed 6002.
    hio2048:     HIO on the same problem, beta = 0.7.
    dbs128:      direct binary search 128^2, two sweeps (seeds 7001 / 7002).
    gs2048q4:    the headline workload (2048^2, seeds 0 / 1, 100 iterations) with 4-level phase.
    gs4096:      Fourier GS 4096^2, continuous, 100 iterations, smoothed-noise target (seed 8001),
                 start phase seed 8002: the field (128 MB) and target leave the L2."""
    import torch

    import paper_2006_10509_gb300 as hg
    import synth

    def gs_plain(n, n_iter, seed_t, seed_p, levels):
        a = torch.from_numpy(synth.blur_target(n, n, SIGMA, seed=seed_t)).to(dev)
        p0 = torch.from_numpy(synth.uniform_phase(n, n, seed=seed_p)).to(dev)
        plan = hg.Plan([n], [n], quant_levels=levels)
        nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
        run = lambda: plan.gs([a], n_iter, init_phase=[p0], nmse_out=nm)  # noqa: E731
        return plan, run, n_iter, "it/s", 36 * n * n, nm, True

    if w == "gs256":
        return gs_plain(256, 20, 1001, 1002, 0)
    if w == "gs2048q4":
        return gs_plain(2048, 100, 0, 1, 4)
    if w == "gs4096":
        return gs_plain(4096, 100, 8001, 8002, 0)
    if w == "fresnel1024":
        h = wd = 1024
        n_iter = 100
        a = torch.from_numpy(synth.spots_target(h, wd, 50, seed=2001)).to(dev)
        p0 = torch.from_numpy(synth.uniform_phase(h, wd, seed=2002)).to(dev)
        plan = hg.Plan([h], [wd], propagation=hg.HG_FRESNEL, wavelength_m=532e-9, pitch_m=8e-6, z_m=[0.1],
                       quant_levels=8)
        nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
        run = lambda: plan.gs([a], n_iter, init_phase=[p0], nmse_out=nm)  # noqa: E731
        return plan, run, n_iter, "it/s", 36 * h * wd, nm, True
    if w in ("mraf2048", "hio2048"):
        h = wd = 2048
        n_iter = 100
        a = torch.from_numpy(synth.spots_target(h, wd, 50, seed=6001)).to(dev)
        p0 = torch.from_numpy(synth.uniform_phase(h, wd, seed=6002)).to(dev)
        mask = torch.zeros((h, wd), dtype=torch.uint8, device=dev)
        mask[h // 8: 3 * h // 8, wd // 8: 3 * wd // 8] = 1
        plan = hg.Plan([h], [wd])
        nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
        if w == "mraf2048":
            run = lambda: plan.mraf([a], 0.5, n_iter, signal_mask=[mask], init_phase=[p0], nmse_out=nm)  # noqa: E731
            return plan, run, n_iter, "it/s", 36 * h * wd, nm, True
        run = lambda: plan.hio([a], 0.7, n_iter, signal_mask=[mask], init_phase=[p0], nmse_out=nm)  # noqa: E731
        # GS's 36 B/px plus the stored input X read and written on the noise region
        return plan, run, n_iter, "it/s", 36 * h * wd + 16 * (h * wd - (h // 4) * (wd // 4)), nm, True
    if w == "dbs128":
        h = wd = 128
        n_sweeps = 2
        a = torch.from_numpy(synth.blur_target(h, wd, SIGMA, seed=7001)).to(dev)
        p0 = torch.from_numpy(synth.uniform_phase(h, wd, seed=7002)).to(dev)
        plan = hg.Plan([h], [wd], quant_levels=2)
        nm = torch.zeros((1, n_sweeps + 1), dtype=torch.float32, device=dev)
        run = lambda: plan.dbs([a], n_sweeps, init_phase=[p0], nmse_out=nm)  # noqa: E731
        # trial flips; the replay plane stays in registers, so no HBM bytes per trial
        return plan, run, n_sweeps * h * wd, "trial flips/s", 0, nm, False
    if w == "ospr":
        h, wd, nt, ns = 1080, 1920, 16, 24
        ts = [torch.from_numpy(synth.symmetrise(synth.blur_target(h, wd, SIGMA, seed=3001 + k))).to(dev)
              for k in range(nt)]
        bits = [torch.zeros((ns, h, (wd + 31) // 32), dtype=torch.int32, device=dev) for _ in range(nt)]
        plan = hg.Plan([h] * nt, [wd] * nt, quant_levels=2)
        nm = torch.zeros((nt, ns), dtype=torch.float32, device=dev)
        run = lambda: plan.ospr(ts, ns, 0, 3000, bits_out=bits, nmse_out=nm)  # noqa: E731
        return plan, run, nt * ns, "subframes/s", 44 * h * wd, nm, False
    raise ValueError(w)


def time_workload(w: str, dev, warmup: int, steps: int, strip_width=None, tune=True) -> dict:
    """Times one configuration over CUDA-graph replays (median of `steps` after `warmup`)."""
    import torch

    plan, run, units, unit, bpu, nm, tunable = config_workload(w, dev)
    width = None
    if tunable:
        if strip_width is not None:
            plan.set_strip_width(0, strip_width)
        elif tune:
            plan.autotune()  # GS strip widths
        width = plan.strip_width(0)
    plan.set_graph(True)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    peak, src = measured_peaks()
    gbs = bpu * units / (ms / 1e3) / 1e9
    line = {"workload": w, "value": units / (ms / 1e3), "unit": unit, "ms_per_run": ms,
            "alg_bytes_per_unit": bpu, "achieved_gb_s": gbs if bpu else None,
            "frac_of_hbm": gbs / peak if bpu else None, "peak_source": src,
            "final_nmse": nm.cpu().numpy()[:, -1].tolist()[:4], "steps": steps, "warmup": warmup, "graph": True}
    if width is not None:
        line["strip_width" if strip_width is not None else ("autotuned_strip_width" if tune else "strip_width")] = width
    plan.close()
    return line


def run_config(args):
    """The remaining single-GPU configurations (see config_workload), each timed over graph replays
    after warm-up, GS strip widths autotuned first unless --strip-width is given."""
    import torch

    from __graft_entry__ import build

    build()
    dev = torch.device("cuda", 0)
    print(json.dumps(time_workload(args.workload, dev, args.warmup, args.steps, args.strip_width)))


def run_gd(args):
    """Prints gd_vs_gs (below) as one JSON line."""
    import torch

    from __graft_entry__ import build

    build()
    print(json.dumps(gd_vs_gs(torch.device("cuda", 0), args.warmup)))


def gd_vs_gs(dev, warmup: int) -> dict:
    """Gradient descent vs multi-plane GS, time to a stated NMSE: 2048^2 phase, Fresnel planes at
    z = 0.08, 0.10, 0.12 m (532 nm, 8 um pitch), target intensities = squared spot images (seeds
    4001..4003, unit energy), start phase uniform (seed 4000).  GD: Adam lr 0.05 for up to 200 steps
    (loss = mean optimal-scale NMSE over planes).  GS: averaged projections, continuous phase, up to
    1000 iterations, plane-mean NMSE per iterate.  Reported: the time each method needs to reach
    NMSE 1e-2, 0.1 and the worse method's final NMSE (None where it never does within its budget)."""
    import numpy as np
    import torch

    import paper_2006_10509_gb300 as hg
    import synth

    n, zs, lam, pitch = 2048, [0.08, 0.10, 0.12], 532e-9, 8e-6
    ts = []
    for p in range(3):
        t = synth.spots_target(n, n, 50, seed=4001 + p).astype(np.float64) ** 2
        ts.append(torch.from_numpy((t / np.sqrt(np.sum(t * t))).astype(np.float32)).to(dev))
    amps = [torch.sqrt(t) for t in ts]
    phi0 = torch.from_numpy(synth.uniform_phase(n, n, seed=4000)).to(dev)
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=lam, pitch_m=pitch, z_m=zs)
    steps, iters = 200, 1000
    # gradient descent
    with hg.Plan([n], [n], **kw) as plan:
        for _ in range(warmup):  # warm-up on a scratch copy
            ph, m, v = phi0.clone(), torch.zeros_like(phi0), torch.zeros_like(phi0)
            plan.gd_step([ph], ts, [m], [v], 1, 0.05)
        ph, m, v = phi0.clone(), torch.zeros_like(phi0), torch.zeros_like(phi0)
        loss = torch.zeros((steps, 4), dtype=torch.float32, device=dev)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize()
        evs[0].record()
        for k in range(steps):
            plan.gd_step([ph], ts, [m], [v], k + 1, 0.05, loss_out=loss[k])
            evs[k + 1].record()
        torch.cuda.synchronize()
        gd_t = np.array([evs[0].elapsed_time(e) for e in evs[1:]])  # ms after step k (loss[k] is before it)
        gd_loss = loss[:, 3].cpu().numpy()
    # multi-plane GS (same start)
    with hg.Plan([n], [n], **kw) as plan:
        nm = torch.zeros((1, iters + 1), dtype=torch.float32, device=dev)
        for _ in range(warmup):
            plan.gs(amps, 10, init_phase=[phi0], nmse_out=nm[:, :11])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.gs(amps, iters, init_phase=[phi0], nmse_out=nm)
        e1.record()
        torch.cuda.synchronize()
        gs_ms = e0.elapsed_time(e1)
        gs_nmse = nm[0].cpu().numpy()

    def first_at(curve, level):
        idx = np.nonzero(curve <= level)[0]
        return int(idx[0]) if len(idx) else None

    def times(level):
        k_gd, k_gs = first_at(gd_loss, level), first_at(gs_nmse, level)
        # loss[k] is the NMSE of the phase before step k: reached after k steps (end of step k-1)
        t_gd = None if k_gd is None else (0.0 if k_gd == 0 else float(gd_t[k_gd - 1]))
        t_gs = None if k_gs is None else k_gs * gs_ms / iters
        return {"gd_ms": t_gd, "gd_steps": k_gd, "gs_ms": t_gs, "gs_iterations": k_gs,
                "faster": None if (t_gd is None and t_gs is None) else
                ("gd" if t_gs is None or (t_gd is not None and t_gd < t_gs) else "gs")}

    gd_final, gs_final = float(gd_loss[-1]), float(gs_nmse[-1])
    plateau = max(gd_final, gs_final)
    line = {"workload": "GD (Adam, hand-written adjoint) vs multi-plane GS, 2048^2, 3 Fresnel planes",
            "metric": "time to NMSE",
            "time_to": {"0.01": times(1e-2), "0.1": times(0.1), f"worse_final={plateau:.4g}": times(plateau)},
            "gd": {"ms_per_step": float(gd_t[-1] / steps), "steps": steps, "final_nmse": gd_final,
                   "alg_gb_s": 172 * n * n / (gd_t[-1] / steps / 1e3) / 1e9},
            "gs": {"ms_per_iter": gs_ms / iters, "iterations": iters, "final_nmse": gs_final,
                   "best_nmse": float(gs_nmse.min()), "best_at": int(np.argmin(gs_nmse)),
                   "alg_gb_s": 108 * n * n / (gs_ms / iters / 1e3) / 1e9},
            "curves": {"gd_loss_every_20": gd_loss[::20].tolist(), "gs_nmse_every_100": gs_nmse[::100].tolist()}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 'secondary' workloads of the headline line")
    ap.add_argument("--tuning", default=None, metavar="W,ROWPLAN,COLPLAN",
                    help="headline: use this strip width and these radix plans instead of the autotuner's")
    ap.add_argument("--workload", default="gs2048", choices=["gs2048", "batch", "gd", *CONFIG_WORKLOADS],
                    help="gs2048: the headline line; batch: the mixed-size serving batch; "
                         "gd: gradient descent vs multi-plane GS, time to NMSE; gs256 / fresnel1024 / ospr: "
                         "the other single-GPU configurations; mraf2048 / hio2048: the MRAF and HIO variants of GS; "
                         "dbs128: direct binary search, 128^2, two sweeps; gs2048q4: the headline with 4-level "
                         "phase; gs4096: GS at 4096^2")
    ap.add_argument("--strip-width", type=int, default=None,
                    help="gs256 / fresnel1024 / mraf2048 / hio2048: use this strip width (-1: the whole run in "
                         "one thread-block cluster) instead of the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "gd":
        run_gd(args)
        return
    if args.workload in CONFIG_WORKLOADS:
        run_config(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
