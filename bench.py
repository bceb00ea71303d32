#!/usr/bin/env python3
"""Benchmark of the operator-split reaction-diffusion step on GB300.

Workload: jittered 100x10x10 um box of 294,780 tets, random 10-species /
20-reaction network, densities 1-100 /um^3, tau = 0.203 ms. One benchmark
step = one steps_run call advancing the simulation by 20 ms: 98 full windows
and one shortened window. The full windows run in the launch form the
simulation's first run picked by timing both (a flow launch: all 98 windows
in one launch, each tile starting when its neighbour tiles finished the
previous window; or one launch per window, replayed from CUDA graphs); the
shortened window is one launch. Metric: tet-updates/s = tets x windows / time.

  value     device time (CUDA events on the simulation's stream) of K steps,
            state resident in HBM; L2 flushed (256 MiB write) before each step,
            outside the timed events.
  e2e       the same metric through the public C ABI with host buffers:
            steps_set_counts_all (H2D), steps_run, steps_get_counts_all (D2H),
            wall clock per step.
  roofline  the step kernel, per window (a flow launch's ncu counts divided
            by its windows). The box's working set sits in L2 and the kernel
            is bound by instruction issue: bound "alu", warp instructions
            (ncu count per window) per second against 152 SMs x 4 schedulers
            x 1 warp instruction per cycle x the sampled SM clock. Beside it,
            `hbm`: algorithmic bytes per launch / average launch time against
            the measured copy bandwidth, on 8S + 52 bytes per tet-update (FP64
            split tables) and on the 8S + 36 bytes this design moves.
  cpu_baseline  the CPU oracle on the host's cores (threaded windows, bit for
            bit the serial oracle) on a bounded sample, with the single-core
            figure, the core count and the CPU model.

--impl reference runs the CPU oracle on all host cores as the reference arm.
With torchrun (N > 1) every rank runs an independent replica on its own GPU
(different seed): weak scaling, value = sum over ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tet-updates/s"
UNIT = "tet-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ["paper_1610_02258_gb300/csrc/steps_step.cuh", "paper_1610_02258_gb300/csrc/steps_kernels.cu",
                  "paper_1610_02258_gb300/csrc/steps_batch.cu", "paper_1610_02258_gb300/csrc/steps_internal.h",
                  "paper_1610_02258_gb300/csrc/steps_device.h", "paper_1610_02258_gb300/csrc/steps_spec.cpp"]


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(name: str):
    """DRAM bytes per launch recorded by ncu in profiles/<name>_traffic.txt,
    or None when the file is missing or the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", name + "_traffic.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(path) if ":" in line)
    except OSError:
        return None
    if kv.get("kernel_sources_sha256_16", "").strip() != kernel_sources_hash():
        return None
    tr = {k.strip(): int(v) for k, v in kv.items() if k.strip() != "kernel_sources_sha256_16"}
    # a flow launch holds several windows: the roofline works per window
    wpl = tr.get("windows_per_launch", 1)
    if wpl > 1:
        for k in ("bytes_per_launch", "read_bytes", "write_bytes", "warp_instructions_per_launch"):
            if k in tr:
                tr[k] = tr[k] // wpl
    return tr


def launch_form(sim):
    """(profile prefix, config keys) of a plain simulation's launch form."""
    block, tune = sim.flow
    keys = {"launch_form": f"flow ({block}-tet tiles)" if block else "window launches",
            "flow_tuning_ms_per_window": {"window_launches": tune[0], "flow": tune[1], "flow_512": tune[2]}
            if tune[0] > 0 else None}
    return (f"flow{block}_kernel" if block else "step_kernel"), keys


def issue_roofline(tr, kernel_s: float, sm_mhz, sms=None):
    """Warp instructions issued per second by the kernel (count per launch from
    the ncu capture, time per launch measured here) against the issue peak:
    SMs x 4 schedulers x 1 warp instruction per cycle x the SM clock sampled
    during the run."""
    if not tr or "warp_instructions_per_launch" not in tr:
        return None
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = sms * 4 * mhz * 1e6
    achieved = tr["warp_instructions_per_launch"] / kernel_s
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp-inst/s", "frac": achieved / peak,
            "warp_instructions_per_window": tr["warp_instructions_per_launch"], "sm_mhz": mhz,
            "note": "instruction count from the ncu capture in profiles/, time from this run"}


def replica_seed(rank: int) -> int:
    """Seed of the replica a rank runs (ranks run independent replicas)."""
    return 3 + rank


def reduce_over_ranks(ms: float, units: float):
    """Whole-job timing over ranks: the slowest rank's time and the units of
    all ranks (torch.distributed must be initialised)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def oracle_rate(w, windows: int, threads: int = 1):
    """Oracle (FP64) on `windows` full windows of the workload, on `threads`
    host threads (threaded windows give the serial result bit for bit)."""
    import oracle
    o = oracle.from_workload(w, prec=64)
    t0 = time.perf_counter()
    for _ in range(windows):
        o.step(o.tau, threads=threads)
    dt = time.perf_counter() - t0
    return w.n_tets * windows / dt, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_baseline(w, windows_all: int, windows_one: int):
    """The oracle on every host core and on one, bounded samples of the workload."""
    cores = host_cores()
    rate_all, dt_all = oracle_rate(w, windows_all, threads=cores)
    rate_one, dt_one = oracle_rate(w, windows_one, threads=1)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{windows_all} full windows of {w.name} ({dt_all:.1f} s) on {cores} threads, FP64",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_core": {"value": rate_one, "unit": UNIT, "cores": 1,
                            "sample": f"{windows_one} full windows ({dt_one:.1f} s), serial C, FP64"}}


def cpu_baseline_dendrite(I, windows_all: int, windows_one: int):
    """The oracle on the dendrite (1.03M tets, 20 species, masked influx), a
    reduced run from its initial counts, on every host core and on one."""
    w = I.config3()
    cores = host_cores()
    rate_all, dt_all = oracle_rate(w, windows_all, threads=cores)
    rate_one, dt_one = oracle_rate(w, windows_one, threads=1)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "workload": w.name,
            "sample": f"{windows_all} full windows ({dt_all:.1f} s) on {cores} threads, FP64",
            "single_core": {"value": rate_one, "unit": UNIT, "cores": 1,
                            "sample": f"{windows_one} full windows ({dt_one:.1f} s), serial C, FP64"}}


def roofline(S: int, masked: bool, tets: int, kernel_s: float, peak: float, peak_kind: str, tr, sm_mhz,
             issue_bound: bool, sms=None):
    """Roofline object of a plain step launch. hbm: algorithmic bytes per
    tet-update, 8S + 52 (counts in and out, neighbours, FP64 split tables,
    FP64 tau G, the volume factor) and the 8S + 36 (+4 with reaction masks)
    this design moves (fixed-point thresholds), over the average launch time,
    against the measured copy bandwidth. issue: warp instructions per launch
    (ncu) over the launch time against the issue peak. The binding one leads."""
    b52 = 8 * S + 52
    b36 = 8 * S + 36 + (4 if masked else 0)
    hbm = {"bound": "hbm", "achieved": tets * b52 / kernel_s / 1e9, "peak": peak, "unit": "GB/s",
           "frac": tets * b52 / kernel_s / 1e9 / peak, "bytes_per_tet_update": b52,
           "achieved_fixed_point": tets * b36 / kernel_s / 1e9, "frac_fixed_point": tets * b36 / kernel_s / 1e9 / peak,
           "bytes_per_tet_update_fixed_point": b36, "peak_source": peak_kind,
           "traffic": tr["bytes_per_launch"] if tr else None, "kernel_us_avg": kernel_s * 1e6}
    iss = issue_roofline(tr, kernel_s, sm_mhz, sms)
    if issue_bound and iss is not None:
        out = {"bound": "alu", "achieved": iss["achieved"], "peak": iss["peak"], "unit": "warp-inst/s",
               "frac": iss["frac"], "traffic": hbm["traffic"],
               "peak_source": f"SMs x 4 schedulers x 1 warp instruction/cycle x {iss['sm_mhz']:.0f} MHz (sampled)",
               "warp_instructions_per_window": iss["warp_instructions_per_window"], "kernel_us_avg": kernel_s * 1e6,
               "note": "working set in L2; bound by instruction issue (ncu issue slots and stalls in profiles/)",
               "hbm": hbm}
        return out
    hbm["issue"] = iss
    return hbm


def measure_batched(args, capi, I, torch, peak, flow=False):
    """Batched form: 256 replicates of config-2-style boxes, sizes log-uniform in
    [10k, 300k] tets, distinct seeds, 20 ms per step, one launch per window for
    all replicates, CUDA-graph replay, autotuned block size. flow: one flow
    launch per L2-sized group of replicates for all full windows of a run
    (256-tet tiles)."""
    sizes = I.batch_sizes(n=args.batch_replicates)
    t0 = time.perf_counter()
    ws = [I.box_for_tets(int(sz), seed=1000 + j) for j, sz in enumerate(sizes)]
    stream = torch.cuda.current_stream()
    sims = [capi.from_workload(w, cuda_stream=stream.cuda_stream) for w in ws]
    setup_s = time.perf_counter() - t0
    batch = capi.Batch(sims, block=256 if flow else 0, cuda_stream=stream.cuda_stream, flow=flow)
    T = np.array([s.nt for s in sims], dtype=np.int64)
    S = ws[0].model.n_species

    def reset():  # every step is the configured 20 ms run from the initial counts
        for s, w in zip(sims, ws):
            s.set_counts(w.counts)

    def step():
        batch.run([s.time + 20e-3 for s in sims])

    reset()
    step()  # autotune + warm
    for _ in range(2):
        reset()
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    w0 = np.array([s.windows for s in sims])
    steps = max(2, min(args.steps, 5))
    ms = 0.0
    for _ in range(steps):
        reset()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    w1 = np.array([s.windows for s in sims])
    units = float(((w1 - w0) * T).sum())
    launches = int(max(w1 - w0))
    achieved = units * (8 * S + 52) / (ms / 1e3) / 1e9
    achieved36 = units * (8 * S + 36) / (ms / 1e3) / 1e9
    blk, _, tune = batch.info
    tr = profile_traffic("step_kernel_batch_flow_config4_32rep" if flow else "step_kernel_batch_config4_32rep")
    # captured on 32 replicates (units_per_launch tets); traffic grows with the tets of a launch
    traffic = tr["bytes_per_launch"] / tr["units_per_launch"] * float(T.sum()) if tr else None
    out = {"value": units / (ms / 1e3), "unit": UNIT, "replicates": len(sims), "tets": int(T.sum()),
           "kernel": "specialised" if batch.specialized else "generic",
           "launch_form": "flow per L2-sized group of replicates" if flow else "one launch per window",
           "tets_min": int(T.min()), "tets_max": int(T.max()), "ms_per_step": ms / steps, "steps": steps,
           "windows_per_step_max": launches / steps, "block": blk, "autotune_ms_per_window": tune,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "bytes_per_tet_update": 8 * S + 52, "achieved_fixed_point": achieved36,
                        "frac_fixed_point": achieved36 / peak, "bytes_per_tet_update_fixed_point": 8 * S + 36,
                        "traffic": traffic,
                        "traffic_note": "ncu DRAM bytes per window on 32 replicates, scaled by tets",
                        "traffic_per_tet_update": (tr["bytes_per_launch"] / tr["units_per_launch"]) if tr else None},
           "setup_s": setup_s, "l2": "working set > L2; also flushed before each step",
           "step": "one batched run of 20 ms per member from its initial counts (reset outside the events)"}
    batch.close()
    for s in sims:
        s.close()
    return out


def measure_dendrite(args, capi, I, torch, peak):
    """Plain form on the dendrite workload: ~1M tets, 20-species calcium
    network with masked influx, tau = 3.3 us. One step is the configured run:
    --dendrite-ms of simulated time (default 50 ms, about 15,000 windows) from
    the initial counts, reset outside the timed region. Its counts and tables
    (~210 MB) exceed L2, so this is the HBM-bound case."""
    t0 = time.perf_counter()
    w = I.config3()
    stream = torch.cuda.current_stream()
    sim = capi.from_workload(w, cuda_stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    t_step = args.dendrite_ms * 1e-3
    host_in = torch.from_numpy(np.ascontiguousarray(w.counts, np.int32)).pin_memory().numpy()

    def step():
        sim.run(sim.time + t_step)

    capi.steps_set_counts_all(sim._sim, host_in)
    step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    w0, _ = capi.steps_get_windows(sim._sim)
    steps = 2
    ms = 0.0
    for _ in range(steps):
        capi.steps_set_counts_all(sim._sim, host_in)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    w1, _ = capi.steps_get_windows(sim._sim)
    windows = w1 - w0
    S = w.model.n_species
    kernel_s = (ms / 1e3) / windows
    prefix, form_keys = launch_form(sim)
    tr = profile_traffic(prefix + "_dendrite")
    out = {"value": w.n_tets * windows / (ms / 1e3), "unit": UNIT, "workload": w.name, "tets": w.n_tets,
           "form": "plain", "kernel": "specialised" if sim.specialized else "generic", **form_keys,
           "species": S, "reactions": w.model.n_reac, "tau_us": sim.tau * 1e6, "sim_ms_per_step": args.dendrite_ms,
           "windows_per_step": windows / steps, "ms_per_step": ms / steps, "steps": steps,
           "roofline": roofline(S, bool(w.reac_masks), w.n_tets, kernel_s, peak, "measured", tr, None, False),
           "setup_s": setup_s, "l2": "working set > L2; also flushed before each step",
           "step": "steps_run over sim_ms_per_step from the initial counts (reset outside the events)"}
    sim.close()
    return out


def measure_cuboid(args, capi, I, torch):
    """Plain form on the 1,920-tet cuboid (A + B <-> C, tau = 0.74 ms): the
    launch-bound case. One step is the configured run, 10 ms of simulated time
    (13 full windows and a shortened one) from the initial counts, reset
    outside the timed region."""
    w = I.config1()
    stream = torch.cuda.current_stream()
    sim = capi.from_workload(w, cuda_stream=stream.cuda_stream)
    t_step = w.t_end
    host_in = np.ascontiguousarray(w.counts, np.int32)

    def step():
        sim.run(sim.time + t_step)

    for _ in range(3):
        capi.steps_set_counts_all(sim._sim, host_in)
        step()
    torch.cuda.synchronize()
    w0, _ = capi.steps_get_windows(sim._sim)
    steps = max(5, min(args.steps, 20))
    ms = 0.0
    for _ in range(steps):
        capi.steps_set_counts_all(sim._sim, host_in)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    w1, _ = capi.steps_get_windows(sim._sim)
    windows = w1 - w0
    out = {"value": w.n_tets * windows / (ms / 1e3), "unit": UNIT, "workload": w.name, "tets": w.n_tets,
           "form": "plain", "kernel": "specialised" if sim.specialized else "generic",
           "sim_ms_per_step": t_step * 1e3, "windows_per_step": windows / steps, "us_per_window": 1e3 * ms / windows,
           "step": "steps_run over sim_ms_per_step from the initial counts (reset outside the events)",
           "bound": "launch/latency (1,920 tets fill 8 blocks of 256)"}
    sim.close()
    return out


def measure_dendrite_recording(args, capi, I, torch):
    """Dendrite with a time-varying influx and recording: the influx rate
    follows a synthetic burst train, changed every 1 ms of simulated time
    (k = k0 (1 + 4 exp(-(t mod 5 ms) / 1 ms))); Ca is recorded every 20 us at
    1% of the tets (device-side snapshots). One step = 2 ms of simulated time."""
    w = I.config3()
    stream = torch.cuda.current_stream()
    sim = capi.from_workload(w, cuda_stream=stream.cuda_stream)
    influx = w.model.n_reac - 1
    k0 = float(w.model.k[influx])
    rng = np.random.default_rng(7)
    rec_tets = np.sort(rng.choice(w.n_tets, w.n_tets // 100, replace=False)).astype(np.int32)
    rec_species = np.array([w.model.names.index("Ca")], np.int32)
    dt_rec, seg = 20e-6, 1e-3
    per_seg = int(seg / dt_rec + 1e-9)
    buf = torch.empty((per_seg, 1, rec_tets.size), dtype=torch.int32, device="cuda")

    def step():
        n = 0
        for _ in range(2):
            t = sim.time
            sim.set_reac_rate(influx, k0 * (1.0 + 4.0 * math.exp(-((t % 5e-3) / 1e-3))))
            n += sim.run_record(t + seg, dt_rec, rec_species, rec_tets, buf.data_ptr(), per_seg)
        return n

    step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    w0, _ = capi.steps_get_windows(sim._sim)
    steps = 3
    t0 = time.perf_counter()
    nrec = 0
    for _ in range(steps):
        nrec += step()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    w1, _ = capi.steps_get_windows(sim._sim)
    out = {"value": w.n_tets * (w1 - w0) / wall, "unit": UNIT, "workload": w.name, "form": "plain",
           "timing": "wall clock (host-driven rate changes and recordings)",
           "sim_ms_per_step": 2.0, "windows_per_step": (w1 - w0) / steps, "recordings_per_step": nrec / steps,
           "recorded_tets": int(rec_tets.size), "dt_rec_us": dt_rec * 1e6, "rate_segment_ms": seg * 1e3,
           "ms_per_step": 1e3 * wall / steps}
    sim.close()
    return out


def measure_served(args, capi, I):
    """Served form: a Poisson stream (50 jobs/s) of jobs from the config 1-3
    generators, 2k-1M tets, t_end 1-100 ms, admitted by a device-memory
    budget, continuously batched (jobs grouped by model structure, each group
    on the kernel compiled for its model when its prototype was created); the
    same jobs alone in plain form, one after another. Then the same jobs at
    saturation: all queued at once, served both ways."""
    import torch
    from paper_1610_02258_gb300 import serve
    jobs = I.served_jobs(args.served_jobs, rate=50.0, seed=21)
    protos = serve.Prototypes()
    t0 = time.perf_counter()
    for j in jobs:
        protos.sim(j.kind, j.size)
    setup_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.8, 64 << 30))
    keys = ("throughput", "p50_s", "p99_s", "mean_s", "makespan_s")
    out = {"jobs": len(jobs), "rate_jobs_per_s": 50.0, "hbm_budget_bytes": budget, "unit": UNIT,
           "prototype_setup_s": setup_s, "kernel": "specialised per model structure (compiled with the prototypes)"}
    same = True
    for label, realtime in (("", True), ("saturated_", False)):
        srv = serve.Server(hbm_budget=budget, max_jobs=128, wave_windows=32)
        srv.protos = protos
        mixed = srv.run(jobs, realtime=realtime)
        s_mixed = serve.summarize(mixed, srv.stats["makespan"])
        alone, mk = serve.run_alone(jobs, protos, realtime=realtime)
        s_alone = serve.summarize(alone, mk)
        same = same and all(np.array_equal(mixed[j.job_id].counts, alone[j.job_id].counts) for j in jobs)
        out[label + "continuous"] = {k: s_mixed[k] for k in keys}
        out[label + "continuous"].update({"max_active": srv.stats["max_active"], "waves": srv.stats["waves"],
                                          "batch_rebuilds": srv.stats["batch_rebuilds"]})
        out[label + "alone_plain"] = {k: s_alone[k] for k in keys}
    out["saturated_note"] = "every job queued at time 0 (arrivals faster than capacity)"
    out["results_identical"] = bool(same)
    protos.close()
    return out


def measure_sweeps(args, capi, I, torch):
    """The paper's density and mesh-coarseness experiments (§3.1) on the box:
    the benchmark network at 0.1x, 1x and 10x its densities, and the box
    meshed with 8, 17 and 26 cubes across (h = 10/8, 10/17, 10/26 um; about
    31k, 295k and 1.05M tets) at the benchmark densities. Each point: one
    20 ms run from the initial counts, device time per window."""
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {"density": [], "mesh": []}

    def timed(w):
        counts = np.ascontiguousarray(w.counts, np.int32)
        sim = capi.from_workload(w, cuda_stream=stream.cuda_stream)
        sim.set_counts(counts)
        sim.run(sim.time + 20e-3)  # warm: the first run also picks the launch form
        ms, wins = 0.0, 0
        for _ in range(2):
            sim.set_counts(counts)
            flush.zero_()
            w0 = sim.windows
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.run(sim.time + 20e-3)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            wins += sim.windows - w0
        out = {"tets": w.n_tets, "molecules_per_tet": float(counts.sum()) / w.n_tets, "tau_us": sim.tau * 1e6,
               "us_per_window": 1e3 * ms / wins, "value": w.n_tets * wins / (ms / 1e3), "unit": UNIT,
               "kernel": "specialised" if sim.specialized else "generic", **launch_form(sim)[1]}
        sim.close()
        return out

    base = I.config2()
    for scale in (0.1, 1.0, 10.0):
        r = timed(base if scale == 1.0 else I.config2(density_scale=scale))
        r["density_scale"] = scale
        res["density"].append(r)
    for n in (8, 17, 26):
        w = base if n == 17 else I.config2(nx=10 * n, ny=n, nz=n, h=10.0 / n * I.UM)
        r = timed(w)
        r["cubes_across"] = n
        res["mesh"].append(r)
    return res


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle.build import build as build_oracle
    build_oracle()
    from paper_1610_02258_gb300 import inputs as I
    w = I.config2()
    windows = 5
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_rate(w, 1, threads=cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(w, windows, threads=cores)
        times.append(dt)
    value = w.n_tets * windows * args.steps / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "tets": w.n_tets, "species": w.model.n_species,
                   "reactions": w.model.n_reac, "sample": f"{windows} full windows per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{windows} full windows of {w.name} per step, C oracle on {cores} threads "
                                   "(threaded windows, the serial result bit for bit)",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi
    from paper_1610_02258_gb300 import inputs as I

    if args.workload == "dendrite":
        w = I.config3(seed=replica_seed(rank))
    else:
        w = I.config2(seed=replica_seed(rank))
    stream = torch.cuda.current_stream()
    sim = capi.from_workload(w, cuda_stream=stream.cuda_stream, block=args.block,
                             flow={"auto": None, "on": True, "off": False}[args.flow])
    tau = sim.tau
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    t_step = args.sim_ms * 1e-3 if args.sim_ms > 0 else w.t_end
    # pinned host copy of the initial counts: every step is the configured run,
    # t_step of simulated time from the initial state
    host_in = torch.from_numpy(np.ascontiguousarray(w.counts, np.int32)).pin_memory().numpy()

    def reset():
        capi.steps_set_counts_all(sim._sim, host_in)

    def step():
        sim.run(sim.time + t_step)

    for _ in range(args.warmup):
        reset()
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    w0, l0 = capi.steps_get_windows(sim._sim)
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        reset()  # outside the events, like the L2 flush
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    w1, l1 = capi.steps_get_windows(sim._sim)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    windows = w1 - w0
    units = w.n_tets * windows
    if world > 1:
        ms_all, units_all = reduce_over_ranks(ms, float(units))
    else:
        ms_all, units_all = ms, float(units)
    value = units_all / (ms_all / 1e3)

    # end to end through the C ABI with host buffers
    # pinned host buffers (page-locked, so the copies run at full DMA speed)
    host_out = torch.empty(host_in.shape, dtype=torch.int32).pin_memory().numpy()
    e2e_steps = max(3, min(args.steps, 10))
    t_e = []
    we0, _ = capi.steps_get_windows(sim._sim)
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        capi.steps_set_counts_all(sim._sim, host_in)
        step()
        capi.steps_get_counts_all(sim._sim, w.model.n_species, w.n_tets, host_out)
        t_e.append(time.perf_counter() - t0)
    we1, _ = capi.steps_get_windows(sim._sim)
    e2e_units = w.n_tets * (we1 - we0)
    e2e = {"value": e2e_units / sum(t_e), "unit": UNIT, "h2d_bytes_per_step": int(host_in.nbytes),
           "d2h_bytes_per_step": int(host_out.nbytes), "host_memory": "pinned"}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return
    S = w.model.n_species
    kernel_s = (ms / 1e3) / windows
    peak, peak_kind = _peaks()
    prefix, form_keys = launch_form(sim)
    tr = profile_traffic(prefix + ("_dendrite" if args.workload == "dendrite" else "_config2"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+fp32", "data": "synthetic",
        "config": {"workload": w.name, "tets": w.n_tets, "species": S, "reactions": w.model.n_reac,
                   "tau_ms": tau * 1e3, "sim_ms_per_step": t_step * 1e3,
                   "windows_per_step": windows / args.steps, "form": "plain",
                   "kernel": "specialised" if sim.specialized else "generic", **form_keys,
                   "l2": "flushed before each timed step (256 MiB write, outside the events)",
                   "step": "steps_run over sim_ms_per_step from the initial counts (reset outside the events)",
                   "parallelism": f"replicas{world}"},
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "roofline": roofline(S, bool(w.reac_masks), w.n_tets, kernel_s, peak, peak_kind, tr,
                             clk["sm_mhz"] if clk else None, issue_bound=args.workload != "dendrite"),
        "clocks": clk,
    }
    if world == 1 and args.sweep:
        line["sweeps"] = measure_sweeps(args, capi, I, torch)
    if world == 1 and not args.no_forms and args.workload == "irregular-box":
        line["forms"] = {"plain": {"value": value, "unit": UNIT, "workload": w.name},
                         "plain_cuboid": measure_cuboid(args, capi, I, torch),
                         "plain_dendrite": measure_dendrite(args, capi, I, torch, peak) if args.dendrite_ms > 0 else None,
                         "dendrite_influx_recording": (measure_dendrite_recording(args, capi, I, torch)
                                                       if args.dendrite_ms > 0 else None),
                         "batched": measure_batched(args, capi, I, torch, peak) if args.batch_replicates > 0 else None,
                         "batched_flow": (measure_batched(args, capi, I, torch, peak, flow=True)
                                          if args.batch_replicates > 0 else None),
                         "served": measure_served(args, capi, I) if args.served_jobs > 0 else None}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, 4 * args.cpu_windows, max(5, args.cpu_windows // 4))
        if args.dendrite_ms > 0 and args.workload == "irregular-box":
            line["cpu_baseline"]["dendrite"] = cpu_baseline_dendrite(I, 20, 5)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-windows", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--batch-replicates", type=int, default=256)
    ap.add_argument("--block", type=int, default=256, choices=[64, 128, 256, 512],
                    help="tile size (threads per block) of the plain run")
    ap.add_argument("--flow", choices=["auto", "on", "off"], default="auto",
                    help="launch form of the plain run's full windows: tuned on the first run (auto), flow launches "
                         "(on) or window launches (off)")
    ap.add_argument("--served-jobs", type=int, default=1000)
    ap.add_argument("--sweep", action="store_true",
                    help="add the density (0.1x/1x/10x) and mesh-size (8/17/26 cubes across) sweeps of the box")
    ap.add_argument("--workload", default="irregular-box", choices=["irregular-box", "dendrite"],
                    help="plain workload of the headline line: the 294,780-tet jittered box (default) or the "
                         "1.03M-tet dendrite")
    ap.add_argument("--sim-ms", type=float, default=0.0,
                    help="simulated ms per step of the headline workload (default: its t_end)")
    ap.add_argument("--dendrite-ms", type=float, default=50.0,
                    help="simulated ms per step of the dendrite measurement, from its initial counts (0 = skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
