"""Served form: continuous batching of simulation jobs on one GPU.

The scheduling is the library's (steps_server_*): jobs are clones of a
prototype simulation, admitted first come first served when a slot is free
and their device memory fits the budget, advanced together in rounds (one
batched run moves every job by up to `wave_windows` windows of its own
length, stopping on its window grid or at its t_end) and retired between
rounds. This module supplies the job stream (mesh generator, size, seed,
t_end, arrival time), feeds arrived jobs to the server and records
latencies. Because every draw is addressed by (job seed, window, tet), a
job's result is the same bits whether it runs alone or in any mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import capi
from . import inputs as I


@dataclass
class JobResult:
    job_id: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    tets: int = 0
    windows: int = 0
    counts: np.ndarray = None

    @property
    def latency(self):
        return self.finish - self.arrival


class Prototypes:
    """One simulation per (generator, size bucket): meshes and tables are built
    once and cloned per job. specialize = 1 compiles the step kernels for each
    model structure here, when the first prototype of that structure is
    created (clones and batches of the same structure reuse them)."""

    def __init__(self, stream=None, specialize: int = 1):
        self.stream = stream
        self.specialize = specialize
        self._w = {}
        self._sim = {}

    def workload(self, kind, size):
        key = (kind, size)
        if key not in self._w:
            self._w[key] = I.make_job_workload(kind, size, seed=1, t_end=1e-3)
        return self._w[key]

    def sim(self, kind, size):
        key = (kind, size)
        if key not in self._sim:
            w = self.workload(kind, size)
            s = capi.Simulation(w.verts, w.tets, w.model, 1, cuda_stream=self.stream, specialize=self.specialize)
            for r, m in w.reac_masks.items():
                s.set_reac_mask(r, m)
            self._sim[key] = s
        return self._sim[key]

    def device_bytes(self):
        return sum(s.device_bytes for s in self._sim.values())

    def close(self):
        for s in self._sim.values():
            s.close()
        self._sim.clear()


def _new_job_sim(protos, spec):
    proto = protos.sim(spec.kind, spec.size)
    w = protos.workload(spec.kind, spec.size)
    s = proto.clone(spec.seed, protos.stream)
    s.set_counts(w.counts)
    return s


class Server:
    """Feeds a stream of jobs, by arrival time, to the library's job server
    (steps_server_*: admission by slots and device-memory budget, batched
    rounds, retirement; all of it native) and collects each job's result and
    latency. The budget covers the prototypes and the running jobs."""

    def __init__(self, hbm_budget: int, max_jobs: int = 64, wave_windows: int = 16, block: int = 256,
                 cuda_stream=None, specialize: int = 1):
        self.budget = int(hbm_budget)
        self.max_jobs = max_jobs
        self.wave_windows = wave_windows
        self.block = block
        self.stream = cuda_stream
        # batches re-form as jobs come and go: a fixed block size (no autotuning windows on
        # every re-formed batch); by default jobs are grouped by model structure and each
        # group runs the kernel compiled for its model when its prototype was created
        # (specialize = 1), so nothing is compiled between requests; -1 runs one batch of
        # every job on the generic kernel
        self.specialize = specialize
        self.protos = Prototypes(cuda_stream, specialize=1 if specialize >= 0 else 0)
        self.stats = {"waves": 0, "max_active": 0, "batch_rebuilds": 0, "launches": 0, "admit_waits": 0}

    def run(self, jobs, realtime: bool = True):
        """Serve `jobs` (list of JobSpec, by arrival). Returns {job_id: JobResult}.
        realtime = False queues every job at time 0 (latency counts from there)."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        results = {j.job_id: JobResult(j.job_id, j.arrival if realtime else 0.0) for j in jobs}
        for j in pending:  # meshes and tables of every kind of job, before the clock starts
            self.protos.sim(j.kind, j.size)
        native = capi.NativeServer(device_budget=max(1, self.budget - self.protos.device_bytes()),
                                   max_jobs=self.max_jobs, wave_windows=self.wave_windows, block=self.block,
                                   specialize=self.specialize, cuda_stream=self.stream)
        try:
            outstanding = {}  # native job id -> JobSpec
            t0 = time.perf_counter()
            nxt = 0
            while nxt < len(pending) or outstanding:
                now = time.perf_counter() - t0
                while nxt < len(pending) and (not realtime or pending[nxt].arrival <= now):
                    spec = pending[nxt]
                    proto = self.protos.sim(spec.kind, spec.size)
                    w = self.protos.workload(spec.kind, spec.size)
                    outstanding[native.submit(proto, spec.seed, w.counts, spec.t_end)] = spec
                    results[spec.job_id].tets = proto.nt
                    nxt += 1
                if not outstanding:
                    if realtime and nxt < len(pending):
                        time.sleep(max(0.0, pending[nxt].arrival - (time.perf_counter() - t0)))
                    continue
                running, _ = native.step()
                st = native.stats()
                self.stats["max_active"] = max(self.stats["max_active"], running)
                if st["queued"] > 0 and running < self.max_jobs:
                    self.stats["admit_waits"] += 1  # the memory budget held jobs back
                now = time.perf_counter() - t0
                for nid in list(outstanding):
                    state, windows, _ = native.state(nid)
                    r = results[outstanding[nid].job_id]
                    if state >= 1 and r.start == 0.0:
                        r.start = now
                    if state == 2:
                        r.counts = native.take_result(nid)
                        r.windows = windows
                        r.finish = now
                        del outstanding[nid]
            self.stats["makespan"] = time.perf_counter() - t0
            st = native.stats()
            self.stats["waves"] = st["rounds"]
            self.stats["batch_rebuilds"] = st["rebuilds"]
            self.stats["launches"] = st["launches"]
        finally:
            native.close()
        return results

    def close(self):
        self.protos.close()


def run_alone(jobs, protos: Prototypes, realtime: bool = True):
    """Each job alone in plain form, one after another in arrival order
    (realtime = False: every job queued at time 0)."""
    pending = sorted(jobs, key=lambda j: j.arrival)
    results = {}
    t0 = time.perf_counter()
    for spec in pending:
        now = time.perf_counter() - t0
        if realtime and spec.arrival > now:
            time.sleep(spec.arrival - now)
        r = JobResult(spec.job_id, spec.arrival if realtime else 0.0, start=time.perf_counter() - t0)
        s = _new_job_sim(protos, spec)
        s.run(spec.t_end)
        r.counts = s.get_counts()
        r.windows = s.windows
        r.tets = s.nt
        r.finish = time.perf_counter() - t0
        s.close()
        results[spec.job_id] = r
    return results, time.perf_counter() - t0


def summarize(results, makespan):
    lat = np.array([r.latency for r in results.values()])
    updates = float(sum(r.tets * r.windows for r in results.values()))
    return {"jobs": len(results), "tet_updates": updates, "makespan_s": makespan,
            "throughput": updates / makespan if makespan > 0 else 0.0,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}
