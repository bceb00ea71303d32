"""Served form: continuous batching of simulation jobs on one GPU.

Host-side scheduling only; every window runs in the CUDA library through the
C ABI (batched launches). Jobs (mesh generator, size, seed, t_end) arrive
over time; a job is admitted, first come first served, when its device
memory fits the budget and a slot is free; its counts and random-number
state stay resident on the device until it finishes. The server advances all
admitted jobs together in waves: each wave is one batched run that moves
every job by up to `wave_windows` windows of its own length, stopping on the
job's window grid (so no extra shortened windows are inserted) or at its
t_end. Jobs that finish leave between waves and their memory is freed; jobs
that arrived meanwhile join the next wave. Because every draw is addressed by
(job seed, window, tet), a job's result is the same bits whether it runs
alone or in any mix.
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
    once and cloned per job."""

    def __init__(self, stream=None):
        self.stream = stream
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
            s = capi.Simulation(w.verts, w.tets, w.model, 1, cuda_stream=self.stream)
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
    def __init__(self, hbm_budget: int, max_jobs: int = 64, wave_windows: int = 16, block: int = 256,
                 cuda_stream=None, specialize: int = -1):
        self.budget = int(hbm_budget)
        self.max_jobs = max_jobs
        self.wave_windows = wave_windows
        self.block = block
        self.stream = cuda_stream
        # batches re-form as jobs come and go: by default a fixed block size (no autotuning
        # windows on every re-formed batch) and the generic batched kernel (no run-time
        # compilation between requests)
        self.specialize = specialize
        self.protos = Prototypes(cuda_stream)
        self.stats = {"waves": 0, "max_active": 0, "batch_rebuilds": 0, "launches": 0, "admit_waits": 0}

    def run(self, jobs, realtime: bool = True):
        """Serve `jobs` (list of JobSpec, by arrival). Returns {job_id: JobResult}."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        results = {j.job_id: JobResult(j.job_id, j.arrival) for j in jobs}
        active = []  # (spec, sim)
        batch = None
        members_key = None
        t0 = time.perf_counter()
        nxt = 0
        while nxt < len(pending) or active:
            now = time.perf_counter() - t0
            # admission: arrived jobs, first come first served, by memory budget and slots
            used = self.protos.device_bytes() + sum(s.device_bytes for _, s in active)
            while nxt < len(pending) and (not realtime or pending[nxt].arrival <= now) and len(active) < self.max_jobs:
                spec = pending[nxt]
                proto = self.protos.sim(spec.kind, spec.size)
                need = proto.device_bytes
                used = self.protos.device_bytes() + sum(s.device_bytes for _, s in active)
                if active and used + need > self.budget:
                    self.stats["admit_waits"] += 1
                    break
                s = _new_job_sim(self.protos, spec)
                results[spec.job_id].start = time.perf_counter() - t0
                results[spec.job_id].tets = s.nt
                active.append((spec, s))
                nxt += 1
            if not active:
                if realtime and nxt < len(pending):
                    time.sleep(max(0.0, pending[nxt].arrival - (time.perf_counter() - t0)))
                continue
            self.stats["max_active"] = max(self.stats["max_active"], len(active))
            key = tuple(id(s) for _, s in active)
            if key != members_key:
                if batch is not None:
                    self.stats["launches"] += batch.info[1]
                    batch.close()
                batch = capi.Batch([s for _, s in active], block=self.block, cuda_stream=self.stream,
                                   specialize=self.specialize)
                members_key = key
                self.stats["batch_rebuilds"] += 1
            # one wave: every job by up to wave_windows windows on its own grid
            targets = []
            for spec, s in active:
                t = s.time
                tgt = t + self.wave_windows * s.tau if np.isfinite(s.tau) else spec.t_end
                targets.append(min(spec.t_end, tgt))
            batch.run(targets)
            self.stats["waves"] += 1
            # retire finished jobs
            keep = []
            for spec, s in active:
                if s.time >= spec.t_end - 1e-12 * max(spec.t_end, 1e-30):
                    r = results[spec.job_id]
                    r.counts = s.get_counts()
                    r.windows = s.windows
                    r.finish = time.perf_counter() - t0
                    s.close()
                else:
                    keep.append((spec, s))
            if len(keep) != len(active):
                if batch is not None:
                    self.stats["launches"] += batch.info[1]
                    batch.close()
                batch = None
                members_key = None
            active = keep
        if batch is not None:
            self.stats["launches"] += batch.info[1]
            batch.close()
        self.stats["makespan"] = time.perf_counter() - t0
        return results

    def close(self):
        self.protos.close()


def run_alone(jobs, protos: Prototypes, realtime: bool = True):
    """Each job alone in plain form, one after another in arrival order."""
    pending = sorted(jobs, key=lambda j: j.arrival)
    results = {}
    t0 = time.perf_counter()
    for spec in pending:
        now = time.perf_counter() - t0
        if realtime and spec.arrival > now:
            time.sleep(spec.arrival - now)
        r = JobResult(spec.job_id, spec.arrival, start=time.perf_counter() - t0)
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
