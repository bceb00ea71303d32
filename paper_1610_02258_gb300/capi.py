"""Python binding of the C ABI in include/steps_gpu.h (argument marshalling
only: every step of the simulation runs in the CUDA library).

The functions keep the C names. Handles are opaque ctypes pointers; arrays
are numpy arrays (host) converted to the C layout. A negative return code
raises StepsError with the library's message. If the compiled library is
absent this module raises on import: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsteps_gpu.so")

STEPS_OCC_MEAN, STEPS_OCC_END = 1, 0
STEPS_REORDER_NONE, STEPS_REORDER_MORTON, STEPS_REORDER_RCM = 0, 1, 2
STEPS_LEAVE_EULER, STEPS_LEAVE_EXP = 0, 1

ERRORS = {-1: "STEPS_ERR_ARG", -2: "STEPS_ERR_MESH", -3: "STEPS_ERR_MODEL", -4: "STEPS_ERR_OOM",
          -5: "STEPS_ERR_CUDA", -6: "STEPS_ERR_TIMEOUT", -7: "STEPS_ERR_STATE"}

# every exported symbol of include/steps_gpu.h
EXPORTS = [
    "steps_options_default", "steps_mesh_create", "steps_mesh_destroy", "steps_mesh_num_tets",
    "steps_model_create", "steps_model_destroy", "steps_sim_create", "steps_sim_destroy",
    "steps_set_counts", "steps_get_counts", "steps_set_counts_all", "steps_get_counts_all",
    "steps_set_reac_mask", "steps_run", "steps_get_time", "steps_get_tau", "steps_get_windows",
    "steps_last_error", "steps_debug_philox", "steps_debug_logf", "steps_run_noalloc",
    "steps_batch_options_default", "steps_batch_create", "steps_batch_destroy", "steps_batch_run",
    "steps_batch_info", "steps_sim_clone", "steps_sim_device_bytes", "steps_set_reac_rate", "steps_run_record",
    "steps_sim_specialized", "steps_sim_flow", "steps_batch_specialized", "steps_sim_shape",
    "steps_server_options_default", "steps_server_create", "steps_server_destroy", "steps_server_submit",
    "steps_server_step", "steps_server_job_state", "steps_server_take_result", "steps_server_stats",
    "steps_debug_host_tables", "steps_debug_wait", "steps_debug_flow_wait",
]


class StepsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class steps_options(ctypes.Structure):
    _fields_ = [("occupancy", ctypes.c_int32), ("reorder", ctypes.c_int32), ("block", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("specialize", ctypes.c_int32), ("leave_law", ctypes.c_int32),
                ("flow", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class steps_batch_options(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("specialize", ctypes.c_int32),
                ("flow", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class steps_server_options(ctypes.Structure):
    _fields_ = [("device_budget", ctypes.c_int64), ("max_jobs", ctypes.c_int32), ("wave_windows", ctypes.c_int32),
                ("block", ctypes.c_int32), ("specialize", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_1610_02258_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "steps_options_default": (None, [ctypes.POINTER(steps_options)]),
        "steps_mesh_create": (ctypes.c_int, [P, i64, P, i64, PP]),
        "steps_mesh_destroy": (None, [P]),
        "steps_mesh_num_tets": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64)]),
        "steps_model_create": (ctypes.c_int, [i32, P, i32, P, P, P, PP]),
        "steps_model_destroy": (None, [P]),
        "steps_sim_create": (ctypes.c_int, [P, P, u64, ctypes.POINTER(steps_options), P, PP]),
        "steps_sim_destroy": (None, [P]),
        "steps_set_counts": (ctypes.c_int, [P, i32, P]),
        "steps_get_counts": (ctypes.c_int, [P, i32, P]),
        "steps_set_counts_all": (ctypes.c_int, [P, P]),
        "steps_get_counts_all": (ctypes.c_int, [P, P]),
        "steps_set_reac_mask": (ctypes.c_int, [P, i32, P]),
        "steps_run": (ctypes.c_int, [P, ctypes.c_double]),
        "steps_get_time": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double)]),
        "steps_get_tau": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double)]),
        "steps_get_windows": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "steps_last_error": (ctypes.c_char_p, []),
        "steps_debug_philox": (ctypes.c_int, [u64, P, i64, P]),
        "steps_debug_logf": (ctypes.c_int, [P, i64, P]),
        "steps_debug_wait": (ctypes.c_int, [ctypes.c_int32, i64]),
        "steps_debug_flow_wait": (ctypes.c_int, [ctypes.c_int32, i64]),
        "steps_run_noalloc": (ctypes.c_int, [P, P, ctypes.c_double]),
        "steps_batch_options_default": (None, [ctypes.POINTER(steps_batch_options)]),
        "steps_batch_create": (ctypes.c_int, [P, i32, ctypes.POINTER(steps_batch_options), P, PP]),
        "steps_batch_destroy": (None, [P]),
        "steps_batch_run": (ctypes.c_int, [P, P]),
        "steps_batch_info": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_float)]),
        "steps_sim_clone": (ctypes.c_int, [P, u64, P, PP]),
        "steps_sim_device_bytes": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64)]),
        "steps_set_reac_rate": (ctypes.c_int, [P, i32, ctypes.c_double]),
        "steps_sim_specialized": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
        "steps_sim_flow": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
        "steps_batch_specialized": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
        "steps_sim_shape": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
        "steps_debug_host_tables": (ctypes.c_int, [P, P, i32, ctypes.POINTER(ctypes.c_double), P, P]),
        "steps_server_options_default": (None, [ctypes.POINTER(steps_server_options)]),
        "steps_server_create": (ctypes.c_int, [ctypes.POINTER(steps_server_options), P, PP]),
        "steps_server_destroy": (None, [P]),
        "steps_server_submit": (ctypes.c_int, [P, P, u64, P, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]),
        "steps_server_step": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "steps_server_job_state": (ctypes.c_int, [P, i64, ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
        "steps_server_take_result": (ctypes.c_int, [P, i64, P]),
        "steps_server_stats": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
        "steps_run_record": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_double, i32, P, i32, P, P, i64,
                                            ctypes.POINTER(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def _check(rc):
    if rc < 0:
        raise StepsError(rc, lib.steps_last_error().decode(errors="replace"))
    return rc


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def steps_options_default():
    o = steps_options()
    lib.steps_options_default(ctypes.byref(o))
    return o


def steps_mesh_create(verts, tets):
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tets, np.int32)
    h = ctypes.c_void_p()
    _check(lib.steps_mesh_create(_ptr(v), v.shape[0], _ptr(t), t.shape[0], ctypes.byref(h)))
    return h


def steps_mesh_destroy(h):
    lib.steps_mesh_destroy(h)


def steps_mesh_num_tets(h):
    n = ctypes.c_int64()
    _check(lib.steps_mesh_num_tets(h, ctypes.byref(n)))
    return n.value


def steps_model_create(diff, lhs, rhs, k):
    d = np.ascontiguousarray(diff, np.float64)
    S = d.shape[0]
    lh = np.ascontiguousarray(lhs, np.int32).reshape(-1, S)
    R = lh.shape[0]
    rh = np.ascontiguousarray(rhs, np.int32).reshape(R, S)
    kk = np.ascontiguousarray(k, np.float64).reshape(R)
    h = ctypes.c_void_p()
    _check(lib.steps_model_create(S, _ptr(d), R, _ptr(lh) if R else None, _ptr(rh) if R else None,
                                  _ptr(kk) if R else None, ctypes.byref(h)))
    return h


def steps_model_destroy(h):
    lib.steps_model_destroy(h)


def steps_sim_create(mesh, model, seed, opt=None, cuda_stream=None):
    h = ctypes.c_void_p()
    _check(lib.steps_sim_create(mesh, model, ctypes.c_uint64(seed), ctypes.byref(opt) if opt is not None else None,
                                ctypes.c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(h)))
    return h


def steps_sim_clone(src, seed, cuda_stream=None):
    h = ctypes.c_void_p()
    _check(lib.steps_sim_clone(src, ctypes.c_uint64(seed), ctypes.c_void_p(cuda_stream) if cuda_stream else None,
                               ctypes.byref(h)))
    return h


def steps_sim_device_bytes(sim):
    n = ctypes.c_int64()
    _check(lib.steps_sim_device_bytes(sim, ctypes.byref(n)))
    return n.value


def steps_sim_destroy(h):
    lib.steps_sim_destroy(h)


def steps_set_counts(sim, species, counts):
    c = np.ascontiguousarray(counts, np.int32)
    _check(lib.steps_set_counts(sim, species, _ptr(c)))


def steps_get_counts(sim, species, nt):
    out = np.empty(nt, np.int32)
    _check(lib.steps_get_counts(sim, species, _ptr(out)))
    return out


def steps_set_counts_all(sim, counts):
    c = np.ascontiguousarray(counts, np.int32)
    _check(lib.steps_set_counts_all(sim, _ptr(c)))


def steps_get_counts_all(sim, n_species, nt, out=None):
    if out is None:
        out = np.empty((n_species, nt), np.int32)
    _check(lib.steps_get_counts_all(sim, _ptr(out)))
    return out


def steps_set_reac_mask(sim, reac, active):
    if active is None:
        _check(lib.steps_set_reac_mask(sim, reac, None))
    else:
        a = np.ascontiguousarray(active, np.uint8)
        _check(lib.steps_set_reac_mask(sim, reac, _ptr(a)))


def steps_run(sim, t_end):
    _check(lib.steps_run(sim, float(t_end)))


def steps_run_noalloc(sim, d_counts_ptr, t_end):
    """Advance on caller-owned device counts (an int pointer to [S * nt] int32,
    species-major, original tet order), allocating nothing."""
    _check(lib.steps_run_noalloc(sim, ctypes.c_void_p(int(d_counts_ptr)), float(t_end)))


def steps_set_reac_rate(sim, reac, k):
    _check(lib.steps_set_reac_rate(sim, int(reac), float(k)))


def steps_run_record(sim, t_end, dt_rec, species, tets, d_out_ptr, max_records):
    """Records into caller-owned device memory at d_out_ptr (int32,
    [max_records][len(species)][len(tets)]); returns the number of recordings."""
    sp = np.ascontiguousarray(species, np.int32)
    tt = np.ascontiguousarray(tets, np.int32)
    n = ctypes.c_int64(0)
    _check(lib.steps_run_record(sim, float(t_end), float(dt_rec), sp.size, _ptr(sp), tt.size, _ptr(tt),
                                ctypes.c_void_p(d_out_ptr), int(max_records), ctypes.byref(n)))
    return n.value


def steps_sim_specialized(sim):
    v = ctypes.c_int32(0)
    _check(lib.steps_sim_specialized(sim, ctypes.byref(v)))
    return bool(v.value)


def steps_sim_flow(sim):
    """(tile size of the flow launches, 0 for window launches; [ms per window of window
    launches, flow at the simulation's block, flow at 512] from the tuning run)."""
    v = ctypes.c_int32(0)
    ms = (ctypes.c_float * 3)()
    _check(lib.steps_sim_flow(sim, ctypes.byref(v), ms))
    return int(v.value), [float(x) for x in ms]


def steps_get_time(sim):
    t = ctypes.c_double()
    _check(lib.steps_get_time(sim, ctypes.byref(t)))
    return t.value


def steps_get_tau(sim):
    t = ctypes.c_double()
    _check(lib.steps_get_tau(sim, ctypes.byref(t)))
    return t.value


def steps_get_windows(sim):
    w, l = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.steps_get_windows(sim, ctypes.byref(w), ctypes.byref(l)))
    return w.value, l.value


def steps_debug_philox(seed, ctr):
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    _check(lib.steps_debug_philox(ctypes.c_uint64(seed), _ptr(c), c.shape[0], _ptr(out)))
    return out


def steps_debug_host_tables(mesh, model, nt, reorder=STEPS_REORDER_MORTON):
    """(tau, thresholds [nt, 4] in the caller's tet order, device order perm)."""
    tau = ctypes.c_double()
    thr = np.empty((nt, 4), np.uint32)
    perm = np.empty(nt, np.int32)
    _check(lib.steps_debug_host_tables(mesh, model, int(reorder), ctypes.byref(tau), _ptr(thr), _ptr(perm)))
    return tau.value, thr, perm


def steps_debug_logf(x):
    a = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(a)
    _check(lib.steps_debug_logf(_ptr(a), a.size, _ptr(out)))
    return out


def steps_debug_wait(deliver, limit_cycles):
    """The step kernel's bounded bulk-copy wait on its own: raises StepsError
    (code -6, STEPS_ERR_TIMEOUT) when the wait ran out."""
    _check(lib.steps_debug_wait(1 if deliver else 0, int(limit_cycles)))


def steps_debug_flow_wait(deliver, limit_cycles):
    """The flow launch's bounded wait for the tiles a tile depends on, on its
    own: raises StepsError (code -6, STEPS_ERR_TIMEOUT) when the wait ran out."""
    _check(lib.steps_debug_flow_wait(1 if deliver else 0, int(limit_cycles)))


def steps_batch_options_default():
    o = steps_batch_options()
    lib.steps_batch_options_default(ctypes.byref(o))
    return o


def steps_batch_create(sim_handles, opt=None, cuda_stream=None):
    arr = (ctypes.c_void_p * len(sim_handles))(*[h.value for h in sim_handles])
    h = ctypes.c_void_p()
    _check(lib.steps_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(sim_handles),
                                  ctypes.byref(opt) if opt is not None else None,
                                  ctypes.c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(h)))
    return h


def steps_batch_destroy(h):
    lib.steps_batch_destroy(h)


def steps_batch_run(batch, t_end):
    t = np.ascontiguousarray(t_end, np.float64)
    _check(lib.steps_batch_run(batch, _ptr(t)))


def steps_batch_info(batch):
    b, l = ctypes.c_int32(), ctypes.c_uint64()
    tm = (ctypes.c_float * 3)()
    _check(lib.steps_batch_info(batch, ctypes.byref(b), ctypes.byref(l), tm))
    return b.value, l.value, list(tm)


class Batch:
    """A batch over existing Simulation objects (kept alive by this object)."""

    def __init__(self, sims, block=0, use_graph=True, cuda_stream=None, specialize=0, flow=False):
        self.sims = list(sims)
        opt = steps_batch_options_default()
        opt.block = block
        opt.use_graph = 1 if use_graph else 0
        opt.specialize = int(specialize)
        opt.flow = 1 if flow else 0
        self._h = steps_batch_create([s._sim for s in self.sims], opt, cuda_stream)

    def run(self, t_end):
        t = np.broadcast_to(np.asarray(t_end, np.float64), (len(self.sims),))
        steps_batch_run(self._h, t)

    @property
    def info(self):
        return steps_batch_info(self._h)

    @property
    def specialized(self):
        v = ctypes.c_int32(0)
        _check(lib.steps_batch_specialized(self._h, ctypes.byref(v)))
        return bool(v.value)

    def close(self):
        if getattr(self, "_h", None):
            steps_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class NativeServer:
    """The library's job server (steps_server_*): jobs are clones of prototype
    Simulation objects, advanced together in batched rounds."""

    def __init__(self, device_budget=0, max_jobs=64, wave_windows=16, block=256, specialize=-1, cuda_stream=None):
        opt = steps_server_options()
        lib.steps_server_options_default(ctypes.byref(opt))
        opt.device_budget = int(device_budget)
        opt.max_jobs = int(max_jobs)
        opt.wave_windows = int(wave_windows)
        opt.block = int(block)
        opt.specialize = int(specialize)
        h = ctypes.c_void_p()
        _check(lib.steps_server_create(ctypes.byref(opt), ctypes.c_void_p(cuda_stream) if cuda_stream else None,
                                       ctypes.byref(h)))
        self._h = h
        self._shape = {}

    def submit(self, proto, seed, counts, t_end):
        """Queue a job on prototype `proto` (a Simulation) from counts [S, nt]
        at time 0 to t_end; returns the job id."""
        c = np.ascontiguousarray(counts, np.int32)
        if c.shape != (proto.S, proto.nt):
            raise ValueError(f"counts must have shape {(proto.S, proto.nt)}")
        job = ctypes.c_int64()
        _check(lib.steps_server_submit(self._h, proto._sim, int(seed), _ptr(c), float(t_end), ctypes.byref(job)))
        self._shape[job.value] = c.shape
        return job.value

    def step(self):
        """One round; returns (jobs running, jobs finished in the round)."""
        r, f = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.steps_server_step(self._h, ctypes.byref(r), ctypes.byref(f)))
        return r.value, f.value

    def state(self, job):
        """(state, windows, time): state 0 queued, 1 running, 2 finished, 3 result taken."""
        st, w, t = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_double()
        _check(lib.steps_server_job_state(self._h, int(job), ctypes.byref(st), ctypes.byref(w), ctypes.byref(t)))
        return st.value, w.value, t.value

    def take_result(self, job):
        out = np.empty(self._shape.pop(job), np.int32)
        _check(lib.steps_server_take_result(self._h, int(job), _ptr(out)))
        return out

    def stats(self):
        r, b, l = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        q, n, by = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib.steps_server_stats(self._h, ctypes.byref(r), ctypes.byref(b), ctypes.byref(l), ctypes.byref(q),
                                      ctypes.byref(n), ctypes.byref(by)))
        return {"rounds": r.value, "rebuilds": b.value, "launches": l.value, "queued": q.value,
                "running": n.value, "device_bytes": by.value}

    def close(self):
        if getattr(self, "_h", None):
            lib.steps_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Simulation:
    """Owns one mesh, model and simulation handle (convenience wrapper over
    the calls above; counts are [S, nt] numpy arrays in the caller's tet order)."""

    def __init__(self, verts, tets, model, seed, occupancy=STEPS_OCC_MEAN, reorder=STEPS_REORDER_MORTON,
                 block=256, use_graph=True, cuda_stream=None, specialize=0, leave_law=0, flow=None):
        self.S = model.n_species
        self.R = model.n_reac
        self.nt = int(np.asarray(tets).shape[0])
        self._mesh = steps_mesh_create(verts, tets)
        self._model = steps_model_create(model.diff, model.lhs, model.rhs, model.k)
        opt = steps_options_default()
        opt.occupancy = occupancy
        opt.reorder = reorder
        opt.block = block
        opt.use_graph = 1 if use_graph else 0
        opt.specialize = int(specialize)
        opt.leave_law = int(leave_law)
        opt.flow = 0 if flow is None else (1 if flow else -1)  # None: tuned
        self._sim = steps_sim_create(self._mesh, self._model, seed, opt, cuda_stream)

    def clone(self, seed, cuda_stream=None):
        """A new Simulation sharing this one's mesh, model and device tables
        (copied on the device), with its own seed, zero counts, time 0."""
        c = Simulation.__new__(Simulation)
        c.S, c.R, c.nt = self.S, self.R, self.nt
        c._mesh = None
        c._model = None
        c._sim = steps_sim_clone(self._sim, seed, cuda_stream)
        return c

    @property
    def device_bytes(self):
        return steps_sim_device_bytes(self._sim)

    def close(self):
        if getattr(self, "_sim", None):
            steps_sim_destroy(self._sim)
            self._sim = None
        if getattr(self, "_model", None):
            steps_model_destroy(self._model)
            self._model = None
        if getattr(self, "_mesh", None):
            steps_mesh_destroy(self._mesh)
            self._mesh = None

    def __del__(self):
        self.close()

    def set_counts(self, counts):
        steps_set_counts_all(self._sim, counts)

    def get_counts(self, out=None):
        return steps_get_counts_all(self._sim, self.S, self.nt, out)

    def set_reac_rate(self, r, k):
        steps_set_reac_rate(self._sim, r, k)

    def run_record(self, t_end, dt_rec, species, tets, d_out_ptr, max_records):
        return steps_run_record(self._sim, t_end, dt_rec, species, tets, d_out_ptr, max_records)

    def set_reac_mask(self, r, mask):
        steps_set_reac_mask(self._sim, r, mask)

    def run(self, t_end):
        steps_run(self._sim, t_end)

    @property
    def time(self):
        return steps_get_time(self._sim)

    @property
    def tau(self):
        return steps_get_tau(self._sim)

    @property
    def specialized(self):
        return steps_sim_specialized(self._sim)

    @property
    def flow(self):
        """(tile size of the flow launches or 0, tuning ms per window [window launches, flow, flow at 512])."""
        return steps_sim_flow(self._sim)

    @property
    def windows(self):
        return steps_get_windows(self._sim)[0]

    @property
    def launches(self):
        return steps_get_windows(self._sim)[1]


def from_workload(w, occupancy=STEPS_OCC_MEAN, seed=None, **kw) -> Simulation:
    sim = Simulation(w.verts, w.tets, w.model, w.seed if seed is None else seed, occupancy=occupancy, **kw)
    sim.set_counts(w.counts)
    for r, m in w.reac_masks.items():
        sim.set_reac_mask(r, m)
    return sim
