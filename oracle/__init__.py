"""CPU oracle of the Parallel STEPS operator-split step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package. The product path (the CUDA library
and its Python binding) never imports it.

``OracleSim`` wraps ``steps_oracle.c`` (plain serial C, FP64), built by
``oracle.build.build()`` with gcc and no floating-point contraction.
``prec=64`` takes every reaction decision in double precision with 53-bit
uniforms (the method's definition); ``prec=32`` takes them with the float
operations and 24-bit uniforms the CUDA kernel uses, so that the two can be
compared element by element.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH, build

OCC, END = 1, 0
EULER, EXP = 0, 1  # leave laws: p = tau d (default) or p = 1 - exp(-tau d)
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            build()
        L = ctypes.CDLL(LIB_PATH)
        c_i64, c_u64, c_u32, c_i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
        P = ctypes.c_void_p
        L.orc_create.restype = P
        L.orc_create.argtypes = [c_i64, P, c_i64, P, ctypes.c_int, P, ctypes.c_int, P, P, P, c_u64,
                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_destroy.argtypes = [P]
        L.orc_set_counts.argtypes = [P, ctypes.c_int, P]
        L.orc_get_counts.argtypes = [P, ctypes.c_int, P]
        L.orc_set_reac_mask.argtypes = [P, ctypes.c_int, P]
        L.orc_set_reac_rate.argtypes = [P, ctypes.c_int, ctypes.c_double]
        L.orc_set_reac_rate.restype = ctypes.c_int
        L.orc_run.argtypes = [P, ctypes.c_double]
        L.orc_run.restype = ctypes.c_int
        L.orc_step.argtypes = [P, ctypes.c_double]
        L.orc_step.restype = ctypes.c_int
        L.orc_run_threads.argtypes = [P, ctypes.c_double, ctypes.c_int]
        L.orc_run_threads.restype = ctypes.c_int
        L.orc_step_threads.argtypes = [P, ctypes.c_double, ctypes.c_int]
        L.orc_step_threads.restype = ctypes.c_int
        L.orc_get_tau.argtypes = [P]
        L.orc_get_tau.restype = ctypes.c_double
        L.orc_get_time.argtypes = [P]
        L.orc_get_time.restype = ctypes.c_double
        L.orc_get_events.argtypes = [P]
        L.orc_get_events.restype = c_i64
        L.orc_get_windows.argtypes = [P]
        L.orc_get_windows.restype = c_u64
        L.orc_get_thresholds.argtypes = [P, P]
        L.orc_get_cumg.argtypes = [P, P]
        L.orc_get_species_thresholds.argtypes = [P, ctypes.c_int, ctypes.c_double, P]
        L.orc_get_species_thresholds.restype = c_u32
        L.orc_set_leave_law.argtypes = [P, ctypes.c_int]
        L.orc_set_leave_law.restype = ctypes.c_int
        L.orc_geometry.argtypes = [c_i64, P, c_i64, P, P, P, P, P, P]
        L.orc_geometry.restype = ctypes.c_int
        L.orc_adjacency.argtypes = [c_i64, c_i64, P, P]
        L.orc_adjacency.restype = ctypes.c_int
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_logf32.argtypes = [ctypes.c_float]
        L.orc_logf32.restype = ctypes.c_float
        L.orc_sample_faces.argtypes = [c_u64, c_u64, c_u32, c_u32, c_i32, P, P]
        L.orc_sample_faces.restype = c_u32
        L.orc_sample_bulk.argtypes = [c_u64, c_u64, c_u32, ctypes.c_int, c_i32, P, P]
        L.orc_logf32_array.argtypes = [P, c_i64, P]
        L.orc_philox_array.argtypes = [c_u64, P, c_i64, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def geometry(verts, tets):
    """(nbr [nt,4], vol [nt], area [nt,4], dist [nt,4], g [nt,4]) of a mesh."""
    verts = np.ascontiguousarray(verts, np.float64)
    tets = np.ascontiguousarray(tets, np.int32)
    nt = tets.shape[0]
    nbr = np.empty((nt, 4), np.int32)
    vol = np.empty(nt)
    area = np.empty((nt, 4))
    dist = np.empty((nt, 4))
    g = np.empty((nt, 4))
    rc = lib().orc_geometry(verts.shape[0], _p(verts), nt, _p(tets), _p(nbr), _p(vol), _p(area), _p(dist), _p(g))
    if rc != 0:
        raise ValueError(f"oracle geometry failed ({rc})")
    return nbr, vol, area, dist, g


def philox(key, ctr):
    """Philox4x32-10 of one (key[2], counter[4]) -> 4 uint32 words."""
    k = np.ascontiguousarray(key, np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    out = np.empty(4, np.uint32)
    lib().orc_philox4x32_10(_p(k), _p(c), _p(out))
    return out


def logf32(x: float) -> float:
    return float(lib().orc_logf32(ctypes.c_float(x)))


def logf32_array(x):
    a = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(a)
    lib().orc_logf32_array(_p(a), a.size, _p(out))
    return out


def philox_array(seed, ctr):
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    lib().orc_philox_array(ctypes.c_uint64(seed), _p(c), c.shape[0], _p(out))
    return out


def sample_faces(seed, window, tet, w0, M, T):
    """Faces chosen by M trial molecules against thresholds T[4];
    returns (counts per face [4], words consumed)."""
    Ta = np.ascontiguousarray(T, np.uint32)
    out = np.zeros(4, np.int32)
    used = lib().orc_sample_faces(seed, window, tet, w0, M, _p(Ta), _p(out))
    return out, int(used)


BULK_MIN = 16  # trial molecules of a species in a tet from which the oracle draws by bit planes


def sample_bulk(seed, window, tet, species, M, T):
    """Faces chosen by M trial molecules of one species drawing by bit planes
    (the path of M >= BULK_MIN); returns counts per face [4]."""
    Ta = np.ascontiguousarray(T, np.uint32)
    out = np.zeros(4, np.int32)
    lib().orc_sample_bulk(seed, window, tet, int(species), int(M), _p(Ta), _p(out))
    return out


class OracleSim:
    """Serial reference simulation. Counts are [S, nt] in the caller's tet order."""

    def __init__(self, verts, tets, model, seed: int, occ: int = OCC, prec: int = 64, leave: int = EULER):
        self._verts = np.ascontiguousarray(verts, np.float64)
        self._tets = np.ascontiguousarray(tets, np.int32)
        self.S = model.n_species
        self.R = model.n_reac
        self.nt = self._tets.shape[0]
        D = np.ascontiguousarray(model.diff, np.float64)
        lhs = np.ascontiguousarray(model.lhs, np.int32).reshape(-1)
        rhs = np.ascontiguousarray(model.rhs, np.int32).reshape(-1)
        k = np.ascontiguousarray(model.k, np.float64)
        if lhs.size == 0:
            lhs = np.zeros(1, np.int32)
            rhs = np.zeros(1, np.int32)
            k = np.zeros(1)
        err = ctypes.c_int(0)
        self._h = lib().orc_create(self._verts.shape[0], _p(self._verts), self.nt, _p(self._tets),
                                   self.S, _p(D), self.R, _p(lhs), _p(rhs), _p(k),
                                   ctypes.c_uint64(seed), occ, prec, ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle create failed ({err.value})")
        if leave != EULER and lib().orc_set_leave_law(self._h, int(leave)) != 0:
            raise ValueError("oracle: bad leave law or out of memory")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_counts(self, counts):
        counts = np.asarray(counts, np.int32)
        for s in range(self.S):
            row = np.ascontiguousarray(counts[s])
            lib().orc_set_counts(self._h, s, _p(row))

    def set_reac_mask(self, r, mask):
        if mask is None:
            lib().orc_set_reac_mask(self._h, r, None)
        else:
            m = np.ascontiguousarray(mask, np.uint8)
            lib().orc_set_reac_mask(self._h, r, _p(m))

    def set_reac_rate(self, r, k):
        if lib().orc_set_reac_rate(self._h, int(r), float(k)) != 0:
            raise ValueError("oracle: bad reaction or rate")

    def get_counts(self):
        out = np.empty((self.S, self.nt), np.int32)
        for s in range(self.S):
            row = np.empty(self.nt, np.int32)
            lib().orc_get_counts(self._h, s, _p(row))
            out[s] = row
        return out

    def run(self, t_end: float, threads: int = 1):
        """Advance to t_end. threads > 1 runs each window on that many host
        threads (gather form); the result is the serial one, bit for bit."""
        if threads > 1:
            if lib().orc_run_threads(self._h, float(t_end), int(threads)) != 0:
                raise ValueError("oracle: bad thread count or out of memory")
        else:
            lib().orc_run(self._h, float(t_end))

    def step(self, tau_k: float, threads: int = 1):
        if threads > 1:
            if lib().orc_step_threads(self._h, float(tau_k), int(threads)) != 0:
                raise ValueError("oracle: bad thread count or out of memory")
        else:
            lib().orc_step(self._h, float(tau_k))

    @property
    def tau(self):
        return lib().orc_get_tau(self._h)

    @property
    def time(self):
        return lib().orc_get_time(self._h)

    @property
    def events(self):
        return lib().orc_get_events(self._h)

    @property
    def windows(self):
        return lib().orc_get_windows(self._h)

    def thresholds(self):
        out = np.empty((self.nt, 4), np.uint32)
        lib().orc_get_thresholds(self._h, _p(out))
        return out

    def cumg(self):
        out = np.empty((self.nt, 4))
        lib().orc_get_cumg(self._h, _p(out))
        return out

    def species_thresholds(self, species: int, tau_k: float):
        """(T [nt, 4] cumulative face thresholds, R_S species scale) that a
        window of length tau_k uses for one species."""
        out = np.empty((self.nt, 4), np.uint32)
        scale = lib().orc_get_species_thresholds(self._h, int(species), float(tau_k), _p(out))
        return out, int(scale)


def from_workload(w, occ: int = OCC, prec: int = 64, seed=None, leave: int = EULER) -> OracleSim:
    sim = OracleSim(w.verts, w.tets, w.model, w.seed if seed is None else seed, occ=occ, prec=prec, leave=leave)
    sim.set_counts(w.counts)
    for r, m in w.reac_masks.items():
        sim.set_reac_mask(r, m)
    return sim
