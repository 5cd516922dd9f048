"""Thin Python binding of libgcharm (include/gcharm.h).

Argument marshalling only: every step of the batched path runs in the CUDA
library.  Host arrays are numpy; device arrays are torch CUDA tensors, used
purely as device memory (their ``data_ptr()`` is handed to the library).
The library must have been built (``paper_2008_05712_gb300.build.build()``);
there is no fallback: importing the binding without the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgcharm.so")

GC_OK = 0
GC_ERR_ARG = -1
GC_ERR_OOM = -2
GC_ERR_POOL_FULL = -3
GC_ERR_UNKNOWN_ID = -4
GC_ERR_BUDGET = -5
GC_ERR_NOT_READY = -6
GC_ERR_TIMEOUT = -7
GC_ERR_CUDA = -8
GC_ERR_STATE = -9
GC_ERR_TOO_LARGE = -10
NOALLOC_MAX_TASKS = 65536
NOALLOC_MAX_TARGETS = 262144

GC_GRAVITY = 0
GC_LJ_PAIR = 1
GC_LJ_SELF = 2
GC_EWALD = 3

GC_COMBINE_ADAPTIVE = 0
GC_COMBINE_ADAPTIVE_WINDOW = 1
GC_COMBINE_STATIC = 2
GC_COMBINE_PER_TASK = 3
GC_COMBINE_GREEDY = 4
GC_SCHED_FIFO = 0
GC_SCHED_LPT = 1
GC_ORDER_FULL = 0
GC_ORDER_SEEDED = 1

NONE32 = 0xFFFFFFFF


class GcConfig(C.Structure):
    _fields_ = [("eps2", C.c_float), ("lj_eps", C.c_float), ("lj_sigma", C.c_float),
                ("lj_rc2", C.c_float), ("md_edge", C.c_float),
                ("id_capacity", C.c_uint64), ("pool_capacity", C.c_uint64),
                ("staging_budget_bytes", C.c_uint64), ("deterministic", C.c_int),
                ("cuda_stream", C.c_void_p), ("ewald_box", C.c_float)]


class GcTask(C.Structure):
    _fields_ = [("task_id", C.c_uint64), ("kind", C.c_uint32), ("n_targets", C.c_uint32),
                ("n_sources", C.c_uint32), ("target_ids", C.POINTER(C.c_uint32)),
                ("source_ids", C.POINTER(C.c_uint32)), ("shift", C.c_int8 * 3)]


_STAT_FIELDS = ["flushes", "tasks", "entries", "unique", "hits", "misses", "updates",
                "evictions", "h2d_bytes", "interactions", "lj_pairs_in_cutoff", "last_unique",
                "last_hits", "last_misses", "last_evictions", "last_staging_bytes",
                "last_waves"]


class GcStats(C.Structure):
    _fields_ = ([(f, C.c_uint64) for f in _STAT_FIELDS] + [("reuse_hist", C.c_uint64 * 8)]
                + [("kernel_launches", C.c_uint64), ("primitive_calls", C.c_uint64),
                   ("stage_ms_sum", C.c_double * 5), ("timed_batches", C.c_uint64)])


class GcServeConfig(C.Structure):
    _fields_ = [("policy", C.c_int), ("max_size", C.c_uint64), ("static_n", C.c_uint64),
                ("window", C.c_uint64), ("max_in_flight", C.c_uint32),
                ("keep_pageable", C.c_uint32), ("poll_ns", C.c_uint64), ("timeout_ns", C.c_uint64),
                ("task_set", C.c_uint64), ("warmup_ns", C.c_uint64), ("drain_ns", C.c_uint64)]


_SERVE_FIELDS = ["tasks", "batches", "interactions", "max_size"]
_SERVE_DFIELDS = ["wall_s", "interactions_per_s", "lat_mean_us", "lat_p50_us", "lat_p99_us",
                  "lat_max_us", "mean_batch", "busy_s"]
_SERVE_TAIL = ["measured", "unserved", "pinned_bytes"]
_SERVE_HOST = ["submit_s", "flush_s", "retire_s"]


class GcServeReport(C.Structure):
    _fields_ = ([(f, C.c_uint64) for f in _SERVE_FIELDS]
                + [(f, C.c_double) for f in _SERVE_DFIELDS]
                + [(f, C.c_uint64) for f in _SERVE_TAIL]
                + [(f, C.c_double) for f in _SERVE_HOST])


_NBODY_FIELDS = ["builds", "seeded_builds", "last_resorted", "timed_builds"]
_NBODY_DFIELDS = ["last_order_ms", "last_tree_ms", "order_ms_sum", "tree_ms_sum"]


class GcNbodyStats(C.Structure):
    _fields_ = ([(f, C.c_uint64) for f in _NBODY_FIELDS]
                + [(f, C.c_double) for f in _NBODY_DFIELDS])


class GcTuning(C.Structure):
    _fields_ = [("wu_max_targets", C.c_uint32), ("schedule", C.c_uint32),
                ("tile_pairs", C.c_uint32), ("comp_block", C.c_uint32),
                ("targets_per_lane", C.c_uint32)]


GC_TUNE_COUNT = 108
_TUNE_FIELDS = ["wu_max_targets", "schedule", "tile_pairs", "comp_block", "targets_per_lane"]


def tune_key(t):
    """Name of a tuning in the autotuner's times:
    'wu,fifo|lpt,tile,block,targets per lane'."""
    return (f"{t['wu_max_targets']},{'lpt' if t['schedule'] else 'fifo'},"
            f"{t['tile_pairs']},{t['comp_block']},{t['targets_per_lane']}")


def tune_order():
    """The autotuner's tunings in the order of its times (gc_autotune)."""
    return [dict(wu_max_targets=w, schedule=s, tile_pairs=tp, comp_block=kb, targets_per_lane=l)
            for w in (8, 16, 32) for s in (0, 1) for tp in (64, 128, 256) for kb in (8, 16, 32)
            for l in (1, 2)]


class GcError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = _lib.gc_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


_lib = None

P = C.c_void_p
U64 = C.c_uint64
U64P = C.POINTER(C.c_uint64)

# name -> argtypes (all return int unless noted)
_SIGS = {
    "gc_pool_create": [C.POINTER(GcConfig), C.POINTER(P)],
    "gc_pool_destroy": [P],
    "gc_pool_upload": [P, P, P, U64],
    "gc_pool_upload_device": [P, P, P, U64],
    "gc_submit": [P, P, U64, U64P],
    "gc_submit_csr": [P, U64, P, P, P, P, P, P, P, U64, U64, C.c_int, U64P],
    "gc_flush": [P],
    "gc_flush_per_task": [P],
    "gc_wait": [P, U64, U64],
    "gc_batch_done": [P, U64, C.POINTER(C.c_int)],
    "gc_join": [P, P],
    "gc_result_rows": [P, U64P],
    "gc_read_batch_results": [P, U64, U64, P],
    "gc_read_batch_rows": [P, U64, U64, U64, P],
    "gc_read_results": [P, P, U64, P],
    "gc_read_totals": [P, P, U64, P],
    "gc_read_totals_async": [P, P, U64, P],
    "gc_pool_upload_async": [P, P, P, U64],
    "gc_totals_device": [P, C.POINTER(P)],
    "gc_reset_totals": [P],
    "gc_stats": [P, C.POINTER(GcStats)],
    "gc_strerror": [C.c_int],
    "gc_read_entry_slots": [P, P, P],
    "gc_read_pack_perm": [P, P, P],
    "gc_batch_sizes": [P, U64P, U64P, U64P],
    "gc_read_residency": [P, P, P, P],
    "gc_read_evicted": [P, P, U64, U64P],
    "gc_build_nbody_tasks": [P, P, U64, C.c_int, C.c_int, C.c_int, U64, P],
    "gc_nbody_set_order": [P, C.c_int],
    "gc_nbody_stats": [P, C.POINTER(GcNbodyStats)],
    "gc_build_nbody_tasks_resident": [P, U64, C.c_int, C.c_int, C.c_int, U64, P],
    "gc_read_nbody_tree": [P] + [P] * 14,
    "gc_build_md_tasks": [P, P, U64, C.c_int, U64, P],
    "gc_build_md_tasks_2d": [P, P, U64, C.c_int, U64, P],
    "gc_read_md_cells": [P, P, P],
    "gc_last_timings": [P, P],
    "gc_gravity_noalloc": [U64, P, P, P, P, U64, C.c_float, P, P],
    "gc_read_batch_values": [P, U64, U64, P],
    "gc_row_values": [P, U64, P],
    "gc_combiner_create": [C.c_int, U64, U64, U64, C.POINTER(P)],
    "gc_combiner_destroy": [P],
    "gc_combiner_arrive": [P, U64, U64],
    "gc_combiner_poll": [P, U64, U64, U64P],
    "gc_combiner_max_interval": [P, U64P],
    "gc_combine_size_from_occupancy": [C.c_double, C.c_uint32, C.c_uint32],
    "gc_max_combine_size": [P, U64P],
    "gc_serve": [P, U64, P, P, P, P, P, P, P, C.POINTER(GcServeConfig), P, P,
                 C.POINTER(GcServeReport)],
    "gc_fp32_peak": [C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "gc_check_wait_expiry": [C.c_void_p, C.c_uint32],
    "gc_set_tuning": [P, C.POINTER(GcTuning)],
    "gc_get_tuning": [P, C.POINTER(GcTuning)],
    "gc_autotune": [P, C.c_int, C.POINTER(GcTuning), P],
    "gc_graph_capture": [P, C.POINTER(P)],
    "gc_graph_launch": [P],
    "gc_graph_wait": [P],
    "gc_graph_rows": [P, U64P],
    "gc_graph_results": [P, U64, U64, P],
    "gc_graph_destroy": [P],
    "gc_reuse_ablation": [P, C.c_int, P],
    "gc_nbody_kick_drift": [P, P, P, P, U64, C.c_double],
}

_RESTYPES = {"gc_strerror": C.c_char_p, "gc_combine_size_from_occupancy": C.c_uint64}


def exported_symbols():
    """Names the header declares (used by the ABI test)."""
    return sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Load libgcharm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_2008_05712_gb300.build.build()")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPES.get(name, C.c_int)
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != GC_OK:
        raise GcError(rc, what)


def _dptr(t):
    """Device pointer of a torch CUDA tensor (contiguous)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Pool:
    """One device pool (chare table + slots + batch + totals)."""

    def __init__(self, id_capacity, pool_capacity, eps2=1e-4, lj_eps=1.0, lj_sigma=1.0,
                 lj_rc2=0.0, md_edge=0.0, staging_budget_bytes=0, stream=None, ewald_box=0.0):
        lib = load()
        cfg = GcConfig()
        cfg.eps2 = eps2
        cfg.lj_eps, cfg.lj_sigma, cfg.lj_rc2, cfg.md_edge = lj_eps, lj_sigma, lj_rc2, md_edge
        cfg.id_capacity, cfg.pool_capacity = int(id_capacity), int(pool_capacity)
        cfg.staging_budget_bytes = int(staging_budget_bytes)
        cfg.deterministic = 1
        cfg.cuda_stream = stream
        cfg.ewald_box = ewald_box
        h = C.c_void_p()
        _check(lib.gc_pool_create(C.byref(cfg), C.byref(h)), "gc_pool_create")
        self.h = h
        self.cfg = cfg
        self.lib = lib

    def close(self):
        if self.h:
            _check(self.lib.gc_pool_destroy(self.h), "gc_pool_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- data -----------------------------------------------------------------
    def upload(self, ids, xyzm):
        ids = np.ascontiguousarray(ids, np.uint32)
        x = np.ascontiguousarray(xyzm, np.float32)
        assert x.shape == (ids.shape[0], 4)
        _check(self.lib.gc_pool_upload(self.h, _p(ids), _p(x), ids.shape[0]), "gc_pool_upload")

    def upload_async(self, ids, xyzm):
        """gc_pool_upload_async: the copies are queued on the pool's stream and
        read later, so the arrays (uint32 ids, float32 (n, 4) values, C-contiguous,
        best in pinned memory) must stay alive and unchanged until the pool's
        work is joined and waited for.  No temporary copies are made."""
        if (not isinstance(ids, np.ndarray) or ids.dtype != np.uint32 or
                not ids.flags["C_CONTIGUOUS"]):
            raise ValueError("ids must be a C-contiguous uint32 array")
        if (not isinstance(xyzm, np.ndarray) or xyzm.dtype != np.float32 or
                xyzm.shape != (ids.shape[0], 4) or not xyzm.flags["C_CONTIGUOUS"]):
            raise ValueError("xyzm must be a C-contiguous float32 array of shape (n, 4)")
        _check(self.lib.gc_pool_upload_async(self.h, _p(ids), _p(xyzm), ids.shape[0]),
               "gc_pool_upload_async")

    def upload_device(self, ids_t, xyzm_t):
        _check(self.lib.gc_pool_upload_device(self.h, _dptr(ids_t), _dptr(xyzm_t),
                                              ids_t.numel()), "gc_pool_upload_device")

    # ---- batching ---------------------------------------------------------------
    def submit_csr(self, kinds, tgt_off, tgt_ids, src_off, src_ids, shifts=None, task_ids=None):
        kinds = np.ascontiguousarray(kinds, np.uint32)
        to = np.ascontiguousarray(tgt_off, np.uint64)
        so = np.ascontiguousarray(src_off, np.uint64)
        tg = np.ascontiguousarray(tgt_ids, np.uint32)
        sr = np.ascontiguousarray(src_ids, np.uint32)
        sh = None if shifts is None else np.ascontiguousarray(shifts, np.int8)
        ti = None if task_ids is None else np.ascontiguousarray(task_ids, np.uint64)
        b = C.c_uint64()
        _check(self.lib.gc_submit_csr(self.h, kinds.shape[0], _p(ti), _p(kinds), _p(sh), _p(to),
                                      _p(tg), _p(so), _p(sr), 0, 0, 0, C.byref(b)),
               "gc_submit_csr")
        return b.value

    def submit_csr_device(self, kinds, tgt_off, tgt_ids, src_off, src_ids, n_tgt, n_src,
                          shifts=None, task_ids=None):
        b = C.c_uint64()
        _check(self.lib.gc_submit_csr(self.h, kinds.numel(), _dptr(task_ids), _dptr(kinds),
                                      _dptr(shifts), _dptr(tgt_off), _dptr(tgt_ids),
                                      _dptr(src_off), _dptr(src_ids), int(n_tgt), int(n_src),
                                      1, C.byref(b)), "gc_submit_csr(device)")
        return b.value

    def submit_tasks(self, tasks):
        """tasks: list of dicts {task_id, kind, targets, sources, shift}."""
        arr = (GcTask * len(tasks))()
        keep = []
        for t, d in zip(arr, tasks):
            tg = np.ascontiguousarray(d["targets"], np.uint32)
            sr = np.ascontiguousarray(d.get("sources", []), np.uint32)
            keep += [tg, sr]
            t.task_id = int(d.get("task_id", 0))
            t.kind = int(d["kind"])
            t.n_targets, t.n_sources = tg.shape[0], sr.shape[0]
            t.target_ids = tg.ctypes.data_as(C.POINTER(C.c_uint32))
            t.source_ids = sr.ctypes.data_as(C.POINTER(C.c_uint32))
            for a, v in enumerate(d.get("shift", (0, 0, 0))):
                t.shift[a] = int(v)
        b = C.c_uint64()
        _check(self.lib.gc_submit(self.h, C.cast(arr, C.c_void_p), len(tasks), C.byref(b)),
               "gc_submit")
        return b.value

    def flush(self):
        _check(self.lib.gc_flush(self.h), "gc_flush")

    def flush_per_task(self):
        _check(self.lib.gc_flush_per_task(self.h), "gc_flush_per_task")

    def done(self, batch):
        d = C.c_int()
        _check(self.lib.gc_batch_done(self.h, int(batch), C.byref(d)), "gc_batch_done")
        return bool(d.value)

    def join(self, stream_handle):
        """Make the CUDA stream (raw handle, e.g. torch's ``cuda_stream``) wait
        for all work the pool has issued (gc_join)."""
        _check(self.lib.gc_join(self.h, C.c_void_p(stream_handle)), "gc_join")

    def wait(self, batch, timeout_ns=0):
        _check(self.lib.gc_wait(self.h, int(batch), int(timeout_ns)), "gc_wait")

    # ---- results ----------------------------------------------------------------
    def result_rows(self):
        r = C.c_uint64()
        _check(self.lib.gc_result_rows(self.h, C.byref(r)), "gc_result_rows")
        return r.value

    def results(self, first=0, n=None):
        """(rows, 8) float32: sum (4) then compensation (4); value = s - c."""
        if n is None:
            n = self.result_rows() - first
        out = np.empty((n, 8), np.float32)
        _check(self.lib.gc_read_batch_results(self.h, first, n, _p(out)),
               "gc_read_batch_results")
        return out

    def values(self, first=0, n=None):
        """(rows, 4) float64 values s - c of the last batch's rows, computed
        on the device (gc_read_batch_values)."""
        if n is None:
            n = self.result_rows() - first
        out = np.empty((n, 4), np.float64)
        _check(self.lib.gc_read_batch_values(self.h, first, n, _p(out)),
               "gc_read_batch_values")
        return out

    def batch_rows(self, batch, first=0, n=None):
        """Result rows of one of the two most recent batches, like results()."""
        if n is None:
            raise ValueError("n is required")
        out = np.empty((n, 8), np.float32)
        _check(self.lib.gc_read_batch_rows(self.h, int(batch), first, n, _p(out)),
               "gc_read_batch_rows")
        return out

    def serve(self, arrival_ns, kinds, tgt_off, tgt_ids, src_off, src_ids, shifts=None,
              policy=GC_COMBINE_GREEDY, max_size=0, static_n=100, window=1024,
              max_in_flight=2, poll_ns=50_000, timeout_ns=0, want_results=False,
              task_set=0, warmup_ns=0, drain_ns=0, keep_pageable=False):
        """Replay an arrival schedule through the serving loop (gc_serve).

        Returns (report dict, latency_ns array, rows or None); rows are the
        result rows of every task in task order, (n_rows, 8) float32.  With
        task_set = m > 0 the CSR arrays hold m tasks, replayed cyclically."""
        arr = np.ascontiguousarray(arrival_ns, np.uint64)
        kinds = np.ascontiguousarray(kinds, np.uint32)
        to = np.ascontiguousarray(tgt_off, np.uint64)
        so = np.ascontiguousarray(src_off, np.uint64)
        tg = np.ascontiguousarray(tgt_ids, np.uint32)
        sr = np.ascontiguousarray(src_ids, np.uint32)
        sh = None if shifts is None else np.ascontiguousarray(shifts, np.int8)
        n = arr.shape[0]
        cfg = GcServeConfig(policy=policy, max_size=max_size, static_n=static_n, window=window,
                            max_in_flight=max_in_flight, poll_ns=poll_ns, timeout_ns=timeout_ns,
                            task_set=task_set, warmup_ns=warmup_ns, drain_ns=drain_ns,
                            keep_pageable=1 if keep_pageable else 0)
        lat = np.zeros(n, np.uint64)
        rows = None
        if want_results:
            n_rows = int(to[-1]) + int(np.sum((so[1:] - so[:-1])[kinds == GC_LJ_PAIR]))
            rows = np.zeros((n_rows, 8), np.float32)
        rep = GcServeReport()
        _check(self.lib.gc_serve(self.h, n, _p(arr), _p(kinds), _p(sh), _p(to), _p(tg), _p(so),
                                 _p(sr), C.byref(cfg), _p(lat), _p(rows), C.byref(rep)),
               "gc_serve")
        d = {f: getattr(rep, f) for f in _SERVE_FIELDS + _SERVE_DFIELDS + _SERVE_TAIL
             + _SERVE_HOST}
        return d, lat, rows

    def read_results(self, task_ids, n_rows):
        ti = np.ascontiguousarray(task_ids, np.uint64)
        out = np.empty((n_rows, 8), np.float32)
        _check(self.lib.gc_read_results(self.h, _p(ti), ti.shape[0], _p(out)), "gc_read_results")
        return out

    def totals(self, ids, out=None):
        """(n, 4) float64 per-id totals; `out` (optional) is a C-contiguous
        float64 array of that shape to fill, e.g. in pinned memory."""
        ids = np.ascontiguousarray(ids, np.uint32)
        if out is None:
            out = np.empty((ids.shape[0], 4), np.float64)
        elif (out.dtype != np.float64 or out.shape != (ids.shape[0], 4) or
              not out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a C-contiguous float64 array of shape (n, 4)")
        _check(self.lib.gc_read_totals(self.h, _p(ids), ids.shape[0], _p(out)), "gc_read_totals")
        return out

    def totals_async(self, ids, out):
        """gc_read_totals_async: `out` (C-contiguous float64 (n, 4), best in
        pinned memory) is filled once the pool's work is joined and waited
        for; ids (C-contiguous uint32) and out must stay alive until then."""
        if (not isinstance(ids, np.ndarray) or ids.dtype != np.uint32 or
                not ids.flags["C_CONTIGUOUS"]):
            raise ValueError("ids must be a C-contiguous uint32 array")
        if (out.dtype != np.float64 or out.shape != (ids.shape[0], 4) or
                not out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a C-contiguous float64 array of shape (n, 4)")
        _check(self.lib.gc_read_totals_async(self.h, _p(ids), ids.shape[0], _p(out)),
               "gc_read_totals_async")
        return out

    def totals_device_ptr(self):
        p = C.c_void_p()
        _check(self.lib.gc_totals_device(self.h, C.byref(p)), "gc_totals_device")
        return p.value

    def reset_totals(self):
        _check(self.lib.gc_reset_totals(self.h), "gc_reset_totals")

    def stats(self):
        s = GcStats()
        _check(self.lib.gc_stats(self.h, C.byref(s)), "gc_stats")
        d = {f: getattr(s, f) for f in _STAT_FIELDS}
        d["reuse_hist"] = list(s.reuse_hist)
        d["kernel_launches"] = s.kernel_launches
        d["primitive_calls"] = s.primitive_calls
        d["stage_ms_sum"] = dict(zip(["residency", "pack", "interact", "scatter", "total"],
                                     list(s.stage_ms_sum)))
        d["timed_batches"] = s.timed_batches
        return d

    def set_tuning(self, wu_max_targets=16, schedule=GC_SCHED_FIFO, tile_pairs=128,
                   comp_block=8, targets_per_lane=1):
        t = GcTuning(wu_max_targets=wu_max_targets, schedule=schedule, tile_pairs=tile_pairs,
                     comp_block=comp_block, targets_per_lane=targets_per_lane)
        _check(self.lib.gc_set_tuning(self.h, C.byref(t)), "gc_set_tuning")

    def tuning(self):
        t = GcTuning()
        _check(self.lib.gc_get_tuning(self.h, C.byref(t)), "gc_get_tuning")
        return {f: getattr(t, f) for f in _TUNE_FIELDS}

    def autotune(self, reps=3, cache=None, key=None):
        """Pick the interaction schedule on the last flushed batch (gc_autotune).

        With ``cache`` (a JSON file path) and ``key`` (a workload name), a
        choice stored under ``key`` is applied without tuning; otherwise the
        tuned choice is stored there.  Returns (choice, times_ms or None)."""
        import json
        if cache and key:
            try:
                with open(cache) as f:
                    stored = json.load(f).get(key)
            except (OSError, ValueError):
                stored = None
            if stored and all(f in stored for f in _TUNE_FIELDS):
                self.set_tuning(*[stored[f] for f in _TUNE_FIELDS])
                return dict(stored), None
        best = GcTuning()
        ms = np.zeros(GC_TUNE_COUNT, np.float32)
        _check(self.lib.gc_autotune(self.h, int(reps), C.byref(best), _p(ms)), "gc_autotune")
        choice = {f: getattr(best, f) for f in _TUNE_FIELDS}
        times = {tune_key(t): float(ms[i]) for i, t in enumerate(tune_order())}
        if cache and key:
            try:
                with open(cache) as f:
                    data = json.load(f)
            except (OSError, ValueError):
                data = {}
            data[key] = dict(choice, times_ms=times)
            with open(cache, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
        return choice, times

    def check_wait_expiry(self, polls=1024):
        """Run the bounded barrier wait's expiry path on the issue stream: the
        next wait() raises GcError(GC_ERR_TIMEOUT) and the pool stays usable."""
        _check(self.lib.gc_check_wait_expiry(self.h, int(polls)), "gc_check_wait_expiry")

    def reuse_ablation(self, reps=3):
        """Fig. 3 of Section 3.2 on the last batch (gc_reuse_ablation)."""
        out = np.zeros(7, np.float64)
        _check(self.lib.gc_reuse_ablation(self.h, int(reps), _p(out)), "gc_reuse_ablation")
        keys = ["kernel_pack_ms", "kernel_indirect_ms", "kernel_sorted_indirect_ms",
                "redundant_host_gather_ms", "redundant_h2d_ms", "redundant_bytes",
                "reuse_fetch_bytes"]
        return dict(zip(keys, out.tolist()))

    def max_combine_size(self):
        v = C.c_uint64()
        _check(self.lib.gc_max_combine_size(self.h, C.byref(v)), "gc_max_combine_size")
        return v.value

    def timings(self):
        ms = np.zeros(5, np.float32)
        _check(self.lib.gc_last_timings(self.h, _p(ms)), "gc_last_timings")
        return dict(zip(["residency", "pack", "interact", "scatter", "total"], ms.tolist()))

    # ---- introspection ----------------------------------------------------------
    def batch_sizes(self):
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(self.lib.gc_batch_sizes(self.h, C.byref(a), C.byref(b), C.byref(c)),
               "gc_batch_sizes")
        return a.value, b.value, c.value

    def entry_slots(self):
        _, nt, ns = self.batch_sizes()
        t = np.empty(nt, np.uint32)
        s = np.empty(ns, np.uint32)
        _check(self.lib.gc_read_entry_slots(self.h, _p(t), _p(s)), "gc_read_entry_slots")
        return t, s

    def pack_perm(self):
        _, nt, ns = self.batch_sizes()
        t = np.empty(nt, np.uint32)
        s = np.empty(ns, np.uint32)
        _check(self.lib.gc_read_pack_perm(self.h, _p(t), _p(s)), "gc_read_pack_perm")
        return t, s

    def residency(self):
        a = np.empty(self.cfg.id_capacity, np.uint32)
        b = np.empty(self.cfg.pool_capacity, np.uint32)
        c = np.empty(self.cfg.pool_capacity, np.uint32)
        _check(self.lib.gc_read_residency(self.h, _p(a), _p(b), _p(c)), "gc_read_residency")
        return a, b, c

    def evicted(self):
        n = C.c_uint64()
        buf = np.empty(self.cfg.pool_capacity, np.uint32)
        _check(self.lib.gc_read_evicted(self.h, _p(buf), buf.shape[0], C.byref(n)),
               "gc_read_evicted")
        return buf[:n.value].copy()

    # ---- task builders ----------------------------------------------------------
    def build_nbody(self, xyzm, bucket_max=32, theta_num=7, theta_den=10, task_id_base=0):
        """xyzm: CUDA tensor (n, 4) or a host numpy float32 (n, 4) array."""
        info = np.zeros(4, np.uint64)
        if isinstance(xyzm, np.ndarray):
            xyzm = np.ascontiguousarray(xyzm, np.float32)
            ptr = _p(xyzm)
        else:
            ptr = _dptr(xyzm)
        _check(self.lib.gc_build_nbody_tasks(self.h, ptr, xyzm.shape[0], bucket_max,
                                             theta_num, theta_den, task_id_base, _p(info)),
               "gc_build_nbody_tasks")
        return dict(n_nodes=int(info[0]), n_buckets=int(info[1]), list_entries=int(info[2]),
                    resorted=int(info[3]))

    def set_order(self, mode):
        """GC_ORDER_SEEDED (default): a build of the same n starts from the
        previous build's Morton order; GC_ORDER_FULL: every build sorts all
        keys.  Both give identical trees (gc_nbody_set_order)."""
        _check(self.lib.gc_nbody_set_order(self.h, int(mode)), "gc_nbody_set_order")

    def nbody_stats(self):
        s = GcNbodyStats()
        _check(self.lib.gc_nbody_stats(self.h, C.byref(s)), "gc_nbody_stats")
        return {f: getattr(s, f) for f in _NBODY_FIELDS + _NBODY_DFIELDS}

    def build_nbody_resident(self, n, bucket_max=32, theta_num=7, theta_den=10,
                             task_id_base=0):
        """As build_nbody, with the positions of particles 0..n-1 read from
        the pool's current values (no second host-to-device copy)."""
        info = np.zeros(4, np.uint64)
        _check(self.lib.gc_build_nbody_tasks_resident(self.h, int(n), bucket_max, theta_num,
                                                      theta_den, task_id_base, _p(info)),
               "gc_build_nbody_tasks_resident")
        return dict(n_nodes=int(info[0]), n_buckets=int(info[1]), list_entries=int(info[2]),
                    resorted=int(info[3]))

    def nbody_tree(self, n, n_nodes, n_buckets, n_list):
        out = dict(sorted_ids=np.empty(n, np.uint32), sorted_keys=np.empty(n, np.uint64),
                   level=np.empty(n_nodes, np.uint8), cell=np.empty((n_nodes, 3), np.uint32),
                   first=np.empty(n_nodes, np.uint32), count=np.empty(n_nodes, np.uint32),
                   leaf=np.empty(n_nodes, np.uint8), size=np.empty(n_nodes, np.uint32),
                   node_xyzm=np.empty((n_nodes, 4), np.float32),
                   bucket_first=np.empty(n_buckets, np.uint32),
                   bucket_count=np.empty(n_buckets, np.uint32),
                   bucket_node=np.empty(n_buckets, np.uint32),
                   list_off=np.empty(n_buckets + 1, np.uint64),
                   list_ids=np.empty(n_list, np.uint32))
        keys = ["sorted_ids", "sorted_keys", "level", "cell", "first", "count", "leaf", "size",
                "node_xyzm", "bucket_first", "bucket_count", "bucket_node", "list_off",
                "list_ids"]
        _check(self.lib.gc_read_nbody_tree(self.h, *[_p(out[k]) for k in keys]),
               "gc_read_nbody_tree")
        return out

    def kick_drift(self, acc_ptr, xyzm_t, vel_t, dt):
        """Leapfrog step on device arrays (gc_nbody_kick_drift); acc_ptr is a
        device address of 4 doubles per particle (e.g. totals_device_ptr())
        or a CUDA float64 tensor."""
        a = acc_ptr if isinstance(acc_ptr, int) else acc_ptr.data_ptr()
        _check(self.lib.gc_nbody_kick_drift(self.h, C.c_void_p(a), _dptr(xyzm_t), _dptr(vel_t),
                                            xyzm_t.shape[0], float(dt)),
               "gc_nbody_kick_drift")

    def nbody_bucket_counts(self, n_buckets):
        """Targets per bucket of the last N-body build, in bucket order."""
        out = np.empty(n_buckets, np.uint32)
        args = [None] * 14
        args[10] = _p(out)                     # bucket_count
        _check(self.lib.gc_read_nbody_tree(self.h, *args), "gc_read_nbody_tree")
        return out

    def nbody_node_values(self, n_nodes):
        """(x, y, z, m) float32 of every node of the last N-body build (node
        k has data id n + k)."""
        out = np.empty((n_nodes, 4), np.float32)
        args = [None] * 14
        args[8] = _p(out)                      # node_xyzm
        _check(self.lib.gc_read_nbody_tree(self.h, *args), "gc_read_nbody_tree")
        return out

    def nbody_sorted_ids(self, n):
        """Particle ids of the last N-body build in Morton (key, id) order."""
        out = np.empty(n, np.uint32)
        _check(self.lib.gc_read_nbody_tree(self.h, _p(out), *([None] * 13)),
               "gc_read_nbody_tree")
        return out

    def build_md(self, cell, m, task_id_base=0, dim=3):
        """cell: CUDA tensor or host numpy array of uint32/int32 cell indices;
        dim 3 (m^3 cells) or 2 (the planar m x m grid)."""
        info = np.zeros(4, np.uint64)
        if isinstance(cell, np.ndarray):
            cell = np.ascontiguousarray(cell, np.uint32)
            ptr, n = _p(cell), cell.shape[0]
        else:
            ptr, n = _dptr(cell), cell.numel()
        fn = self.lib.gc_build_md_tasks if dim == 3 else self.lib.gc_build_md_tasks_2d
        _check(fn(self.h, ptr, n, m, task_id_base, _p(info)), "gc_build_md_tasks")
        return dict(tasks=int(info[0]), tgt_entries=int(info[1]), src_entries=int(info[2]))

    def md_cells(self, n, m, dim=3):
        start = np.empty(m ** dim + 1, np.uint32)
        atoms = np.empty(n, np.uint32)
        _check(self.lib.gc_read_md_cells(self.h, _p(start), _p(atoms)), "gc_read_md_cells")
        return start, atoms


class Graph:
    """A pending batch captured as a replayable CUDA graph (gc_graph_*)."""

    def __init__(self, pool):
        h = C.c_void_p()
        _check(pool.lib.gc_graph_capture(pool.h, C.byref(h)), "gc_graph_capture")
        self.h, self.lib, self.pool = h, pool.lib, pool

    def launch(self):
        _check(self.lib.gc_graph_launch(self.h), "gc_graph_launch")

    def wait(self):
        _check(self.lib.gc_graph_wait(self.h), "gc_graph_wait")

    def results(self):
        r = C.c_uint64()
        _check(self.lib.gc_graph_rows(self.h, C.byref(r)), "gc_graph_rows")
        out = np.empty((r.value, 8), np.float32)
        _check(self.lib.gc_graph_results(self.h, 0, r.value, _p(out)), "gc_graph_results")
        return out

    def close(self):
        if self.h:
            _check(self.lib.gc_graph_destroy(self.h), "gc_graph_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def value(res):
    """FP64 values of compensated result rows (rows, 8) float32 -> (rows, 4)
    float64, computed by the library (gc_row_values)."""
    rows = np.ascontiguousarray(res, np.float32)
    if rows.ndim != 2 or rows.shape[1] != 8:
        raise ValueError("expected result rows of shape (n, 8)")
    out = np.empty((rows.shape[0], 4), np.float64)
    _check(load().gc_row_values(_p(rows), rows.shape[0], _p(out)), "gc_row_values")
    return out


def gravity_noalloc(tgt_off, tgt_xyzm, src_off, src_xyzm, n_tgt_total, eps2, out_rows,
                    stream=None):
    """Softened gravity of a CSR batch already in device memory, without any
    allocation, for callers that cannot allocate when they need the result
    (a framework whose allocator already holds the device memory budget,
    latency-critical threads that must not take cudaMalloc/cudaFree's
    device-wide synchronisation).  Offsets are int64 CUDA tensors of
    n_tasks + 1 entries, values float32 (n, 4) CUDA tensors, out a float32
    (n_tgt_total, 8) CUDA tensor, all on the current device; the call is
    queued on ``stream`` (a raw cudaStream_t handle; None = the legacy
    default stream).  Shapes and types are checked here, before the library
    is called, because the library cannot see the tensors' sizes."""
    import torch
    dev = torch.cuda.current_device()
    n_tgt_total = int(n_tgt_total)
    for name, t in (("tgt_off", tgt_off), ("src_off", src_off), ("tgt_xyzm", tgt_xyzm),
                    ("src_xyzm", src_xyzm), ("out_rows", out_rows)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name}: on cuda:{t.device.index}, not the current device cuda:{dev}")
    for name, t in (("tgt_off", tgt_off), ("src_off", src_off)):
        if t.dtype != torch.int64 or t.dim() != 1 or t.numel() < 1:
            raise ValueError(f"{name}: expected a 1-D int64 tensor of n_tasks + 1 offsets")
    if src_off.numel() != tgt_off.numel():
        raise ValueError("tgt_off and src_off must hold the same number of offsets")
    for name, t in (("tgt_xyzm", tgt_xyzm), ("src_xyzm", src_xyzm)):
        if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 4:
            raise ValueError(f"{name}: expected a float32 tensor of shape (n, 4)")
    if tgt_xyzm.shape[0] < n_tgt_total:
        raise ValueError("tgt_xyzm holds fewer than n_tgt_total rows")
    if out_rows.dtype != torch.float32 or tuple(out_rows.shape) != (n_tgt_total, 8):
        raise ValueError("out_rows: expected a float32 tensor of shape (n_tgt_total, 8)")
    lib = load()
    _check(lib.gc_gravity_noalloc(tgt_off.numel() - 1, _dptr(tgt_off), _dptr(tgt_xyzm),
                                  _dptr(src_off), _dptr(src_xyzm), n_tgt_total,
                                  float(eps2), _dptr(out_rows), stream),
           "gc_gravity_noalloc")


class Combiner:
    """The combining policy of Section 3.1 (host-side; times in ns)."""

    def __init__(self, policy, max_size=0, static_n=0, window=0):
        lib = load()
        h = C.c_void_p()
        _check(lib.gc_combiner_create(policy, max_size, static_n, window, C.byref(h)),
               "gc_combiner_create")
        self.h, self.lib = h, lib

    def arrive(self, t_ns, count=1):
        _check(self.lib.gc_combiner_arrive(self.h, int(t_ns), int(count)), "gc_combiner_arrive")

    def poll(self, t_ns, queued):
        v = C.c_uint64()
        _check(self.lib.gc_combiner_poll(self.h, int(t_ns), int(queued), C.byref(v)),
               "gc_combiner_poll")
        return v.value

    def max_interval(self):
        v = C.c_uint64()
        _check(self.lib.gc_combiner_max_interval(self.h, C.byref(v)), "gc_combiner_max_interval")
        return v.value

    def close(self):
        if self.h:
            self.lib.gc_combiner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_peak():
    """Measured FP32 TFLOP/s of the current device (paired-FMA probe)."""
    lib = load()
    tf, ms = C.c_double(), C.c_double()
    _check(lib.gc_fp32_peak(C.byref(tf), C.byref(ms)), "gc_fp32_peak")
    return tf.value


def combine_size_from_occupancy(occupancy, max_blocks_per_sm, n_sm):
    return load().gc_combine_size_from_occupancy(float(occupancy), int(max_blocks_per_sm),
                                                 int(n_sm))
