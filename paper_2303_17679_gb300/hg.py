"""Thin Python binding of the C ABI in include/hg.h.

Every function has the name of the C entry point it calls and only marshals
arguments: host arrays are numpy arrays, device arrays are CUDA tensors (or
raw device pointers), streams are torch streams (or raw cudaStream_t
values).  All computation happens in libhg.so; if the library cannot be
loaded, every call raises - there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhg.so")

HG_OK = 0
HG_STOP = 1
HG_ERR_INVALID = -1
HG_ERR_UNSUPPORTED = -2
HG_ERR_OOM = -3
HG_ERR_CUDA = -4
HG_ERR_TIMEOUT = -5
HG_ERR_STATE = -6
HG_MEM_HOST = 0
HG_MEM_DEVICE = 1
HG_MAX_K = 64

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class hg_options(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("subrounds", ctypes.c_int32),
        ("rating_max_net_size", ctypes.c_int32),
        ("contraction_limit_factor", ctypes.c_int32),
        ("fingerprint_bits", ctypes.c_int32),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("rate_warp_max_d", ctypes.c_int32),
        ("rate_pair_max_d", ctypes.c_int32),
        ("rate_quad_max_d", ctypes.c_int32),
        ("rate_block_max_d", ctypes.c_int32),
        ("lp_block_min_deg", ctypes.c_int32),
        ("blocking_sync", ctypes.c_int32),
        ("graph_path", ctypes.c_int32),
        ("community_detection", ctypes.c_int32),
    ]

    TUNABLE = ("rate_warp_max_d", "rate_pair_max_d", "rate_quad_max_d", "rate_block_max_d",
               "lp_block_min_deg")


class hg_job(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("m", ctypes.c_int32),
        ("net_offsets", ctypes.c_void_p), ("pins", ctypes.c_void_p),
        ("net_weights", ctypes.c_void_p), ("node_weights", ctypes.c_void_p),
        ("k", ctypes.c_int32), ("eps_ppm", ctypes.c_int32), ("max_passes", ctypes.c_int32),
        ("part_out", ctypes.c_void_p), ("tag", ctypes.c_int64),
    ]


class hg_job_result(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_int64), ("tag", ctypes.c_int64),
        ("status", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("objective", ctypes.c_int64), ("level_pins", ctypes.c_int64),
        ("est_bytes", ctypes.c_int64),
        ("t_submit_ns", ctypes.c_int64), ("t_start_ns", ctypes.c_int64), ("t_end_ns", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class hg_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in (
        "ms_transpose", "ms_rating", "ms_approve", "ms_contract", "ms_project", "ms_phi",
        "ms_lp_gain", "ms_lp_select", "ms_lp_apply", "ms_objective", "ms_initial")] + [
        (name, ctypes.c_int64) for name in (
            "launches", "rating_launches", "rating_pin_visits", "rating_nodes",
            "rating_incidences", "lp_incidences", "lp_nodes", "lp_gain_launches")] + [
        ("ms_rating_kernels", ctypes.c_double), ("ms_lp_gain_kernels", ctypes.c_double),
        ("ms_rating_refresh", ctypes.c_double),
        ("ms_rating_class", ctypes.c_double * 8), ("rating_visits_class", ctypes.c_int64 * 8),
        ("ms_lp_select_kernels", ctypes.c_double), ("ms_lp_apply_kernels", ctypes.c_double),
        ("lp_moved_incidences", ctypes.c_int64), ("lp_passes", ctypes.c_int64),
        ("timing_failures", ctypes.c_int64), ("ms_communities", ctypes.c_double),
        ("louvain_levels", ctypes.c_int64), ("louvain_rounds", ctypes.c_int64),
        ("louvain_moves", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class HgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {hg_strerror(status)} ({status})")


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Loads libhg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libhg.so not found at {p}: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        i32, i64, vp, P = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER
        H = ctypes.c_void_p
        sig = {
            "hg_default_options": (None, [P(hg_options)]),
            "hg_create": (ctypes.c_int, [i32, i32, vp, vp, vp, vp, i32, P(hg_options), vp, P(H)]),
            "hg_coarsen_level": (ctypes.c_int, [H, i32, P(i32), P(i32), P(i32), P(i64)]),
            "hg_num_levels": (ctypes.c_int, [H, P(i32)]),
            "hg_level_info": (ctypes.c_int, [H, i32, P(i32), P(i32), P(i64)]),
            "hg_initial_partition": (ctypes.c_int, [H, i32, i32, vp]),
            "hg_project": (ctypes.c_int, [H, i32, vp, vp]),
            "hg_lp_refine": (ctypes.c_int, [H, i32, i32, i32, i32, vp, P(i64), P(i64)]),
            "hg_objective": (ctypes.c_int, [H, i32, i32, vp, P(i64)]),
            "hg_pin_counts": (ctypes.c_int, [H, i32, i32, vp, vp, vp, vp]),
            "hg_recalculate_gains": (ctypes.c_int, [H, i32, i32, vp, i32, vp, vp, vp]),
            "hg_gain_table": (ctypes.c_int, [H, i32, i32, vp, vp, vp]),
            "hg_gain_table_move": (ctypes.c_int, [H, i32, i32, vp, i32, vp, vp, vp, vp]),
            "hg_objective_noalloc": (ctypes.c_int, [i32, i32, i64, vp, vp, vp, vp, i32, vp, vp,
                                                    P(i64), vp]),
            "hg_partition": (ctypes.c_int, [H, i32, i32, i32, vp, P(i64)]),
            "hg_get_level": (ctypes.c_int, [H, i32, vp, vp, vp, vp, vp, vp]),
            "hg_get_incidence": (ctypes.c_int, [H, i32, vp, vp]),
            "hg_truncate": (ctypes.c_int, [H, i32]),
            "hg_enable_timing": (ctypes.c_int, [H, i32]),
            "hg_get_stats": (ctypes.c_int, [H, P(hg_stats)]),
            "hg_reset_stats": (ctypes.c_int, [H]),
            "hg_destroy": (ctypes.c_int, [H]),
            "hg_trim_memory": (ctypes.c_int, []),
            "hg_level_is_graph": (ctypes.c_int, [H, i32, P(i32)]),
            "hg_detect_communities": (ctypes.c_int, [H, P(i32)]),
            "hg_get_communities": (ctypes.c_int, [H, i32, vp]),
            "hg_calibrate_smem_atomics": (ctypes.c_int, [vp, P(ctypes.c_double),
                                                         P(ctypes.c_double)]),
            "hg_exec_create": (ctypes.c_int, [i32, i64, P(hg_options), P(H)]),
            "hg_exec_submit": (ctypes.c_int, [H, P(hg_job), P(i64)]),
            "hg_exec_wait": (ctypes.c_int, [H, i32, i32, P(hg_job_result), P(i32)]),
            "hg_exec_pending": (ctypes.c_int, [H, P(i32), P(i32)]),
            "hg_exec_now_ns": (ctypes.c_int64, []),
            "hg_exec_destroy": (ctypes.c_int, [H]),
            "hg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "hg_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return ["hg_default_options", "hg_create", "hg_coarsen_level", "hg_num_levels",
            "hg_level_info", "hg_initial_partition", "hg_project", "hg_lp_refine",
            "hg_objective", "hg_pin_counts", "hg_recalculate_gains", "hg_gain_table", "hg_gain_table_move",
            "hg_objective_noalloc", "hg_partition", "hg_get_level", "hg_get_incidence",
            "hg_truncate", "hg_enable_timing", "hg_get_stats", "hg_reset_stats", "hg_destroy", "hg_trim_memory", "hg_level_is_graph", "hg_detect_communities", "hg_get_communities", "hg_calibrate_smem_atomics",
            "hg_exec_create", "hg_exec_submit", "hg_exec_wait", "hg_exec_pending",
            "hg_exec_now_ns", "hg_exec_destroy", "hg_strerror", "hg_version"]


# ------------------------------------------------------------------ helpers

def _ptr(x):
    """Device or host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())  # torch tensor


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc: int, where: str, allow=(HG_OK,)):
    if rc not in allow:
        raise HgError(rc, where)
    return rc


def hg_strerror(status: int) -> str:
    return load().hg_strerror(status).decode()


def hg_version() -> str:
    return load().hg_version().decode()


def hg_default_options() -> hg_options:
    o = hg_options()
    load().hg_default_options(ctypes.byref(o))
    return o


class TorchAllocator:
    """Device allocation hooks backed by PyTorch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self._torch = torch
        self._device = device
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, size, _ctx):
        stream = self._torch.cuda.current_stream(self._device)
        return self._torch.cuda.caching_allocator_alloc(int(size), self._device, stream)

    def _do_free(self, ptr, _ctx):
        self._torch.cuda.caching_allocator_delete(int(ptr))

    def install(self, opt: hg_options):
        opt.dev_alloc = self._alloc
        opt.dev_free = self._free


# ------------------------------------------------------------------ entry points

def hg_create(n, m, net_offsets, pins, net_weights=None, node_weights=None, mem=HG_MEM_HOST,
              opt: hg_options | None = None, stream=None):
    """Returns an opaque handle (ctypes.c_void_p)."""
    h = ctypes.c_void_p()
    rc = load().hg_create(int(n), int(m), _ptr(net_offsets), _ptr(pins), _ptr(net_weights),
                          _ptr(node_weights), int(mem), ctypes.byref(opt) if opt else None,
                          _stream(stream), ctypes.byref(h))
    _check(rc, "hg_create")
    return h


def hg_coarsen_level(h, k):
    """Returns (status, level, n, m, p); status is HG_OK or HG_STOP."""
    lv, n, m, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    rc = load().hg_coarsen_level(h, int(k), ctypes.byref(lv), ctypes.byref(n), ctypes.byref(m),
                                 ctypes.byref(p))
    _check(rc, "hg_coarsen_level", (HG_OK, HG_STOP))
    return rc, lv.value, n.value, m.value, p.value


def hg_num_levels(h) -> int:
    x = ctypes.c_int32()
    _check(load().hg_num_levels(h, ctypes.byref(x)), "hg_num_levels")
    return x.value


def hg_detect_communities(h) -> int:
    """Detects communities on level 0 (before coarsening); returns their number."""
    x = ctypes.c_int32()
    _check(load().hg_detect_communities(h, ctypes.byref(x)), "hg_detect_communities")
    return x.value


def hg_get_communities(h, level):
    n, _, _ = hg_level_info(h, level)
    out = np.zeros(max(n, 1), np.int32)
    _check(load().hg_get_communities(h, int(level), _ptr(out)), "hg_get_communities")
    return out[:n]


def hg_level_is_graph(h, level) -> bool:
    x = ctypes.c_int32()
    _check(load().hg_level_is_graph(h, int(level), ctypes.byref(x)), "hg_level_is_graph")
    return bool(x.value)


def hg_level_info(h, level):
    n, m, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().hg_level_info(h, int(level), ctypes.byref(n), ctypes.byref(m), ctypes.byref(p)),
           "hg_level_info")
    return n.value, m.value, p.value


def hg_initial_partition(h, level, k, part):
    _check(load().hg_initial_partition(h, int(level), int(k), _ptr(part)), "hg_initial_partition")


def hg_project(h, coarse_level, coarse_part, fine_part):
    _check(load().hg_project(h, int(coarse_level), _ptr(coarse_part), _ptr(fine_part)), "hg_project")


def hg_lp_refine(h, level, k, eps_ppm, max_passes, part):
    """Returns (objective, moves)."""
    obj, mv = ctypes.c_int64(), ctypes.c_int64()
    _check(load().hg_lp_refine(h, int(level), int(k), int(eps_ppm), int(max_passes), _ptr(part),
                               ctypes.byref(obj), ctypes.byref(mv)), "hg_lp_refine")
    return obj.value, mv.value


def hg_objective(h, level, k, part) -> int:
    obj = ctypes.c_int64()
    _check(load().hg_objective(h, int(level), int(k), _ptr(part), ctypes.byref(obj)), "hg_objective")
    return obj.value


def hg_pin_counts(h, level, k, part):
    """Returns (phi [m, k] int32, lambda [m] uint64, block weights [k] int64) on the host."""
    n, m, _ = hg_level_info(h, level)
    phi = np.zeros((max(m, 1), k), np.int32)
    lam = np.zeros(max(m, 1), np.uint64)
    bw = np.zeros(k, np.int64)
    _check(load().hg_pin_counts(h, int(level), int(k), _ptr(part), _ptr(phi), _ptr(lam), _ptr(bw)),
           "hg_pin_counts")
    return phi[:m], lam[:m], bw


def hg_recalculate_gains(h, level, k, part, move_nodes, move_targets, gains):
    """All arrays are device tensors; gains (int64, len(move_nodes)) is written."""
    _check(load().hg_recalculate_gains(h, int(level), int(k), _ptr(part), int(len(move_nodes)),
                                       _ptr(move_nodes), _ptr(move_targets), _ptr(gains)),
           "hg_recalculate_gains")


def hg_gain_table(h, level, k, part, benefit, penalty):
    """Device tensors: benefit int64 [n], penalty int64 [n, k] are written."""
    _check(load().hg_gain_table(h, int(level), int(k), _ptr(part), _ptr(benefit), _ptr(penalty)),
           "hg_gain_table")


def hg_gain_table_move(h, level, k, part, move_nodes, move_targets, benefit, penalty):
    """Device tensors; part, benefit and penalty are updated in place."""
    _check(load().hg_gain_table_move(h, int(level), int(k), _ptr(part), int(len(move_nodes)),
                                     _ptr(move_nodes), _ptr(move_targets), _ptr(benefit),
                                     _ptr(penalty)), "hg_gain_table_move")


def hg_objective_noalloc(n, m, p, net_offsets, pins, net_weights, node_weights, k, part,
                         stream=None):
    """Objective and block weights of a partition of a device CSR, computed
    without a handle and without any device allocation.  Returns
    (objective, block weights [k] int64 numpy array)."""
    obj = ctypes.c_int64()
    bw = np.zeros(max(int(k), 1), np.int64)
    _check(load().hg_objective_noalloc(int(n), int(m), int(p), _ptr(net_offsets), _ptr(pins),
                                       _ptr(net_weights), _ptr(node_weights), int(k), _ptr(part),
                                       _stream(stream), ctypes.byref(obj), _ptr(bw)),
           "hg_objective_noalloc")
    return obj.value, bw[:k]


def hg_partition(h, k, eps_ppm, max_passes, part) -> int:
    obj = ctypes.c_int64()
    _check(load().hg_partition(h, int(k), int(eps_ppm), int(max_passes), _ptr(part),
                               ctypes.byref(obj)), "hg_partition")
    return obj.value


def hg_get_level(h, level, with_map=False):
    """Returns dict(offsets, pins, net_w, node_w[, map, rep]) as numpy arrays."""
    n, m, p = hg_level_info(h, level)
    out = dict(offsets=np.zeros(m + 1, np.int32), pins=np.zeros(max(p, 1), np.int32),
               net_w=np.zeros(max(m, 1), np.int32), node_w=np.zeros(max(n, 1), np.int32))
    mp = np.zeros(max(n, 1), np.int32) if with_map else None
    rp = np.zeros(max(n, 1), np.int32) if with_map else None
    _check(load().hg_get_level(h, int(level), _ptr(out["offsets"]), _ptr(out["pins"]),
                               _ptr(out["net_w"]), _ptr(out["node_w"]), _ptr(mp), _ptr(rp)),
           "hg_get_level")
    out["pins"], out["net_w"], out["node_w"] = out["pins"][:p], out["net_w"][:m], out["node_w"][:n]
    if with_map:
        out["map"], out["rep"] = mp[:n], rp[:n]
    return out


def hg_get_incidence(h, level):
    n, m, p = hg_level_info(h, level)
    off = np.zeros(n + 1, np.int32)
    nets = np.zeros(max(p, 1), np.int32)
    _check(load().hg_get_incidence(h, int(level), _ptr(off), _ptr(nets)), "hg_get_incidence")
    return off, nets[:p]


def hg_truncate(h, level):
    _check(load().hg_truncate(h, int(level)), "hg_truncate")


def hg_enable_timing(h, flags=1):
    """flags: 1 = per-phase event timing (synchronizing), 2 = event pair around
    every rating / gain kernel launch (no synchronization); 0 = off."""
    _check(load().hg_enable_timing(h, int(flags)), "hg_enable_timing")


def hg_get_stats(h) -> dict:
    s = hg_stats()
    _check(load().hg_get_stats(h, ctypes.byref(s)), "hg_get_stats")
    return s.as_dict()


def hg_reset_stats(h):
    _check(load().hg_reset_stats(h), "hg_reset_stats")


def hg_destroy(h):
    if h:
        load().hg_destroy(h)


def hg_calibrate_smem_atomics(stream=None):
    """Shared-memory atomic adds per second (32-bit, 64-bit) on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().hg_calibrate_smem_atomics(_stream(stream), ctypes.byref(a), ctypes.byref(b)),
           "hg_calibrate_smem_atomics")
    return a.value, b.value


def hg_trim_memory():
    """Returns the memory cached in the library's pool of the current device."""
    _check(load().hg_trim_memory(), "hg_trim_memory")


# ------------------------------------------------------------------ executor

def hg_exec_create(slots, mem_budget_bytes=0, opt: hg_options | None = None):
    ex = ctypes.c_void_p()
    _check(load().hg_exec_create(int(slots), int(mem_budget_bytes),
                                 ctypes.byref(opt) if opt else None, ctypes.byref(ex)),
           "hg_exec_create")
    return ex


def hg_exec_submit(ex, job: hg_job) -> int:
    t = ctypes.c_int64()
    _check(load().hg_exec_submit(ex, ctypes.byref(job), ctypes.byref(t)), "hg_exec_submit")
    return t.value


def hg_exec_wait(ex, max_results=64, timeout_ms=-1):
    buf = (hg_job_result * int(max_results))()
    cnt = ctypes.c_int32()
    _check(load().hg_exec_wait(ex, int(max_results), int(timeout_ms), buf, ctypes.byref(cnt)),
           "hg_exec_wait")
    return [buf[i].as_dict() for i in range(cnt.value)]


def hg_exec_pending(ex):
    q, r = ctypes.c_int32(), ctypes.c_int32()
    _check(load().hg_exec_pending(ex, ctypes.byref(q), ctypes.byref(r)), "hg_exec_pending")
    return q.value, r.value


def hg_exec_now_ns() -> int:
    return int(load().hg_exec_now_ns())


def hg_exec_destroy(ex):
    if ex:
        load().hg_exec_destroy(ex)


class Executor:
    """Keeps each job's host arrays alive until its result has been returned.

    Slots overlap on the device only as far as the CUDA runtime gives their
    streams separate hardware queues: set CUDA_DEVICE_MAX_CONNECTIONS=32 in
    the environment before the process creates its CUDA context."""

    def __init__(self, slots, mem_budget_bytes=0, opt: hg_options | None = None):
        self.ex = hg_exec_create(slots, mem_budget_bytes, opt)
        self.live = {}

    def submit(self, hgr, k, eps_ppm=30000, max_passes=5, tag=0):
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w)]
        part = np.zeros(max(hgr.n, 1), np.int32)
        job = hg_job(n=int(hgr.n), m=int(hgr.m), net_offsets=arrs[0].ctypes.data,
                     pins=arrs[1].ctypes.data if len(arrs[1]) else None,
                     net_weights=arrs[2].ctypes.data, node_weights=arrs[3].ctypes.data,
                     k=int(k), eps_ppm=int(eps_ppm), max_passes=int(max_passes),
                     part_out=part.ctypes.data, tag=int(tag))
        t = hg_exec_submit(self.ex, job)
        self.live[t] = (arrs, part[:hgr.n])
        return t

    def wait(self, max_results=64, timeout_ms=-1):
        out = []
        for r in hg_exec_wait(self.ex, max_results, timeout_ms):
            r["part"] = self.live.pop(r["ticket"])[1]
            out.append(r)
        return out

    def close(self):
        hg_exec_destroy(self.ex)
        self.ex = None
        self.live.clear()
