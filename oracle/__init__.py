"""CPU oracle for the deterministic coarsen + label-propagation level.

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, loads or calls it.

The arithmetic lives in ``oracle.cpp`` (plain single-threaded C++17, built
with g++); this module only marshals numpy arrays through ctypes and composes
the multilevel loop of Algorithm 1 from the per-level routines.  Inputs are
any object with the attributes ``n, m, offsets, pins, net_w, node_w``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (host C++ only; no CUDA)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32, i64, u64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
            lib.o_mix64.restype = u64
            lib.o_mix64.argtypes = [u64]
            lib.o_subround_clustering.restype = i32
            lib.o_subround_clustering.argtypes = [u64, i32, i32, i32]
            lib.o_subround_lp.restype = i32
            lib.o_subround_lp.argtypes = [u64, i32, i32, i32, i32]
            lib.o_pin_counts.argtypes = [i32, i32, vp, vp, i32, vp, vp, vp]
            lib.o_objective.restype = i64
            lib.o_objective.argtypes = [i32, i32, vp, vp, vp, i32, vp]
            lib.o_gains.argtypes = [i32, i32, vp, vp, vp, i32, vp, vp]
            lib.o_block_weights.argtypes = [i32, vp, i32, vp, vp]
            lib.o_gain_table.argtypes = [i32, i32, vp, vp, vp, i32, vp, vp, vp]
            lib.o_recalculate_gains.restype = i32
            lib.o_recalculate_gains.argtypes = [i32, i32, vp, vp, vp, i32, vp, i32, vp, vp, vp]
            lib.o_balance_limit.restype = i64
            lib.o_balance_limit.argtypes = [i64, i32, i32]
            lib.o_lp_refine.restype = i32
            lib.o_lp_refine.argtypes = [i32, i32, vp, vp, vp, vp, i32, i32, i32, u64, i32, i32,
                                        vp, vp, vp, vp, vp, vp, vp]
            lib.o_lp_subround.restype = i32
            lib.o_lp_subround.argtypes = [i32, i32, vp, vp, vp, vp, i32, i32, i32, u64, i32, i32,
                                          i32, vp, vp, vp, vp, vp, vp]
            lib.o_coarsen.restype = i32
            lib.o_coarsen.argtypes = [i32, i32, vp, vp, vp, vp, i64, i32, i32, i32, i32, u64, i32,
                                      vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.o_bipartite.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
            lib.o_louvain_best_move.restype = i32
            lib.o_louvain_best_move.argtypes = [i32, vp, vp, vp, vp, vp, vp, i32]
            lib.o_louvain_aggregate.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.o_communities.argtypes = [i32, i32, vp, vp, vp, i32, u64, i32, i32, vp, vp]
            lib.o_contract.restype = i32
            lib.o_contract.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.o_project.argtypes = [i32, vp, vp, vp]
            lib.o_initial_partition.argtypes = [i32, vp, i32, u64, vp]
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return ctypes.c_void_p(a.ctypes.data)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Level:
    """A hypergraph level in net-major CSR (same attribute names as the inputs)."""
    n: int
    m: int
    offsets: np.ndarray
    pins: np.ndarray
    net_w: np.ndarray
    node_w: np.ndarray
    name: str = ""

    @property
    def p(self) -> int:
        return int(self.offsets[-1])


def _arrs(hg):
    return (_i32(hg.offsets), _i32(hg.pins), _i32(hg.net_w), _i32(hg.node_w))


# ------------------------------------------------------------------ hashing

def mix64(x: int) -> int:
    return int(_L().o_mix64(x & 0xFFFFFFFFFFFFFFFF))


def subround_clustering(seed: int, level: int, u: int, S: int) -> int:
    return int(_L().o_subround_clustering(seed, level, u, S))


def subround_lp(seed: int, level: int, pass_: int, u: int, S: int) -> int:
    return int(_L().o_subround_lp(seed, level, pass_, u, S))


# --------------------------------------------------------- partition values

def pin_counts(hg, k: int, part):
    off, pins, _, _ = _arrs(hg)
    part = _i32(part)
    phi = np.zeros((hg.m, k), dtype=np.int32)
    lam = np.zeros(hg.m, dtype=np.uint64)
    _L().o_pin_counts(hg.n, hg.m, _p(off), _p(pins), k, _p(part), _p(phi), _p(lam))
    return phi, lam


def objective(hg, k: int, part) -> int:
    off, pins, w, _ = _arrs(hg)
    part = _i32(part)
    return int(_L().o_objective(hg.n, hg.m, _p(off), _p(pins), _p(w), k, _p(part)))


def gains(hg, k: int, part) -> np.ndarray:
    off, pins, w, _ = _arrs(hg)
    part = _i32(part)
    out = np.zeros((hg.n, k), dtype=np.int64)
    _L().o_gains(hg.n, hg.m, _p(off), _p(pins), _p(w), k, _p(part), _p(out))
    return out


def gain_table(hg, k: int, part):
    """(b [n] int64, p [n, k] int64) of Sec. 6.2 for partition `part`."""
    off, pins, w, _ = _arrs(hg)
    part = _i32(part)
    b = np.zeros(max(hg.n, 1), np.int64)
    p = np.zeros((max(hg.n, 1), k), np.int64)
    _L().o_gain_table(hg.n, hg.m, _p(off), _p(pins), _p(w), k, _p(part), _p(b), _p(p))
    return b[:hg.n], p[:hg.n]


def recalculate_gains(hg, k: int, part, nodes, targets) -> np.ndarray:
    """Exact gains of the move sequence (nodes[i] -> targets[i], in this
    order) from partition `part` (Sec. 6.3)."""
    off, pins, w, _ = _arrs(hg)
    part, nodes, targets = _i32(part), _i32(nodes), _i32(targets)
    out = np.zeros(max(len(nodes), 1), np.int64)
    rc = _L().o_recalculate_gains(hg.n, hg.m, _p(off), _p(pins), _p(w), k, _p(part), len(nodes),
                                  _p(nodes), _p(targets), _p(out))
    if rc != 0:
        raise ValueError("invalid move sequence")
    return out[:len(nodes)]


def block_weights(hg, k: int, part) -> np.ndarray:
    c = _i32(hg.node_w)
    part = _i32(part)
    out = np.zeros(k, dtype=np.int64)
    _L().o_block_weights(hg.n, _p(c), k, _p(part), _p(out))
    return out


def balance_limit(W: int, k: int, eps_ppm: int) -> int:
    return int(_L().o_balance_limit(W, k, eps_ppm))


# ---------------------------------------------------------- label propagation

def lp_refine(hg, k: int, part, eps_ppm: int = 30000, S: int = 16, seed: int = 1, level: int = 0,
              max_passes: int = 5, want_phi: bool = False, want_trace: bool = False):
    off, pins, w, c = _arrs(hg)
    part = _i32(part).copy()
    obj = ctypes.c_int64(0)
    moves = ctypes.c_int64(0)
    passes = ctypes.c_int32(0)
    phi = np.zeros((hg.m, k), dtype=np.int32) if want_phi else None
    tc = np.zeros(max(1, max_passes * S), dtype=np.int64) if want_trace else None
    ta = np.zeros(max(1, max_passes * S), dtype=np.int64) if want_trace else None
    rc = _L().o_lp_refine(hg.n, hg.m, _p(off), _p(pins), _p(w), _p(c), k, eps_ppm, S, seed, level,
                          max_passes, _p(part), ctypes.byref(obj), ctypes.byref(moves),
                          ctypes.byref(passes), _p(phi), _p(tc), _p(ta))
    if rc != 0:
        raise ValueError(f"o_lp_refine rejected its arguments ({rc})")
    out = dict(part=part, objective=int(obj.value), moves=int(moves.value), passes=int(passes.value))
    if want_phi:
        out["phi"] = phi
    if want_trace:
        out["candidates"] = tc[: max_passes * S].reshape(max_passes, S)
        out["applied"] = ta[: max_passes * S].reshape(max_passes, S)
    return out


def lp_subround(hg, k: int, part, eps_ppm: int, S: int, seed: int, level: int, pass_: int, s: int):
    """One sub-round; returns (new_part, moves) with moves a structured record array."""
    off, pins, w, c = _arrs(hg)
    part = _i32(part).copy()
    n = hg.n
    u = np.zeros(max(n, 1), np.int32)
    fr = np.zeros(max(n, 1), np.int32)
    to = np.zeros(max(n, 1), np.int32)
    g = np.zeros(max(n, 1), np.int64)
    ap = np.zeros(max(n, 1), np.int8)
    cnt = _L().o_lp_subround(n, hg.m, _p(off), _p(pins), _p(w), _p(c), k, eps_ppm, S, seed, level,
                             pass_, s, _p(part), _p(u), _p(fr), _p(to), _p(g), _p(ap))
    if cnt < 0:
        raise ValueError("o_lp_subround rejected its arguments")
    moves = dict(u=u[:cnt].copy(), src=fr[:cnt].copy(), dst=to[:cnt].copy(), gain=g[:cnt].copy(),
                 applied=ap[:cnt].astype(bool))
    return part, moves


# -------------------------------------------------------------- coarsening

def coarsen(hg, W: int, k: int, S: int = 16, T: int = 1000, factor: int = 160, seed: int = 1,
            level: int = 0, comm=None):
    """One clustering + contraction level.  Returns None when no level is
    built (n <= factor * k), else a dict with the coarse Level and traces.
    comm: community of every node (candidates stay inside u's community);
    the result then also holds the coarse nodes' communities."""
    off, pins, w, c = _arrs(hg)
    cm = None if comm is None else _i32(comm)
    ccomm = np.zeros(max(hg.n, 1), np.int32)
    n, m, p = hg.n, hg.m, int(off[-1])
    rep = np.zeros(max(n, 1), np.int32)
    target = np.zeros(max(n, 1), np.int32)
    rated = np.zeros(max(n, 1), np.int32)
    mp = np.zeros(max(n, 1), np.int32)
    on, om, op = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    coff = np.zeros(m + 1, np.int32)
    cpins = np.zeros(max(p, 1), np.int32)
    cw = np.zeros(max(m, 1), np.int32)
    cc = np.zeros(max(n, 1), np.int32)
    stop_after = ctypes.c_int32(0)
    rc = _L().o_coarsen(n, m, _p(off), _p(pins), _p(w), _p(c), W, k, S, T, factor, seed, level,
                        _p(rep), _p(target), _p(rated), _p(mp), ctypes.byref(on), ctypes.byref(om),
                        ctypes.byref(op), _p(coff), _p(cpins), _p(cw), _p(cc),
                        ctypes.byref(stop_after), _p(cm), _p(ccomm))
    if rc == 1:
        return None
    n2, m2, p2 = on.value, om.value, op.value
    lvl = Level(n2, m2, coff[: m2 + 1].copy(), cpins[:p2].copy(), cw[:m2].copy(), cc[:n2].copy())
    out = dict(level=lvl, rep=rep[:n].copy(), target=target[:n].copy(), rated_in=rated[:n].copy(),
               map=mp[:n].copy(), stop_after=bool(stop_after.value))
    if comm is not None:
        out["comm"] = ccomm[:n2].copy()
    return out


# ------------------------------------------------------------ communities

def bipartite(hg):
    """Bipartite graph of Sec. 4: (V, offsets int64 [V+1], adj int32, weights int64)."""
    off, pins, w, _ = _arrs(hg)
    V = hg.n + hg.m
    p = int(off[-1])
    boff = np.zeros(V + 1, np.int64)
    badj = np.zeros(max(2 * p, 1), np.int32)
    bw = np.zeros(max(2 * p, 1), np.int64)
    _L().o_bipartite(hg.n, hg.m, _p(off), _p(pins), _p(w), _p(boff), _p(badj), _p(bw))
    return V, boff, badj[: 2 * p], bw[: 2 * p]


def louvain_best_move(V, off, adj, w, self_w, cl, vol, i) -> int:
    """Target cluster of vertex i under the state (cl, vol), or -1."""
    a = [np.ascontiguousarray(x, t) for x, t in ((off, np.int64), (adj, np.int32), (w, np.int64),
                                                 (self_w, np.int64), (cl, np.int32), (vol, np.int64))]
    return int(_L().o_louvain_best_move(V, *[_p(x) for x in a], i))


def louvain_aggregate(V, off, adj, w, self_w, cl):
    """(V2, off2, adj2, w2, self2, cid) of the aggregation of clustering cl."""
    a = [np.ascontiguousarray(x, t) for x, t in ((off, np.int64), (adj, np.int32), (w, np.int64),
                                                 (self_w, np.int64), (cl, np.int32))]
    e = max(len(adj), 1)
    V2 = ctypes.c_int32(0)
    off2 = np.zeros(V + 1, np.int64)
    adj2 = np.zeros(e, np.int32)
    w2 = np.zeros(e, np.int64)
    self2 = np.zeros(max(V, 1), np.int64)
    cid = np.zeros(max(V, 1), np.int32)
    _L().o_louvain_aggregate(V, *[_p(x) for x in a], ctypes.byref(V2), _p(off2), _p(adj2), _p(w2),
                             _p(self2), _p(cid))
    v2 = V2.value
    q = int(off2[v2])
    return v2, off2[: v2 + 1].copy(), adj2[:q].copy(), w2[:q].copy(), self2[:v2].copy(), cid[:V].copy()


def communities(hg, S: int = 16, seed: int = 1, max_rounds: int = 5, max_levels: int = 32):
    """(community of every node, Louvain levels aggregated, vertex moves)."""
    off, pins, w, _ = _arrs(hg)
    comm = np.zeros(max(hg.n, 1), np.int32)
    stats = np.zeros(2, np.int64)
    _L().o_communities(hg.n, hg.m, _p(off), _p(pins), _p(w), S, seed, max_rounds, max_levels,
                       _p(comm), _p(stats))
    return comm[: hg.n].copy(), int(stats[0]), int(stats[1])


def contract(hg, rep):
    """Contraction of the clustering rep (Sec. 4.2).  Returns (Level, map)."""
    off, pins, w, c = _arrs(hg)
    rep = _i32(rep)
    n, m, p = hg.n, hg.m, int(off[-1])
    mp = np.zeros(max(n, 1), np.int32)
    on, om, op = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    coff = np.zeros(m + 1, np.int32)
    cpins = np.zeros(max(p, 1), np.int32)
    cw = np.zeros(max(m, 1), np.int32)
    cc = np.zeros(max(n, 1), np.int32)
    rc = _L().o_contract(n, m, _p(off), _p(pins), _p(w), _p(c), _p(rep), _p(mp), ctypes.byref(on),
                         ctypes.byref(om), ctypes.byref(op), _p(coff), _p(cpins), _p(cw), _p(cc))
    if rc != 0:
        raise ValueError("rep is not a valid representative array")
    n2, m2, p2 = on.value, om.value, op.value
    lvl = Level(n2, m2, coff[: m2 + 1].copy(), cpins[:p2].copy(), cw[:m2].copy(), cc[:n2].copy())
    return lvl, mp[:n].copy()


def project(fine_map, coarse_part) -> np.ndarray:
    fine_map = _i32(fine_map)
    coarse_part = _i32(coarse_part)
    out = np.zeros(len(fine_map), np.int32)
    _L().o_project(len(fine_map), _p(fine_map), _p(coarse_part), _p(out))
    return out


def initial_partition(node_w, k: int, seed: int) -> np.ndarray:
    c = _i32(node_w)
    out = np.zeros(len(c), np.int32)
    _L().o_initial_partition(len(c), _p(c), k, seed, _p(out))
    return out


# --------------------------------------------------------- multilevel loop

@dataclass
class VCycle:
    levels: list = field(default_factory=list)     # Level objects, finest first
    maps: list = field(default_factory=list)       # maps[l]: level l -> level l+1
    parts: list = field(default_factory=list)      # final partition per level
    objectives: list = field(default_factory=list) # objective after LP per level
    moves: list = field(default_factory=list)
    initial_objective: int = 0
    communities: object = None                     # community of every node (or None)


def multilevel(hg, k: int, eps_ppm: int = 30000, S: int = 16, T: int = 1000, factor: int = 160,
               seed: int = 1, max_passes: int = 5, max_levels: int = 64,
               communities_first: bool = False) -> VCycle:
    """Algorithm 1 restricted to the deterministic path: coarsen until a stop
    rule fires, seeded initial partition of the coarsest level, then label
    propagation on every level from the coarsest to the finest, projecting
    between levels.  communities_first: detect communities (Sec. 4) before
    coarsening and keep every contraction inside a community."""
    W = int(np.asarray(hg.node_w, dtype=np.int64).sum())
    vc = VCycle()
    vc.levels.append(hg)
    comm = communities(hg, S, seed)[0] if communities_first else None
    vc.communities = comm
    for lv in range(max_levels):
        r = coarsen(vc.levels[-1], W, k, S, T, factor, seed, lv, comm)
        if r is None:
            break
        vc.maps.append(r["map"])
        vc.levels.append(r["level"])
        if comm is not None:
            comm = r["comm"]
        if r["stop_after"]:
            break
    L = len(vc.levels) - 1
    part = initial_partition(vc.levels[L].node_w, k, seed)
    vc.initial_objective = objective(vc.levels[L], k, part)
    parts = [None] * (L + 1)
    objs = [0] * (L + 1)
    mv = [0] * (L + 1)
    for lv in range(L, -1, -1):
        if lv < L:
            part = project(vc.maps[lv], part)
        res = lp_refine(vc.levels[lv], k, part, eps_ppm, S, seed, lv, max_passes)
        part = res["part"]
        parts[lv] = part
        objs[lv] = res["objective"]
        mv[lv] = res["moves"]
    vc.parts, vc.objectives, vc.moves = parts, objs, mv
    return vc
