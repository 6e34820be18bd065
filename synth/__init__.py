"""Seeded synthetic hypergraphs shaped like the paper's benchmark classes.

This module generates inputs only.  It holds none of the partitioner's
arithmetic and is imported by the tests and the benchmark, which hand the
same arrays to the CPU oracle and to the CUDA library.

The paper evaluates on SuiteSparse matrices, SAT instances (primal, literal,
dual) and VLSI netlists (Sec. 12, "Benchmark Instances"); none of those sets
is available here, so the workloads below are seeded stand-ins with the
shapes the benchmark descriptions call for (net-size laws, degree skew,
weight ranges, k and epsilon).  The recipes are also written out in the
design notes of the repository.

Random source: xoshiro256** seeded through SplitMix64 (see synth.c).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (plain gcc, host only)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i64, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.syn_splitmix64_first.restype = u64
            lib.syn_splitmix64_first.argtypes = [u64]
            lib.syn_xoshiro_stream.argtypes = [u64, i64, vp]
            lib.syn_sizes_geometric.argtypes = [u64, i64, dbl, i32, i32, vp]
            lib.syn_sizes_zipf.argtypes = [u64, i64, dbl, i32, i32, vp]
            lib.syn_sizes_powerlaw.argtypes = [u64, i64, dbl, dbl, dbl, vp]
            lib.syn_pins_uniform.argtypes = [u64, i32, i64, vp, vp]
            lib.syn_pins_uniform.restype = ctypes.c_int
            lib.syn_pins_preferential.argtypes = [u64, i32, i64, vp, vp]
            lib.syn_pins_preferential.restype = ctypes.c_int
            lib.syn_uniform_ints.argtypes = [u64, i64, i32, i32, vp]
            lib.syn_uniform_doubles.argtypes = [u64, i64, vp]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- raw streams

def splitmix64_first(seed: int) -> int:
    """First SplitMix64 output for the given 64-bit state."""
    return int(_L().syn_splitmix64_first(seed & 0xFFFFFFFFFFFFFFFF))


def xoshiro_stream(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _L().syn_xoshiro_stream(seed & 0xFFFFFFFFFFFFFFFF, count, _p(out))
    return out


def sub_seed(seed: int, *tags: int) -> int:
    """Derive an independent stream seed from a run seed and integer tags."""
    x = seed & 0xFFFFFFFFFFFFFFFF
    for t in tags:
        x = splitmix64_first(x ^ ((t * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF))
    return x


def uniform_ints(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int32)
    _L().syn_uniform_ints(seed, count, lo, hi, _p(out))
    return out


def uniform_doubles(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _L().syn_uniform_doubles(seed, count, _p(out))
    return out


# ---------------------------------------------------------------- containers

@dataclass
class Hypergraph:
    """Net-major CSR: the pins of net e are pins[offsets[e]:offsets[e+1]]."""
    n: int
    m: int
    offsets: np.ndarray   # int32 [m+1]
    pins: np.ndarray      # int32 [p]
    net_w: np.ndarray     # int32 [m]
    node_w: np.ndarray    # int32 [n]
    name: str = ""

    @property
    def p(self) -> int:
        return int(self.offsets[-1])

    def total_node_weight(self) -> int:
        return int(self.node_w.astype(np.int64).sum())


def sizes_geometric(seed, m, prob, base, cap):
    out = np.empty(m, dtype=np.int32)
    _L().syn_sizes_geometric(seed, m, prob, base, cap, _p(out))
    return out


def sizes_zipf(seed, m, s, lo, hi):
    out = np.empty(m, dtype=np.int32)
    _L().syn_sizes_zipf(seed, m, s, lo, hi, _p(out))
    return out


def sizes_powerlaw(seed, m, alpha, lo, hi):
    out = np.empty(m, dtype=np.int32)
    _L().syn_sizes_powerlaw(seed, m, alpha, float(lo), float(hi), _p(out))
    return out


def _offsets(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def pins_for(seed, n, sizes, preferential=False):
    off64 = _offsets(sizes)
    pins = np.empty(int(off64[-1]), dtype=np.int32)
    fn = _L().syn_pins_preferential if preferential else _L().syn_pins_uniform
    rc = fn(seed, n, len(sizes), _p(off64), _p(pins))
    if rc != 0:
        raise ValueError(f"pin generation failed ({rc})")
    if off64[-1] >= 2 ** 31:
        raise ValueError("too many pins for int32 offsets")
    return off64.astype(np.int32), pins


def make(seed, n, m, sizes, preferential, node_w_range, net_w_range, name=""):
    off, pins = pins_for(sub_seed(seed, 2), n, sizes, preferential)
    nw = (np.ones(n, np.int32) if node_w_range is None
          else uniform_ints(sub_seed(seed, 3), n, *node_w_range))
    ew = (np.ones(m, np.int32) if net_w_range is None
          else uniform_ints(sub_seed(seed, 4), m, *net_w_range))
    return Hypergraph(n, m, off, pins, ew, nw, name)


# ---------------------------------------------------------------- workloads

def random_uniform(seed: int, n: int, m: int, geom_p: float = 0.3, cap: int = 64,
                   node_w=None, net_w=None, name="random") -> Hypergraph:
    """Net sizes 2 + Geometric(geom_p) capped at cap, pins uniform without repeats."""
    sizes = sizes_geometric(sub_seed(seed, 1), m, geom_p, 2, min(cap, n))
    return make(seed, n, m, sizes, False, node_w, net_w, name)


def uniform_10k(seed: int = 1) -> Hypergraph:
    """Plain single level: n = m = 10,000, unit weights, sizes 2 + Geom(0.3) <= 64."""
    return random_uniform(seed, 10_000, 10_000, name="uniform10k")


def zipf_preferential(seed: int, n: int, m: int, s: float = 2.2, lo: int = 2, hi: int = 1024,
                      w_lo: int = 1, w_hi: int = 10, name="zipf") -> Hypergraph:
    """Zipf(s) net sizes on [lo, hi], preferential pins, weights uniform in [w_lo, w_hi]."""
    sizes = sizes_zipf(sub_seed(seed, 1), m, s, lo, min(hi, n))
    return make(seed, n, m, sizes, True, (w_lo, w_hi), (w_lo, w_hi), name)


def zipf_1m(seed: int = 1, n: int = 1_000_000, m: int | None = None) -> Hypergraph:
    """Full hierarchy workload: n = m = 1e6, Zipf(2.2) sizes in [2, 1024],
    heavy-tailed node degrees, node and net weights uniform in [1, 10]."""
    return zipf_preferential(seed, n, n if m is None else m, name=f"zipf_n{n}")


def graph_preferential(seed: int, n: int, m: int, w_lo: int = 1, w_hi: int = 10,
                       name="graph") -> Hypergraph:
    """A graph as a hypergraph whose nets all have two pins: m edges with
    preferential endpoints (heavy-tailed degrees; parallel edges possible),
    node and edge weights uniform in [w_lo, w_hi]."""
    sizes = np.full(m, 2, dtype=np.int32)
    return make(seed, n, m, sizes, True, (w_lo, w_hi), (w_lo, w_hi), name)


def graph_uniform(seed: int, n: int, m: int, name="graph_uniform") -> Hypergraph:
    """m edges with uniform endpoints, unit weights."""
    return random_uniform(seed, n, m, geom_p=1.0, cap=2, name=name)


def large_net_stress(seed: int, n: int, m: int, big_every: int = 100, big_lo: int = 1000,
                     big_hi: int = 100_000, alpha: float = 4.0, force_first: int | None = None,
                     name="stress") -> Hypergraph:
    """99 % small nets (2 + Geom(0.3) <= 16), every big_every-th net large with
    size density x^-alpha on [big_lo, big_hi]; net 0 forced to force_first pins."""
    sizes = sizes_geometric(sub_seed(seed, 1), m, 0.3, 2, 16)
    big = np.arange(0, m, big_every)
    hi = min(big_hi, n)
    sizes[big] = sizes_powerlaw(sub_seed(seed, 5), len(big), alpha, min(big_lo, hi), hi)
    if force_first is not None:
        sizes[0] = min(force_first, n)
    return make(seed, n, m, sizes, False, None, (1, 100), name)


def large_net_4m(seed: int = 1, n: int = 4_000_000, m: int = 2_000_000) -> Hypergraph:
    """Large-net stress: n = 4e6, m = 2e6, 1 % nets of 1k-100k pins, net 0 = 100k pins."""
    return large_net_stress(seed, n, m, force_first=100_000, name=f"large_net_n{n}")


def batch_instances(seed: int = 1, count: int = 512, n_lo: int = 1000, n_hi: int = 200_000):
    """Batch of independent instances: n log-uniform in [n_lo, n_hi], m/n in
    [0.5, 3], sizes as uniform_10k, weights in [1, 10], k in {2,4,8,16,32}."""
    u = uniform_doubles(sub_seed(seed, 40), 3 * count).reshape(count, 3)
    ks = (2, 4, 8, 16, 32)
    out = []
    for i in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[i, 0] * (math.log(n_hi) - math.log(n_lo)))))
        m = max(1, int(round(n * (0.5 + 2.5 * u[i, 1]))))
        k = ks[min(4, int(u[i, 2] * 5))]
        hg = random_uniform(sub_seed(seed, 41, i), n, m, node_w=(1, 10), net_w=(1, 10),
                            name=f"batch_{i}")
        out.append((hg, k))
    return out


def poisson_arrivals(seed: int = 1, rate: float = 200.0, duration: float = 60.0,
                     pins_lo: float = 1e4, pins_hi: float = 2e6):
    """Poisson arrivals: list of (arrival_s, request_seed, target_pins, k)."""
    cap = int(rate * duration * 2 + 100)
    u = uniform_doubles(sub_seed(seed, 50), 3 * cap).reshape(cap, 3)
    t = 0.0
    out = []
    for i in range(cap):
        t += -math.log(1.0 - u[i, 0]) / rate
        if t >= duration:
            break
        pins = math.exp(math.log(pins_lo) + u[i, 1] * (math.log(pins_hi) - math.log(pins_lo)))
        k = (2, 8, 32)[min(2, int(u[i, 2] * 3))]
        out.append((t, sub_seed(seed, 51, i), int(round(pins)), k))
    return out


def poisson_request(req_seed: int, target_pins: int) -> Hypergraph:
    """One serving request: m = n = round(pins / 6.8), Zipf(2.2) sizes in [2, 1024]."""
    m = max(2, int(round(target_pins / 6.8)))
    sizes = sizes_zipf(sub_seed(req_seed, 1), m, 2.2, 2, min(1024, m))
    return make(req_seed, m, m, sizes, False, None, None, name="poisson_req")

