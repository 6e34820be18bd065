"""Small hand-built hypergraphs for the tests (inputs only, no method arithmetic)."""
from dataclasses import dataclass

import numpy as np


@dataclass
class H:
    n: int
    m: int
    offsets: np.ndarray
    pins: np.ndarray
    net_w: np.ndarray
    node_w: np.ndarray

    @property
    def p(self):
        return int(self.offsets[-1])


def from_nets(n, nets, net_w=None, node_w=None):
    sizes = [len(e) for e in nets]
    off = np.zeros(len(nets) + 1, np.int32)
    off[1:] = np.cumsum(sizes) if nets else []
    pins = np.array([v for e in nets for v in e], dtype=np.int32)
    w = np.ones(len(nets), np.int32) if net_w is None else np.asarray(net_w, np.int32)
    c = np.ones(n, np.int32) if node_w is None else np.asarray(node_w, np.int32)
    return H(n, len(nets), off, pins, w, c)


def nets_of(hg):
    return [list(hg.pins[hg.offsets[e]:hg.offsets[e + 1]]) for e in range(hg.m)]


def random_hypergraph(rng, n, m, max_size, w_hi=1, c_hi=1):
    nets = []
    for _ in range(m):
        s = int(rng.integers(1, min(max_size, n) + 1))
        nets.append(sorted(rng.choice(n, size=s, replace=False).tolist()))
    w = rng.integers(1, w_hi + 1, size=m)
    c = rng.integers(1, c_hi + 1, size=n)
    return from_nets(n, nets, w, c)
