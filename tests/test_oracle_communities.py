"""Pins of the oracle's community detection (Sec. 4 "Community-Aware
Coarsening", Sec. 11 "Deterministic Louvain Method") against what the
definitions fix, independently of the oracle's own arithmetic:

* the bipartite graph: one edge per pin, symmetric, every edge of net e
  weighted floor(w(e) 2^20 / |e|), within 2^-20 of the model weight w(e)/|e|;
* every move decision against the modularity of Newman and Girvan evaluated
  from its definition in exact rational arithmetic (Q before and after the
  move, for every candidate cluster): the chosen cluster is the argmax of the
  change (ties to the smaller id) and the vertex moves only if Q increases;
* aggregation: the modularity of a clustering equals that of the singleton
  clustering of the aggregated graph, and the total degree is kept;
* communities never span two connected components of the bipartite graph,
  and the detected clustering has a higher modularity than the singletons;
* community-aware coarsening: every cluster lies in one community; with a
  single community it equals the unrestricted coarsening, with one community
  per node nothing is contracted."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from tests.tiny import from_nets, random_hypergraph


def modularity(V, off, adj, w, self_w, cl):
    """Q = (1/2W) sum_ij (A_ij - k_i k_j / 2W) [c_i = c_j], A_ii = 2 self_i."""
    k = [Fraction(2 * int(self_w[i]) + sum(int(x) for x in w[off[i]:off[i + 1]])) for i in range(V)]
    two_w = sum(k)
    if two_w == 0:
        return Fraction(0)
    inside = Fraction(0)
    for i in range(V):
        inside += 2 * int(self_w[i])
        for q in range(off[i], off[i + 1]):
            if cl[adj[q]] == cl[i]:
                inside += int(w[q])
    vol = {}
    for i in range(V):
        vol[cl[i]] = vol.get(cl[i], 0) + k[i]
    return inside / two_w - sum((v / two_w) ** 2 for v in vol.values())


def random_graph(rng, V, E, wmax=9, self_max=3):
    edges = {}
    while len(edges) < E:
        a, b = (int(x) for x in rng.integers(0, V, size=2))
        if a != b:
            edges[(min(a, b), max(a, b))] = int(rng.integers(1, wmax + 1))
    adj = [[] for _ in range(V)]
    for (a, b), x in edges.items():
        adj[a].append((b, x))
        adj[b].append((a, x))
    off = np.zeros(V + 1, np.int64)
    off[1:] = np.cumsum([len(a) for a in adj])
    flat = np.array([b for a in adj for b, _ in a], np.int32)
    ws = np.array([x for a in adj for _, x in a], np.int64)
    self_w = rng.integers(0, self_max + 1, size=V).astype(np.int64)
    return off, flat, ws, self_w


def degrees(V, off, w, self_w):
    return np.array([2 * self_w[i] + w[off[i]:off[i + 1]].sum() for i in range(V)], np.int64)


def test_bipartite_graph_structure_and_weights(oracle_mod):
    rng = np.random.default_rng(1)
    hgr = random_hypergraph(rng, 30, 25, 7, w_hi=50)
    V, off, adj, w = oracle_mod.bipartite(hgr)
    assert V == hgr.n + hgr.m
    nets = [list(hgr.pins[hgr.offsets[e]:hgr.offsets[e + 1]]) for e in range(hgr.m)]
    pairs = set()
    for i in range(V):
        for q in range(off[i], off[i + 1]):
            pairs.add((i, int(adj[q]), int(w[q])))
    for e, pe in enumerate(nets):
        model = Fraction(int(hgr.net_w[e]), len(pe))
        for v in pe:
            got = [x for (a, b, x) in pairs if a == v and b == hgr.n + e]
            assert len(got) == 1 and (hgr.n + e, v, got[0]) in pairs
            assert 0 <= model - Fraction(got[0], 2 ** 20) < Fraction(1, 2 ** 20)
        assert off[hgr.n + e + 1] - off[hgr.n + e] == len(pe)
    assert len(adj) == 2 * hgr.p


@pytest.mark.parametrize("seed", range(6))
def test_move_decisions_maximise_exact_modularity(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    V = 9
    off, adj, w, self_w = random_graph(rng, V, 14)
    k = degrees(V, off, w, self_w)
    for trial in range(4):
        cl = rng.integers(0, V, size=V).astype(np.int32)
        vol = np.zeros(V, np.int64)
        for i in range(V):
            vol[cl[i]] += k[i]
        q0 = modularity(V, off, adj, w, self_w, cl)
        for i in range(V):
            cands = sorted({int(cl[adj[q]]) for q in range(off[i], off[i + 1])} - {int(cl[i])})
            best, best_dq = -1, None
            for c in cands:
                moved = cl.copy()
                moved[i] = c
                dq = modularity(V, off, adj, w, self_w, moved) - q0
                if best_dq is None or dq > best_dq:
                    best, best_dq = c, dq
            want = best if best_dq is not None and best_dq > 0 else -1
            got = oracle_mod.louvain_best_move(V, off, adj, w, self_w, cl, vol, i)
            assert got == want, (seed, trial, i, got, want)


@pytest.mark.parametrize("seed", range(4))
def test_aggregation_keeps_modularity_and_degrees(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    V = 12
    off, adj, w, self_w = random_graph(rng, V, 25)
    cl = rng.integers(0, 5, size=V).astype(np.int32)
    V2, off2, adj2, w2, self2, cid = oracle_mod.louvain_aggregate(V, off, adj, w, self_w, cl)
    assert V2 == len(set(cl.tolist()))
    assert degrees(V, off, w, self_w).sum() == degrees(V2, off2, w2, self2).sum()
    single = np.arange(V2, dtype=np.int32)
    assert modularity(V, off, adj, w, self_w, cl) == modularity(V2, off2, adj2, w2, self2, single)
    # the coarse vertex of a cluster is the rank of its id
    used = sorted(set(cl.tolist()))
    assert [int(cid[c]) for c in used] == list(range(V2))
    # aggregating the singleton clustering gives the graph back
    ident = np.arange(V, dtype=np.int32)
    V3, off3, adj3, w3, self3, _ = oracle_mod.louvain_aggregate(V, off, adj, w, self_w, ident)
    assert V3 == V and np.array_equal(self3, self_w)
    for i in range(V):
        a = sorted(zip(adj[off[i]:off[i + 1]].tolist(), w[off[i]:off[i + 1]].tolist()))
        b = sorted(zip(adj3[off3[i]:off3[i + 1]].tolist(), w3[off3[i]:off3[i + 1]].tolist()))
        assert a == b


def test_communities_stay_inside_components_and_raise_modularity(oracle_mod):
    # three groups of nodes with nets only inside a group
    nets = []
    rng = np.random.default_rng(7)
    for g in range(3):
        base = 40 * g
        for _ in range(60):
            size = int(rng.integers(2, 6))
            nets.append(sorted((base + rng.choice(40, size=size, replace=False)).tolist()))
    hgr = from_nets(120, nets, rng.integers(1, 10, size=len(nets)))
    comm, levels, moves = oracle_mod.communities(hgr, S=4, seed=3)
    assert moves > 0 and levels >= 1
    for c in set(comm.tolist()):
        groups = {int(v) // 40 for v in np.nonzero(comm == c)[0]}
        assert len(groups) == 1
    assert sorted(set(comm.tolist())) == list(range(comm.max() + 1))
    # modularity of the node communities extended to the net vertices (each
    # net joins the community holding most of its pin weight) beats singletons
    V, off, adj, w = oracle_mod.bipartite(hgr)
    cl = np.zeros(V, np.int32)
    cl[:hgr.n] = comm
    for e in range(hgr.m):
        pe = hgr.pins[hgr.offsets[e]:hgr.offsets[e + 1]]
        cl[hgr.n + e] = np.bincount(comm[pe]).argmax()
    zeros = np.zeros(V, np.int64)
    assert modularity(V, off, adj, w, zeros, cl) > modularity(V, off, adj, w, zeros,
                                                              np.arange(V, dtype=np.int32))
    again = oracle_mod.communities(hgr, S=4, seed=3)
    assert np.array_equal(again[0], comm)


def test_community_aware_coarsening(oracle_mod):
    hgr = synth.zipf_1m(5, n=3000)
    W = int(hgr.node_w.sum())
    comm, _, _ = oracle_mod.communities(hgr, S=16, seed=5)
    r = oracle_mod.coarsen(hgr, W, 4, 16, 1000, 10, 5, 0, comm)
    assert np.all(comm[r["rep"]] == comm)          # every cluster inside one community
    assert np.all(r["comm"][r["map"]] == comm)     # coarse communities follow the map
    one = oracle_mod.coarsen(hgr, W, 4, 16, 1000, 10, 5, 0, np.zeros(hgr.n, np.int32))
    plain = oracle_mod.coarsen(hgr, W, 4, 16, 1000, 10, 5, 0)
    assert np.array_equal(one["rep"], plain["rep"])
    assert np.array_equal(one["level"].pins, plain["level"].pins)
    alone = oracle_mod.coarsen(hgr, W, 4, 16, 1000, 10, 5, 0, np.arange(hgr.n, dtype=np.int32))
    assert alone["level"].n == hgr.n and alone["stop_after"]
