"""Pins for the oracle's partition values: objective, pin counts, gains.

None of these re-types the oracle's formulas: each compares against a library
routine on a special case (networkx edge cut on 2-pin nets, numpy bincount
for pin counts), a closed form, an invariance, or a brute-force consistency
between two different definitions of the paper (the gain of Sec. 6 against
the objective difference it is meant to measure).
"""
import itertools

import networkx as nx
import numpy as np
import pytest

from tests.tiny import from_nets, random_hypergraph


def test_mix64_published_vectors(oracle_mod):
    # SplitMix64 (Steele, Lea, Flood 2014): the generator seeded with 0 first
    # outputs 0xe220a8397b1dcdaf; seeded with 1234567, 6457827717110365317.
    assert oracle_mod.mix64(0) == 0xE220A8397B1DCDAF
    assert oracle_mod.mix64(1234567) == 6457827717110365317


@pytest.mark.parametrize("k", [2, 3, 5])
def test_graph_objective_is_weighted_edge_cut(oracle_mod, k):
    # Sec. 2: on plain graphs the connectivity metric reduces to the edge cut.
    rng = np.random.default_rng(10 + k)
    n = 40
    pairs = set()
    while len(pairs) < 120:
        a, b = rng.choice(n, size=2, replace=False)
        pairs.add((int(min(a, b)), int(max(a, b))))
    pairs = sorted(pairs)
    w = rng.integers(1, 9, size=len(pairs))
    hg = from_nets(n, [list(p) for p in pairs], w)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for (a, b), x in zip(pairs, w):
        G.add_edge(a, b, weight=int(x))
    for trial in range(10):
        part = rng.integers(0, k, size=n).astype(np.int32)
        total = G.size(weight="weight")
        inside = sum(G.subgraph(np.flatnonzero(part == b).tolist()).size(weight="weight")
                     for b in range(k))
        assert oracle_mod.objective(hg, k, part) == total - inside
        if k == 2:
            S = np.flatnonzero(part == 0).tolist()
            T = np.flatnonzero(part == 1).tolist()
            assert oracle_mod.objective(hg, k, part) == nx.cut_size(G, S, T, weight="weight")


def test_single_net_closed_form(oracle_mod):
    # one net over all nodes spread over j non-empty blocks contributes (j-1) w
    n, k = 12, 6
    hg = from_nets(n, [list(range(n))], [7])
    for j in range(1, k + 1):
        part = (np.arange(n) % j).astype(np.int32)
        assert oracle_mod.objective(hg, k, part) == (j - 1) * 7


def test_objective_invariances(oracle_mod):
    rng = np.random.default_rng(3)
    hg = random_hypergraph(rng, 30, 50, 8, w_hi=5)
    k = 4
    part = rng.integers(0, k, size=hg.n).astype(np.int32)
    f = oracle_mod.objective(hg, k, part)
    # relabelling blocks
    perm = rng.permutation(k).astype(np.int32)
    assert oracle_mod.objective(hg, k, perm[part]) == f
    # relabelling nodes consistently in the pins and the partition
    pi = rng.permutation(hg.n)
    hg2 = from_nets(hg.n, [[int(pi[v]) for v in hg.pins[hg.offsets[e]:hg.offsets[e + 1]]]
                           for e in range(hg.m)], hg.net_w)
    part2 = np.empty_like(part)
    part2[pi] = part
    assert oracle_mod.objective(hg2, k, part2) == f
    # all nodes in one block: nothing is cut
    assert oracle_mod.objective(hg, k, np.zeros(hg.n, np.int32)) == 0


def test_pin_counts_match_bincount(oracle_mod):
    rng = np.random.default_rng(4)
    hg = random_hypergraph(rng, 50, 80, 12)
    for k in (2, 7, 64):
        part = rng.integers(0, k, size=hg.n).astype(np.int32)
        phi, lam = oracle_mod.pin_counts(hg, k, part)
        for e in range(hg.m):
            pe = hg.pins[hg.offsets[e]:hg.offsets[e + 1]]
            ref = np.bincount(part[pe], minlength=k)
            assert np.array_equal(phi[e], ref)
            assert phi[e].sum() == len(pe)
            bits = [(int(lam[e]) >> i) & 1 for i in range(k)]
            assert bits == [int(x > 0) for x in ref]


@pytest.mark.parametrize("seed", range(4))
def test_gain_equals_objective_difference_exhaustive(oracle_mod, seed):
    # Sec. 6: g_u(V_t) is the decrease of f_{lambda-1} when u alone moves to V_t.
    # Checked for every node, every target and every partition of tiny inputs.
    rng = np.random.default_rng(100 + seed)
    n = 6
    k = 2 + seed % 2
    hg = random_hypergraph(rng, n, 7, 5, w_hi=4)
    for assign in itertools.product(range(k), repeat=n):
        part = np.array(assign, dtype=np.int32)
        f = oracle_mod.objective(hg, k, part)
        g = oracle_mod.gains(hg, k, part)
        for u in range(n):
            for t in range(k):
                if t == part[u]:
                    continue
                moved = part.copy()
                moved[u] = t
                assert g[u, t] == f - oracle_mod.objective(hg, k, moved)


def test_balance_limit_examples(oracle_mod):
    # L_max = (1 + eps) * ceil(c(V)/k) (Sec. 2) with eps = 0.03
    assert oracle_mod.balance_limit(10_000, 2, 30000) == 5150
    assert oracle_mod.balance_limit(10_001, 2, 30000) == 5151   # ceil -> 5001, 5151.03
    assert oracle_mod.balance_limit(4, 2, 30000) == 2           # 2.06 rounds down
    assert oracle_mod.balance_limit(7, 8, 0) == 1
