"""Pins for the oracle's contraction (Sec. 4.2) and projection (Algorithm 1).

Checks: a hand-worked example, conservation laws, preservation of the
objective under projection, the identity clustering, canonical order, and a
brute-force frozenset construction of the contracted net set on small inputs.
"""
import numpy as np
import pytest

from tests.tiny import from_nets, nets_of, random_hypergraph


def random_rep(rng, n, n_clusters):
    heads = np.sort(rng.choice(n, size=n_clusters, replace=False))
    rep = heads[rng.integers(0, n_clusters, size=n)].astype(np.int32)
    rep[heads] = heads
    return rep


def test_hand_worked_identical_nets(oracle_mod):
    # nets {0,1,2} and {0,1,3}; clustering 3 into 2's cluster; net {2,3} collapses
    hg = from_nets(5, [[0, 1, 2], [0, 1, 3], [2, 3], [3, 4]], [1, 1, 4, 3], [1, 2, 3, 4, 5])
    rep = np.array([0, 1, 2, 2, 4], np.int32)
    lv, mp = oracle_mod.contract(hg, rep)
    assert lv.n == 4
    assert mp.tolist() == [0, 1, 2, 2, 3]
    assert lv.node_w.tolist() == [1, 2, 7, 5]
    # {0,1,2} and {0,1,3} become the same coarse net {0,1,2} of weight 1 + 1;
    # {2,3} becomes the single pin {2} and is removed; {3,4} becomes {2,3}
    assert nets_of(lv) == [[0, 1, 2], [2, 3]]
    assert lv.net_w.tolist() == [2, 3]


def brute_force_contract(hg, rep):
    reps = sorted(set(int(r) for r in rep))
    cid = {r: i for i, r in enumerate(reps)}
    groups = {}
    order = []
    for e, pins in enumerate(nets_of(hg)):
        s = frozenset(cid[int(rep[v])] for v in pins)
        if len(s) < 2:
            continue
        if s not in groups:
            groups[s] = 0
            order.append(s)
        groups[s] += int(hg.net_w[e])
    return [sorted(s) for s in order], [groups[s] for s in order], len(reps)


@pytest.mark.parametrize("seed", range(6))
def test_contract_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = 40
    hg = random_hypergraph(rng, n, 60, 6, w_hi=7, c_hi=4)
    rep = random_rep(rng, n, int(rng.integers(5, 30)))
    lv, mp = oracle_mod.contract(hg, rep)
    nets, weights, n2 = brute_force_contract(hg, rep)
    assert lv.n == n2
    assert nets_of(lv) == nets
    assert lv.net_w.tolist() == weights


@pytest.mark.parametrize("seed", range(4))
def test_contract_conservation_and_objective(oracle_mod, seed):
    rng = np.random.default_rng(20 + seed)
    n = 200
    hg = random_hypergraph(rng, n, 300, 9, w_hi=9, c_hi=9)
    rep = random_rep(rng, n, 60)
    lv, mp = oracle_mod.contract(hg, rep)
    # total node weight is conserved
    assert lv.node_w.sum() == hg.node_w.sum()
    # net weight: everything except nets that collapse to one pin
    collapsed = sum(int(hg.net_w[e]) for e, pins in enumerate(nets_of(hg))
                    if len({int(mp[v]) for v in pins}) < 2)
    assert lv.net_w.sum() == hg.net_w.sum() - collapsed
    # pins strictly ascending within every coarse net, no single-pin nets
    for pins in nets_of(lv):
        assert len(pins) >= 2 and all(a < b for a, b in zip(pins, pins[1:]))
    # the objective of a coarse partition equals that of its projection
    for k in (2, 5):
        for _ in range(5):
            cpart = rng.integers(0, k, size=lv.n).astype(np.int32)
            fpart = oracle_mod.project(mp, cpart)
            assert np.array_equal(fpart, cpart[mp])
            assert oracle_mod.objective(lv, k, cpart) == oracle_mod.objective(hg, k, fpart)


def test_identity_clustering(oracle_mod):
    rng = np.random.default_rng(7)
    n = 30
    base = random_hypergraph(rng, n, 40, 5, w_hi=3)
    nets = nets_of(base)
    # add duplicates (in another pin order) and single-pin nets
    extra = [list(reversed(nets[3])), list(nets[3]), [5], list(reversed(nets[10]))]
    hg = from_nets(n, nets + extra, list(base.net_w) + [2, 1, 9, 4])
    lv, mp = oracle_mod.contract(hg, np.arange(n, dtype=np.int32))
    assert mp.tolist() == list(range(n))
    assert lv.n == n
    seen = {}
    order = []
    for e, pins in enumerate(nets_of(hg)):
        s = tuple(sorted(pins))
        if len(s) < 2:
            continue
        if s not in seen:
            seen[s] = 0
            order.append(s)
        seen[s] += int(hg.net_w[e])
    assert [tuple(x) for x in nets_of(lv)] == order
    assert lv.net_w.tolist() == [seen[s] for s in order]


def test_invalid_rep_rejected(oracle_mod):
    hg = from_nets(3, [[0, 1, 2]])
    with pytest.raises(ValueError):
        oracle_mod.contract(hg, np.array([1, 2, 2], np.int32))  # rep[0]=1 is not a representative
