"""Pins for the oracle's deterministic clustering (Sec. 4.1 rating, contraction
limit and c_max; Sec. 11 "Deterministic Clustering for Coarsening").

The specific clustering is the oracle's rule (the paper prints no example
with values), so the pins are: a closed form on perfect matchings, the rating
choice against exact rational arithmetic on the replayed state of every
sub-round (including exact ties), and replayed invariants of the sub-round
approval rule (admissible targets, (c asc, id asc) prefixes that are maximal
under c_max, joins only in a node's own sub-round, the n/2.5 stop rule and
the level stop rules).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from tests.tiny import from_nets, nets_of, random_hypergraph


def cmax_of(W, k, factor):
    return -(-W // (factor * k))


class Replay:
    """Reconstructs the state at the start of every sub-round from the
    oracle's trace (rep, target, rated_in) so the rules can be re-checked."""

    def __init__(self, oracle_mod, hg, r, S, seed, level):
        n = hg.n
        self.n, self.S = n, S
        self.c = hg.node_w.astype(np.int64)
        self.rep, self.target, self.rated = r["rep"], r["target"], r["rated_in"]
        self.sr = np.array([oracle_mod.subround_clustering(seed, level, u, S) for u in range(n)])
        self.joined_at = np.where(self.rep != np.arange(n), self.rated, -1)
        self.first_member = np.full(n, S, dtype=np.int64)
        for u in range(n):
            if self.rep[u] != u:
                self.first_member[self.rep[u]] = min(self.first_member[self.rep[u]], self.joined_at[u])

    def rep_at(self, s):
        """rep at the start of sub-round s"""
        out = np.arange(self.n)
        j = (self.joined_at >= 0) & (self.joined_at < s)
        out[j] = self.rep[j]
        return out

    def cw_start(self, C, s):
        rep_s = self.rep_at(s)
        return int(self.c[rep_s == C].sum())

    def unclustered_at(self, C, s):
        joined_before = self.rep[C] != C and self.joined_at[C] < s
        return (not joined_before) and self.first_member[C] >= s

    def clusters_at(self, s):
        return self.n - int(((self.joined_at >= 0) & (self.joined_at < s)).sum())


def replay_checks(oracle_mod, hg, r, W, k, S, T, factor, seed, level):
    R = Replay(oracle_mod, hg, r, S, seed, level)
    n, c, rep, target, rated, sr = R.n, R.c, R.rep, R.target, R.rated, R.sr
    cmax = cmax_of(W, k, factor)
    assert np.all(rep[rep] == rep)
    for u in range(n):
        if rated[u] >= 0:
            assert rated[u] == sr[u]
        if rep[u] != u:
            assert rated[u] >= 0 and target[u] == rep[u]
    # admissible targets
    for u in np.flatnonzero(target >= 0):
        s, C = rated[u], target[u]
        assert C != u
        assert not (R.unclustered_at(C, s) and sr[C] == s)
        assert R.cw_start(C, s) + c[u] <= cmax
    # approval groups: (c asc, id asc) prefix, maximal under c_max
    contested = 0
    for s in range(S):
        for C in np.unique(target[(rated == s) & (target >= 0)]):
            members = np.flatnonzero((rated == s) & (target == C))
            order = sorted(members.tolist(), key=lambda x: (c[x], x))
            acc = [rep[x] == C for x in order]
            na = sum(acc)
            assert acc == [True] * na + [False] * (len(order) - na)
            total = R.cw_start(C, s) + sum(int(c[x]) for x in order[:na])
            assert total <= cmax
            if na < len(order):
                contested += 1
                assert total + c[order[na]] > cmax
    # the n/2.5 rule: no node is rated in a sub-round that starts with 5*clusters <= 2n
    boundary = False
    for s in range(S):
        clusters = R.clusters_at(s)
        boundary |= 5 * clusters == 2 * n
        if 5 * clusters <= 2 * n:
            assert not np.any(rated >= s)
        else:
            for u in np.flatnonzero(sr == s):
                if R.unclustered_at(u, s):
                    assert rated[u] == s
    # final cluster weights
    cw = np.zeros(n, np.int64)
    np.add.at(cw, rep, c)
    sizes = np.bincount(rep, minlength=n)
    assert np.all((cw <= cmax) | (sizes <= 1) | (rep != np.arange(n)))
    return dict(contested=contested, boundary=boundary)


def exact_ratings(R, hg, u, s, T, cmax):
    """r(u, C) of Sec. 4.1 in exact rationals on the state at the start of s,
    over the admissible clusters C; each net counts once per cluster."""
    rep_s = R.rep_at(s)
    out = {}
    deg = 0
    for e, pins in enumerate(nets_of(hg)):
        if u not in pins:
            continue
        deg += 1
        size = len(pins)
        if size < 2 or size > T:
            continue
        for C in {int(rep_s[v]) for v in pins}:
            if C == u or (R.unclustered_at(C, s) and R.sr[C] == s):
                continue
            if R.cw_start(C, s) + R.c[u] > cmax:
                continue
            out[C] = out.get(C, Fraction(0)) + Fraction(int(hg.net_w[e]), size - 1)
    return out, deg


def test_perfect_matching_closed_form(oracle_mod):
    q, S, seed = 300, 4, 11
    n = 2 * q
    hg = from_nets(n, [[2 * i, 2 * i + 1] for i in range(q)])
    r = oracle_mod.coarsen(hg, n, 2, S=S, T=1000, factor=1, seed=seed, level=0)
    sr = [oracle_mod.subround_clustering(seed, 0, u, S) for u in range(n)]
    same = 0
    for i in range(q):
        a, b = 2 * i, 2 * i + 1
        if sr[a] == sr[b]:
            # the partner is an unclustered node of the same sub-round: no candidate
            same += 1
            assert r["rep"][a] == a and r["rep"][b] == b
            assert r["target"][a] == -1 and r["target"][b] == -1
        else:
            first, second = (a, b) if sr[a] < sr[b] else (b, a)
            assert r["rep"][first] == second and r["rep"][second] == second
    assert r["level"].n == q + same
    assert r["level"].m == same
    assert r["level"].node_w.sum() == n


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_clustering_invariants_random(oracle_mod, seed):
    hg = synth.random_uniform(seed, 1500, 1500, node_w=(1, 6), net_w=(1, 5))
    W = int(hg.node_w.sum())
    k, S, T, factor = 2, 6, 12, 100   # c_max around 27: many approval groups are contested
    r = oracle_mod.coarsen(hg, W, k, S=S, T=T, factor=factor, seed=seed, level=seed)
    st = replay_checks(oracle_mod, hg, r, W, k, S, T, factor, seed, seed)
    assert st["contested"] > 0
    assert r["level"].n < hg.n


def test_clustering_invariants_heavy_tailed(oracle_mod):
    hg = synth.zipf_1m(5, n=3000)
    W = int(hg.node_w.sum())
    k, S, T, factor = 2, 8, 200, 2
    r = oracle_mod.coarsen(hg, W, k, S=S, T=T, factor=factor, seed=5, level=0)
    replay_checks(oracle_mod, hg, r, W, k, S, T, factor, 5, 0)


@pytest.mark.parametrize("seed", [4, 5, 6, 7])
def test_rating_against_exact_rationals(oracle_mod, seed):
    # every rated node, in every sub-round, on the replayed cluster state: the
    # chosen cluster's exact rating is within the Q20 flooring bound
    # (deg(u) * 2^-20) of the exact maximum, and equal to it when the maximum
    # is separated from the runner-up by more than twice that bound
    rng = np.random.default_rng(seed)
    n, S, T, k, factor = 70, 4, 6, 2, 4
    hg = random_hypergraph(rng, n, 110, 9, w_hi=13, c_hi=3)
    W = int(hg.node_w.sum())
    cmax = cmax_of(W, k, factor)
    r = oracle_mod.coarsen(hg, W, k, S=S, T=T, factor=factor, seed=seed, level=0)
    R = Replay(oracle_mod, hg, r, S, seed, 0)
    eps = Fraction(1, 2 ** 20)
    checked = later = 0
    for u in np.flatnonzero(r["rated_in"] >= 0):
        s = int(r["rated_in"][u])
        ratings, deg = exact_ratings(R, hg, int(u), s, T, cmax)
        t = int(r["target"][u])
        if not ratings:
            assert t == -1
            continue
        assert t in ratings
        best = max(ratings.values())
        bound = deg * eps
        assert ratings[t] >= best - bound
        ranked = sorted(ratings.values(), reverse=True)
        if len(ranked) == 1 or ranked[0] - ranked[1] > 2 * bound:
            assert ratings[t] == best
        checked += 1
        later += s > 0
    assert checked > 10 and later > 5


def test_rating_counts_a_net_once_per_cluster(oracle_mod):
    # nets whose pins already share a cluster: with exact power-of-two
    # denominators (|e| - 1 in {1, 2, 4, 8}) the Q20 value is exact, so the
    # chosen cluster must be an exact maximiser and, among exact ties, the
    # smallest id
    hits = 0
    for seed in range(30):
        rng = np.random.default_rng(1000 + seed)
        n = 40
        nets = []
        for _ in range(70):
            size = int(rng.choice([2, 3, 5, 9]))
            nets.append(sorted(rng.choice(n, size=size, replace=False).tolist()))
        hg = from_nets(n, nets, rng.integers(1, 3, size=len(nets)))
        W = n
        S, T, k, factor = 3, 16, 2, 2
        cmax = cmax_of(W, k, factor)
        r = oracle_mod.coarsen(hg, W, k, S=S, T=T, factor=factor, seed=seed, level=0)
        R = Replay(oracle_mod, hg, r, S, seed, 0)
        for u in np.flatnonzero(r["rated_in"] > 0):
            s = int(r["rated_in"][u])
            ratings, _ = exact_ratings(R, hg, int(u), s, T, cmax)
            t = int(r["target"][u])
            if not ratings:
                assert t == -1
                continue
            best = max(ratings.values())
            assert t == min(C for C, x in ratings.items() if x == best)
            rep_s = R.rep_at(s)
            hits += any(len({int(rep_s[v]) for v in e}) < len(e) for e in nets if u in e)
    assert hits > 0


def test_stop_rule_boundary_scan(oracle_mod):
    # many tiny instances; the replay asserts the 5 * clusters <= 2n rule in
    # every sub-round, and some instance must sit exactly on the boundary
    boundary = 0
    for seed in range(120):
        rng = np.random.default_rng(seed)
        n = 10 + int(rng.integers(0, 3)) * 5
        hg = random_hypergraph(rng, n, 2 * n, 4)
        S = 3
        r = oracle_mod.coarsen(hg, n, 1, S=S, T=1000, factor=1, seed=seed, level=0)
        st = replay_checks(oracle_mod, hg, r, n, 1, S, 1000, 1, seed, 0)
        boundary += st["boundary"]
    assert boundary > 0


def test_heavy_node_stays_alone(oracle_mod):
    n = 400
    nets = [[i, (i + 1) % n] for i in range(n)] + [[0, 5, 9, 13]]
    c = np.ones(n, np.int32)
    c[0] = 50
    hg = from_nets(n, nets, None, c)
    W = int(c.sum())
    k, factor = 2, 20  # c_max = ceil(449 / 40) = 12 < 50
    r = oracle_mod.coarsen(hg, W, k, S=4, T=1000, factor=factor, seed=3, level=0)
    assert r["rep"][0] == 0
    assert not np.any((r["rep"] == 0) & (np.arange(n) != 0))
    replay_checks(oracle_mod, hg, r, W, k, 4, 1000, factor, 3, 0)


def test_cluster_weight_cap_rounds_up(oracle_mod):
    # c_max = ceil(W / (f k)): W = 9, f k = 2 gives 5, so a pair of weights 2
    # and 3 may merge (floor would give 4 and forbid it)
    hg = from_nets(3, [[0, 1]], None, [2, 3, 4])
    seed = next(x for x in range(100)
                if oracle_mod.subround_clustering(x, 0, 0, 2) != oracle_mod.subround_clustering(x, 0, 1, 2))
    r = oracle_mod.coarsen(hg, 9, 1, S=2, T=1000, factor=2, seed=seed, level=0)
    assert r["level"].n == 2 and sorted(r["level"].node_w.tolist()) == [4, 5]


def test_level_stop_rules(oracle_mod):
    hg = synth.random_uniform(9, 320, 300)
    W = int(hg.node_w.sum())
    # n <= factor * k: no level is built
    assert oracle_mod.coarsen(hg, W, 2, factor=160) is None
    assert oracle_mod.coarsen(hg, W, 2, factor=159) is not None
    # no nets: nothing can cluster, the level is a copy and coarsening ends
    empty = from_nets(50, [])
    r = oracle_mod.coarsen(empty, 50, 2, factor=1)
    assert r["level"].n == 50 and r["level"].m == 0 and r["stop_after"]
