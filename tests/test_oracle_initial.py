"""Pins for the seeded initial partition (a stand-in for Sec. 5's portfolio)
and for the multilevel loop of Algorithm 1 composed from the oracle."""
import numpy as np

import synth


def test_initial_partition_unit_weights_round_robin(oracle_mod):
    # unit weights: the lightest-block rule deals nodes round-robin along the
    # order of (mix64(seed ^ 2^63 ^ u), u)
    n, k, seed = 1000, 7, 42
    keys = np.array([oracle_mod.mix64(seed ^ (1 << 63) ^ u) for u in range(n)], dtype=np.uint64)
    order = np.lexsort((np.arange(n), keys))
    expect = np.empty(n, np.int32)
    expect[order] = np.arange(n) % k
    part = oracle_mod.initial_partition(np.ones(n, np.int32), k, seed)
    assert np.array_equal(part, expect)


def test_initial_partition_weighted_spread(oracle_mod):
    rng = np.random.default_rng(5)
    c = rng.integers(1, 40, size=5000).astype(np.int32)
    for k in (2, 8, 64):
        part = oracle_mod.initial_partition(c, k, 9)
        bw = np.bincount(part, weights=c, minlength=k)
        # greedy to the lightest block keeps the spread below the heaviest node
        assert bw.max() - bw.min() <= c.max()


def test_multilevel_projection_preserves_objective(oracle_mod):
    hg = synth.zipf_1m(2, n=4000)
    k = 4
    vc = oracle_mod.multilevel(hg, k, seed=2, factor=20)
    L = len(vc.levels) - 1
    assert L >= 2
    W = int(hg.node_w.sum())
    for lv in range(L):
        # the refined coarse partition, projected, has the same objective
        proj = oracle_mod.project(vc.maps[lv], vc.parts[lv + 1])
        assert oracle_mod.objective(vc.levels[lv], k, proj) == vc.objectives[lv + 1]
        # and refinement on the finer level does not make it worse here
        assert vc.objectives[lv] <= vc.objectives[lv + 1]
        assert int(vc.levels[lv + 1].node_w.sum()) == W
    lmax = oracle_mod.balance_limit(W, k, 30000)
    assert np.all(oracle_mod.block_weights(hg, k, vc.parts[0]) <= lmax)
