"""Pins for the oracle's exact gains of a move sequence (Sec. 6.3): each
gain equals the objective difference of performing that move after the
earlier ones, with the objective recomputed from scratch (a definition
independent of the pin-count bookkeeping), and the gains telescope to the
total objective change.  Bad sequences are rejected."""
import numpy as np
import pytest

from tests.tiny import from_nets


def random_instance(rng, n, m, max_size):
    nets = []
    for _ in range(m):
        sz = int(rng.integers(2, max_size + 1))
        nets.append(sorted(rng.choice(n, size=min(sz, n), replace=False).tolist()))
    w = rng.integers(1, 9, size=m).tolist()
    return from_nets(n, nets, w)


@pytest.mark.parametrize("seed", range(6))
def test_gains_equal_sequential_objective_differences(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 6))
    hg = random_instance(rng, 12, 15, 6)
    part = rng.integers(0, k, size=hg.n).astype(np.int32)
    nodes = rng.permutation(hg.n)[: int(rng.integers(1, hg.n + 1))].astype(np.int32)
    targets = np.array([(int(part[u]) + 1 + int(rng.integers(0, k - 1))) % k for u in nodes],
                       np.int32)
    g = oracle_mod.recalculate_gains(hg, k, part, nodes, targets)
    cur = part.copy()
    f_prev = oracle_mod.objective(hg, k, cur)
    f0 = f_prev
    for i, (u, t) in enumerate(zip(nodes, targets)):
        cur[u] = t
        f = oracle_mod.objective(hg, k, cur)
        assert g[i] == f_prev - f
        f_prev = f
    assert int(g.sum()) == f0 - f_prev


def test_hand_worked_sequence(oracle_mod):
    hg = from_nets(4, [[0, 1, 2, 3]], [5])
    part = np.array([0, 0, 1, 1], np.int32)
    g = oracle_mod.recalculate_gains(hg, 3, part, [0, 1, 2], [1, 2, 0])
    assert g.tolist() == [0, 0, -5]
    # the same moves in another order: 1->2 first splits the net into three
    # blocks (-5), then 0->1 empties block 0 (+5), then 2->0 reopens it (-5)
    g2 = oracle_mod.recalculate_gains(hg, 3, part, [1, 0, 2], [2, 1, 0])
    assert g2.tolist() == [-5, 5, -5]


def test_bad_sequences_rejected(oracle_mod):
    hg = from_nets(4, [[0, 1, 2, 3]], [5])
    part = np.array([0, 0, 1, 1], np.int32)
    for nodes, targets in (([0, 0], [1, 2]), ([0], [0]), ([0], [3]), ([5], [1])):
        with pytest.raises(ValueError):
            oracle_mod.recalculate_gains(hg, 3, part, nodes, targets)
