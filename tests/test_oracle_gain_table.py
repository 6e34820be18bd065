"""Pins for the oracle's gain table (Sec. 6.2): b(u) - p(u, V_t) equals the
gain g_u(V_t) of Sec. 6 (itself pinned by exhaustive objective differences)
for every node and every other block; p(u, Pi[u]) = 0 (u is a pin of its
own block in every incident net); a node alone in all its nets has
b(u) = w(I(u)); the table is unchanged by renaming blocks consistently."""
import numpy as np
import pytest

from tests.tiny import from_nets


def random_instance(rng, n, m, max_size):
    nets = []
    for _ in range(m):
        sz = int(rng.integers(2, max_size + 1))
        nets.append(sorted(rng.choice(n, size=min(sz, n), replace=False).tolist()))
    return from_nets(n, nets, rng.integers(1, 9, size=m).tolist())


@pytest.mark.parametrize("seed", range(5))
def test_table_matches_gains(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 7))
    hg = random_instance(rng, 30, 40, 8)
    part = rng.integers(0, k, size=hg.n).astype(np.int32)
    b, p = oracle_mod.gain_table(hg, k, part)
    g = oracle_mod.gains(hg, k, part)
    for u in range(hg.n):
        assert p[u, part[u]] == 0
        for t in range(k):
            if t != part[u]:
                assert b[u] - p[u, t] == g[u, t]
    # consistent renaming of the blocks permutes the penalty columns only
    perm = rng.permutation(k)
    b2, p2 = oracle_mod.gain_table(hg, k, perm[part].astype(np.int32))
    assert np.array_equal(b2, b)
    assert np.array_equal(p2[:, perm], p)


def test_isolated_blocks_closed_form(oracle_mod):
    hg = from_nets(4, [[0, 1], [0, 2], [0, 3]], [2, 3, 4])
    part = np.array([0, 1, 1, 1], np.int32)
    b, p = oracle_mod.gain_table(hg, 3, part)
    assert b[0] == 9                       # node 0 alone in block 0 in all three nets
    assert p[0].tolist() == [0, 0, 9]      # block 2 holds no pin of any net
    assert b[1] == 2 and p[1].tolist() == [0, 0, 2]  # node 1 alone in block 1 in net {0, 1}
