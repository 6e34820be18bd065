"""Full-size inputs on the GPU (the n = m = 1e6 Zipf hypergraph and the 4M-node
large-net hypergraph), in the configuration bench.py times
(S = 16, T = 1000, f = 160).  The oracle cannot run these sizes in a test,
so the results are checked by
  * sampled outputs: the target of sampled nodes that joined a cluster in the
    first sub-round of level 0, recomputed on the host from the rating of
    Sec. 4.1 (every cluster is a singleton at that point, so r(u, C) sums the
    floored Q20 terms of the rated nets shared with C);
  * properties that hold at any size: conservation of node weight, the
    cluster weight limit, the coarse id map, canonical coarse nets (sorted
    distinct pins, no single-pin net, no two identical nets) and their summed
    weights (Sec. 4.2);
  * the whole V-cycle: objective equal to the oracle's objective of the
    returned partition, balance, bit-identical repeat runs (Sec. 11)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_17679_gb300 import hg  # noqa: E402

S, T, FACTOR, SEED = 16, 1000, 160, 1
MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def mix64_np(x):
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def subrounds(n, level):
    u = np.arange(n, dtype=np.uint64)
    key = np.uint64(SEED) ^ (np.uint64(level) << np.uint64(32)) ^ u
    return (mix64_np(key) % np.uint64(S)).astype(np.int64)


def incidence(off, pins, n):
    sizes = np.diff(off)
    net_of = np.repeat(np.arange(len(sizes), dtype=np.int64), sizes)
    order = np.argsort(pins, kind="stable")
    ioff = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(pins, minlength=n), out=ioff[1:])
    return ioff, net_of[order]


def expected_target(u, off, pins, w, c, ioff, inets, c_max, sr0):
    """argmax over admissible C of r(u, C), ties to the smaller C, at the start
    of sub-round 0 of a level; -1 without an admissible candidate."""
    es = inets[ioff[u]:ioff[u + 1]]
    sz = off[es + 1] - off[es]
    keep = (sz >= 2) & (sz <= T)
    es, sz = es[keep], sz[keep]
    if len(es) == 0:
        return -1
    terms = (w[es].astype(np.int64) << 20) // (sz - 1)
    vs = np.concatenate([pins[off[e]:off[e + 1]] for e in es]).astype(np.int64)
    tv = np.repeat(terms, sz)
    ok = (vs != u) & ~sr0[vs] & (c[vs].astype(np.int64) + int(c[u]) <= c_max)
    vs, tv = vs[ok], tv[ok]
    if len(vs) == 0:
        return -1
    cand, inv = np.unique(vs, return_inverse=True)
    r = np.zeros(len(cand), np.int64)
    np.add.at(r, inv, tv)
    return int(cand[np.flatnonzero(r == r.max())[0]])


def test_vectorised_subround_hash_matches_the_oracle(oracle_mod):
    rng = np.random.default_rng(5)
    for level in (0, 3):
        us = rng.integers(0, 4_000_000, size=200)
        sr = subrounds(4_000_000, level)[us]
        assert [oracle_mod.subround_clustering(SEED, level, int(u), S) for u in us] == list(sr)


def check_level0(hgr, k, samples=300):
    stream = torch.cuda.current_stream()
    opt = hg.hg_default_options()
    opt.seed, opt.subrounds, opt.rating_max_net_size, opt.contraction_limit_factor = SEED, S, T, FACTOR
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST, opt,
                     stream)
    try:
        rc = hg.hg_coarsen_level(h, k)[0]
        assert rc == hg.HG_OK
        L0 = hg.hg_get_level(h, 0, with_map=True)
        L1 = hg.hg_get_level(h, 1)
    finally:
        hg.hg_destroy(h)
    off = np.asarray(hgr.offsets, np.int64)
    pins = np.asarray(hgr.pins, np.int64)
    w = np.asarray(hgr.net_w, np.int64)
    c = np.asarray(hgr.node_w, np.int64)
    n = hgr.n
    W = int(c.sum())
    c_max = -(-W // (FACTOR * k))
    rep, mp = L0["rep"].astype(np.int64), L0["map"].astype(np.int64)

    # coarse ids: rank of the representative
    reps = np.unique(rep)
    assert np.all(rep[reps] == reps)
    assert np.array_equal(mp, np.searchsorted(reps, rep))
    n1 = len(reps)
    assert len(L1["node_w"]) == n1
    # node weights conserved; clusters of two or more nodes within c_max
    cw = np.bincount(mp, weights=c, minlength=n1).astype(np.int64)
    assert np.array_equal(cw, L1["node_w"].astype(np.int64))
    members = np.bincount(mp, minlength=n1)
    assert np.all(cw[members >= 2] <= c_max)

    # coarse nets: sorted distinct pins, at least two, no two identical, and
    # the total weight of the nets that keep two or more coarse pins
    off1 = L1["offsets"].astype(np.int64)
    p1 = L1["pins"].astype(np.int64)
    sz1 = np.diff(off1)
    assert np.all(sz1 >= 2) and np.all((p1 >= 0) & (p1 < n1))
    net1 = np.repeat(np.arange(len(sz1)), sz1)
    same_net = net1[1:] == net1[:-1]
    assert np.all(p1[1:][same_net] > p1[:-1][same_net])
    keys = set()
    for e in range(len(sz1)):
        keys.add(p1[off1[e]:off1[e + 1]].tobytes())
    assert len(keys) == len(sz1)
    sz = np.diff(off)
    net_of = np.repeat(np.arange(hgr.m), sz)
    cp = mp[pins]
    order = np.lexsort((cp, net_of))
    cs, ns = cp[order], net_of[order]
    first = np.ones(len(cs), bool)
    first[1:] = (cs[1:] != cs[:-1]) | (ns[1:] != ns[:-1])
    distinct = np.bincount(ns[first], minlength=hgr.m)
    assert int(L1["net_w"].astype(np.int64).sum()) == int(w[distinct >= 2].sum())

    # sampled targets of the nodes that joined a cluster in sub-round 0
    sr = subrounds(n, 0)
    sr0 = sr == 0
    moved = np.flatnonzero(sr0 & (rep != np.arange(n)))
    assert len(moved) > 0
    rng = np.random.default_rng(17)
    pick = rng.choice(moved, size=min(samples, len(moved)), replace=False)
    ioff, inets = incidence(off, pins, n)
    for u in pick:
        assert rep[u] == expected_target(int(u), off, pins, w, c, ioff, inets, c_max, sr0), int(u)
    return n1


def check_vcycle(hgr, k, oracle_mod):
    stream = torch.cuda.current_stream()
    opt = hg.hg_default_options()
    opt.seed = SEED
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    args = (d(hgr.offsets), d(hgr.pins), d(hgr.net_w), d(hgr.node_w))
    parts, objs = [], []
    for _ in range(2):
        h = hg.hg_create(hgr.n, hgr.m, *args, hg.HG_MEM_DEVICE, opt, stream)
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        try:
            objs.append(hg.hg_partition(h, k, 30000, 5, part))
        finally:
            hg.hg_destroy(h)
        parts.append(part.cpu().numpy())
    assert objs[0] == objs[1] and np.array_equal(parts[0], parts[1])
    part = parts[0]
    assert part.min() >= 0 and part.max() < k
    assert objs[0] == oracle_mod.objective(hgr, k, part)
    bw = np.bincount(part, weights=np.asarray(hgr.node_w, np.int64), minlength=k)
    W = int(np.asarray(hgr.node_w, np.int64).sum())
    assert bw.max() <= oracle_mod.balance_limit(W, k, 30000)


def test_zipf1m_level0_full_size():
    n1 = check_level0(synth.zipf_1m(SEED), 8)
    assert n1 < 1_000_000


def test_zipf1m_vcycle_full_size(oracle_mod):
    check_vcycle(synth.zipf_1m(SEED), 8, oracle_mod)


def test_large_net_4m_level0_full_size():
    check_level0(synth.large_net_4m(SEED), 64, samples=200)


def test_large_net_4m_vcycle_full_size(oracle_mod):
    check_vcycle(synth.large_net_4m(SEED), 64, oracle_mod)
