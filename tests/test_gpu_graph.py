"""The graph path (Sec. 10): levels whose nets all have two pins keep one
adjacency array; the rating reads neighbours directly and label propagation
takes g(u, t) = w(u, V_t) - w(u, V_Pi(u)) from the neighbours' blocks without
pin counts.  Graphs are hypergraphs, so the oracle is the same: every level,
map, partition, objective and move count of the V-cycle must equal the
oracle's and the hypergraph path's (hg_options.graph_path = 1) exactly."""
import numpy as np
import pytest

import synth
from tests.tiny import from_nets
from tests.vcycle_records import compare_records, gpu_records, oracle_records

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_17679_gb300 import hg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def opt_for(seed, factor, graph_path=0):
    o = hg.hg_default_options()
    o.seed, o.contraction_limit_factor, o.graph_path = seed, factor, graph_path
    return o


def hub_graph(seed=5, n=40_000, m=80_000, hub_deg=9000):
    """A uniform random graph plus a hub joined to hub_deg random nodes, so
    the hub's rating goes to the split classes."""
    base = synth.graph_uniform(seed, n, m)
    rng = np.random.default_rng(seed)
    others = rng.choice(np.arange(1, n), size=hub_deg, replace=False).astype(np.int32)
    extra = np.stack([np.zeros(hub_deg, np.int32), others], axis=1).reshape(-1)
    off = np.concatenate([base.offsets, base.p + 2 * np.arange(1, hub_deg + 1)]).astype(np.int32)
    pins = np.concatenate([base.pins, extra]).astype(np.int32)
    w = np.concatenate([base.net_w, rng.integers(1, 5, size=hub_deg).astype(np.int32)])
    return synth.Hypergraph(n, m + hub_deg, off, pins, w, base.node_w.copy(), "hub_graph")


def cases():
    return {
        "uniform_k2": (synth.graph_uniform(1, 20_000, 50_000), 2, 40),
        "preferential_k8": (synth.graph_preferential(2, 60_000, 200_000), 8, 20),
        "weighted_k32": (synth.graph_preferential(3, 30_000, 120_000, 1, 100), 32, 4),
        "hub_k4": (hub_graph(), 4, 40),
    }


@pytest.mark.parametrize("name", list(cases()))
def test_graph_vcycle_matches_oracle_and_hypergraph_path(oracle_mod, name):
    hgr, k, factor = cases()[name]
    seed = 17
    vc = oracle_mod.multilevel(hgr, k, 30000, S=16, T=1000, factor=factor, seed=seed,
                               max_passes=5)
    want = oracle_records(vc)
    got, initial = gpu_records(hg, torch, hgr, k, 30000, 5, opt_for(seed, factor))
    assert all(r["graph"] for r in got if r["m"] > 0), "graph levels not detected"
    assert initial == vc.initial_objective
    compare_records(got, want)
    general, initial_h = gpu_records(hg, torch, hgr, k, 30000, 5, opt_for(seed, factor, 1))
    assert not any(r["graph"] for r in general)
    assert initial_h == initial
    compare_records(general, want)


def test_non_graph_levels_use_the_hypergraph_path():
    g = from_nets(6, [[0, 1], [1, 2], [2, 3, 4], [4, 5]])
    stream = torch.cuda.current_stream()
    h = hg.hg_create(g.n, g.m, g.offsets, g.pins, g.net_w, g.node_w, hg.HG_MEM_HOST, None, stream)
    try:
        assert not hg.hg_level_is_graph(h, 0)
    finally:
        hg.hg_destroy(h)
    g2 = from_nets(4, [[0, 1], [1, 2], [2, 3]])
    h = hg.hg_create(g2.n, g2.m, g2.offsets, g2.pins, g2.net_w, g2.node_w, hg.HG_MEM_HOST, None,
                     stream)
    try:
        assert hg.hg_level_is_graph(h, 0)
    finally:
        hg.hg_destroy(h)


@pytest.mark.parametrize("k", [2, 8, 64])
def test_graph_lp_and_objective_from_a_random_partition(oracle_mod, k):
    hgr = synth.graph_preferential(9, 20_000, 70_000, 1, 10)
    rng = np.random.default_rng(k)
    part0 = rng.integers(0, k, size=hgr.n).astype(np.int32)
    stream = torch.cuda.current_stream()
    o = opt_for(23, 160)
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w,
                     hg.HG_MEM_HOST, o, stream)
    try:
        assert hg.hg_level_is_graph(h, 0)
        d = torch.from_numpy(part0.copy()).cuda()
        assert hg.hg_objective(h, 0, k, d) == oracle_mod.objective(hgr, k, part0)
        obj, moves = hg.hg_lp_refine(h, 0, k, 30000, 3, d)
        ref = oracle_mod.lp_refine(hgr, k, part0, 30000, S=16, seed=23, level=0, max_passes=3)
        assert np.array_equal(d.cpu().numpy(), ref["part"])
        assert obj == ref["objective"] and moves == ref["moves"]
    finally:
        hg.hg_destroy(h)


@pytest.mark.parametrize("k", [2, 16, 64])
def test_graph_gain_table_matches_oracle_and_moves(oracle_mod, k):
    """The graph form of the gain table (from w(u, V_i)) equals the oracle's
    table of Sec. 6.2; a concurrent move set then gives the new partition's
    table (the moves run through the hypergraph update rules)."""
    hgr = synth.graph_preferential(31, 15_000, 50_000, 1, 20)
    rng = np.random.default_rng(k + 1)
    part0 = rng.integers(0, k, size=hgr.n).astype(np.int32)
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w,
                     hg.HG_MEM_HOST, None, stream)
    try:
        assert hg.hg_level_is_graph(h, 0)
        d = torch.from_numpy(part0.copy()).cuda()
        b = torch.zeros(hgr.n, dtype=torch.int64, device="cuda")
        p = torch.zeros((hgr.n, k), dtype=torch.int64, device="cuda")
        hg.hg_gain_table(h, 0, k, d, b, p)
        rb, rp = oracle_mod.gain_table(hgr, k, part0)
        assert np.array_equal(b.cpu().numpy(), rb) and np.array_equal(p.cpu().numpy(), rp)
        nodes = rng.permutation(hgr.n)[: hgr.n // 5].astype(np.int32)
        targets = ((part0[nodes] + 1 + rng.integers(0, k - 1, size=len(nodes))) % k).astype(np.int32)
        hg.hg_gain_table_move(h, 0, k, d, torch.from_numpy(nodes).cuda(),
                              torch.from_numpy(targets).cuda(), b, p)
        part1 = part0.copy()
        part1[nodes] = targets
        assert np.array_equal(d.cpu().numpy(), part1)
        rb, rp = oracle_mod.gain_table(hgr, k, part1)
        assert np.array_equal(b.cpu().numpy(), rb) and np.array_equal(p.cpu().numpy(), rp)
    finally:
        hg.hg_destroy(h)
