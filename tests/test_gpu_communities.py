"""Community detection on the GPU (Sec. 4 "Community-Aware Coarsening",
Sec. 11 "Deterministic Louvain Method") against the oracle: the community of
every node must be identical, and so must every level, map, partition,
objective and move count of the community-aware V-cycle.  All arithmetic is
integer (Q20 edge weights, 128-bit modularity comparisons), so comparisons
are exact."""
import numpy as np
import pytest

import synth
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


def cases():
    return {
        "zipf20k": synth.zipf_1m(3, n=20_000),
        "uniform10k": synth.uniform_10k(2),
        "weighted": synth.random_uniform(5, 5000, 8000, node_w=(1, 50), net_w=(1, 1000)),
        # nets of 300..9000 pins: net vertices above the shared-table degree
        "stress": synth.large_net_stress(4, 40_000, 20_000, big_lo=300, big_hi=9000,
                                         force_first=9000),
        "graph": synth.graph_preferential(6, 30_000, 90_000),
    }


def make_opt(seed, S=16, factor=160, communities=0):
    o = hg.hg_default_options()
    o.seed, o.subrounds, o.contraction_limit_factor = seed, S, factor
    o.community_detection = communities
    return o


@pytest.mark.parametrize("name", list(cases()))
@pytest.mark.parametrize("S,seed", [(16, 1), (5, 9)])
def test_communities_match_oracle(oracle_mod, name, S, seed):
    hgr = cases()[name]
    want, levels, moves = oracle_mod.communities(hgr, S=S, seed=seed)
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     make_opt(seed, S), stream)
    try:
        count = hg.hg_detect_communities(h)
        got = hg.hg_get_communities(h, 0)
        st = hg.hg_get_stats(h)
    finally:
        hg.hg_destroy(h)
    assert np.array_equal(got, want), int((got != want).sum())
    assert count == len(set(want.tolist()))
    assert st["louvain_levels"] == levels and st["louvain_moves"] == moves


@pytest.mark.parametrize("name,k,factor", [("zipf20k", 8, 20), ("stress", 16, 8),
                                           ("graph", 4, 40)])
def test_community_aware_vcycle_matches_oracle(oracle_mod, name, k, factor):
    hgr = cases()[name]
    seed = 13
    vc = oracle_mod.multilevel(hgr, k, 30000, S=16, T=1000, factor=factor, seed=seed,
                               max_passes=5, communities_first=True)
    opt = make_opt(seed, factor=factor, communities=1)
    # the V-cycle through hg_partition (communities first) ...
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     opt, stream)
    try:
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        obj = hg.hg_partition(h, k, 30000, 5, part)
        assert np.array_equal(part.cpu().numpy(), vc.parts[0])
        assert obj == vc.objectives[0]
        assert np.array_equal(hg.hg_get_communities(h, 0), vc.communities)
        top = hg.hg_num_levels(h) - 1
        coarse_comm = hg.hg_get_communities(h, top)
        mp = np.arange(hgr.n)
        for lv in range(top):
            mp = hg.hg_get_level(h, lv, with_map=True)["map"][mp]
        assert np.array_equal(coarse_comm[mp], vc.communities)
    finally:
        hg.hg_destroy(h)
    # ... and level by level (every CSR, map and partition)
    o2 = make_opt(seed, factor=factor)
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     o2, stream)
    try:
        hg.hg_detect_communities(h)
        while hg.hg_coarsen_level(h, k)[0] == hg.HG_OK:
            pass
        assert hg.hg_num_levels(h) == len(vc.levels)
        for lv in range(1, len(vc.levels)):
            got = hg.hg_get_level(h, lv)
            for key in ("offsets", "pins", "net_w", "node_w"):
                assert np.array_equal(got[key], getattr(vc.levels[lv], key)), (lv, key)
            assert np.array_equal(hg.hg_get_level(h, lv - 1, with_map=True)["map"],
                                  vc.maps[lv - 1])
    finally:
        hg.hg_destroy(h)


def test_detection_after_coarsening_is_rejected():
    hgr = synth.uniform_10k(3)
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, None, None, hg.HG_MEM_HOST,
                     make_opt(1, factor=10), stream)
    try:
        with pytest.raises(hg.HgError) as ei:
            hg.hg_get_communities(h, 0)
        assert ei.value.status == hg.HG_ERR_STATE
        hg.hg_coarsen_level(h, 2)
        with pytest.raises(hg.HgError) as ei:
            hg.hg_detect_communities(h)
        assert ei.value.status == hg.HG_ERR_STATE
    finally:
        hg.hg_destroy(h)
