"""Results do not depend on the launch mapping: the rating team cutoffs and
the label-propagation warp/block cutoff (the autotuner's knobs) are set to
extremes that move every node to another kernel, and the hierarchy, the
partition and the objective stay bit-identical."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_17679_gb300 import autotune, hg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


MAPPINGS = [
    {},  # built-in defaults
    {"rate_warp_max_d": 1, "rate_pair_max_d": 1, "rate_quad_max_d": 1, "rate_block_max_d": 1,
     "lp_block_min_deg": 1},  # every rated node split over the grid, every LP node a block
    {"rate_warp_max_d": 32, "rate_pair_max_d": 64, "rate_quad_max_d": 128,
     "rate_block_max_d": 256, "lp_block_min_deg": 1 << 20},  # small teams, LP warps only
]


def run(hgr, k, mapping):
    opt = autotune.apply(hg.hg_default_options(), mapping)
    opt.contraction_limit_factor = 10
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     opt, stream)
    try:
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        obj = hg.hg_partition(h, k, 30000, 5, part)
        levels = [hg.hg_get_level(h, lv)["pins"] for lv in range(hg.hg_num_levels(h))]
        return obj, part.cpu().numpy(), levels
    finally:
        hg.hg_destroy(h)


@pytest.mark.parametrize("name", ["zipf", "stress", "weighted"])
def test_mapping_does_not_change_results(name):
    hgr, k = {
        "zipf": (synth.zipf_1m(3, n=30_000), 8),
        "stress": (synth.large_net_stress(4, 40_000, 20_000, big_lo=300, big_hi=9000), 16),
        "weighted": (synth.random_uniform(5, 5000, 8000, node_w=(1, 50), net_w=(1, 1000)), 4),
    }[name]
    ref = run(hgr, k, MAPPINGS[0])
    for mp in MAPPINGS[1:]:
        got = run(hgr, k, mp)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1])
        assert len(got[2]) == len(ref[2])
        assert all(np.array_equal(a, b) for a, b in zip(got[2], ref[2]))
