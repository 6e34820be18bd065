"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs.  All arithmetic is integer, so every
comparison is exact (bit-identical arrays and objectives)."""
import numpy as np
import pytest

import synth
from tests.tiny import from_nets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_17679_gb300 import hg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_opt(seed=1, S=16, T=1000, factor=160, fp_bits=0):
    o = hg.hg_default_options()
    o.seed, o.subrounds, o.rating_max_net_size = seed, S, T
    o.contraction_limit_factor, o.fingerprint_bits = factor, fp_bits
    return o


def create(hgr, opt, device_input=False):
    stream = torch.cuda.current_stream()
    if device_input:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
        off, pins, w, c = t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w)
        h = hg.hg_create(hgr.n, hgr.m, off, pins, w, c, hg.HG_MEM_DEVICE, opt, stream)
        torch.cuda.synchronize()
        return h
    return hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w,
                        hg.HG_MEM_HOST, opt, stream)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


# ---------------------------------------------------------------- inputs

def tiny_cases():
    out = {}
    out["single_net"] = from_nets(6, [[0, 1, 2, 3, 4, 5]], [3])
    out["isolated"] = from_nets(12, [[0, 1], [1, 2], [2, 3], [5, 6, 7]], [1, 2, 3, 4])
    out["identical"] = from_nets(10, [[0, 1, 2], [2, 1, 0], [3, 4], [4, 3], [0, 1, 2], [5, 6, 7, 8]],
                                 [1, 2, 3, 4, 5, 6])
    out["heavy_node"] = from_nets(8, [[i, (i + 1) % 8] for i in range(8)], None,
                                  [40, 1, 1, 1, 1, 1, 1, 1])
    return out


def medium_cases():
    return {
        "uniform10k": synth.uniform_10k(1),
        "zipf20k": synth.zipf_1m(3, n=20_000),
        "stress": synth.large_net_stress(4, 40_000, 20_000, big_lo=300, big_hi=9000,
                                         force_first=9000),
        "weighted": synth.random_uniform(5, 5000, 8000, node_w=(1, 50), net_w=(1, 1000)),
    }


# ---------------------------------------------------------------- structure

@pytest.mark.parametrize("name", ["uniform10k", "stress"])
@pytest.mark.parametrize("device_input", [False, True])
def test_incidence_is_the_transpose(name, device_input):
    hgr = medium_cases()[name]
    h = create(hgr, make_opt(), device_input)
    try:
        off, nets = hg.hg_get_incidence(h, 0)
    finally:
        hg.hg_destroy(h)
    # independent transpose by numpy: stable argsort of the pins
    net_of_pin = np.repeat(np.arange(hgr.m, dtype=np.int32), np.diff(hgr.offsets))
    order = np.argsort(hgr.pins, kind="stable")
    ref_off = np.zeros(hgr.n + 1, np.int64)
    np.add.at(ref_off, hgr.pins.astype(np.int64) + 1, 1)
    ref_off = np.cumsum(ref_off)
    assert np.array_equal(off, ref_off)
    ref_nets = net_of_pin[order]
    for u in np.random.default_rng(0).choice(hgr.n, 500):
        a, b = off[u], off[u + 1]
        assert np.array_equal(np.sort(nets[a:b]), ref_nets[a:b])


@pytest.mark.parametrize("k", [2, 7, 64])
def test_objective_and_pin_counts(oracle_mod, k):
    hgr = medium_cases()["zipf20k"]
    h = create(hgr, make_opt())
    try:
        rng = np.random.default_rng(k)
        for _ in range(3):
            part = rng.integers(0, k, size=hgr.n).astype(np.int32)
            dpart = dev(part)
            assert hg.hg_objective(h, 0, k, dpart) == oracle_mod.objective(hgr, k, part)
            phi, lam, bw = hg.hg_pin_counts(h, 0, k, dpart)
            rphi, rlam = oracle_mod.pin_counts(hgr, k, part)
            assert np.array_equal(phi, rphi) and np.array_equal(lam, rlam)
            assert np.array_equal(bw, oracle_mod.block_weights(hgr, k, part))
    finally:
        hg.hg_destroy(h)


# ---------------------------------------------------------------- coarsening

def compare_level(h, level, ref_level):
    got = hg.hg_get_level(h, level)
    assert np.array_equal(got["offsets"], ref_level.offsets)
    assert np.array_equal(got["pins"], ref_level.pins)
    assert np.array_equal(got["net_w"], ref_level.net_w)
    assert np.array_equal(got["node_w"], ref_level.node_w)


def check_one_level(oracle_mod, hgr, k, opt, level=0):
    W = int(hgr.node_w.sum())
    ref = oracle_mod.coarsen(hgr, W, k, S=opt.subrounds, T=opt.rating_max_net_size,
                             factor=opt.contraction_limit_factor, seed=opt.seed, level=level)
    h = create(hgr, opt)
    try:
        rc, lv, n2, m2, p2 = hg.hg_coarsen_level(h, k)
        if ref is None:
            assert rc == hg.HG_STOP
            return
        assert rc == hg.HG_OK and lv == 1
        got = hg.hg_get_level(h, 0, with_map=True)
        assert np.array_equal(got["rep"], ref["rep"])
        assert np.array_equal(got["map"], ref["map"])
        assert (n2, m2, p2) == (ref["level"].n, ref["level"].m, ref["level"].p)
        compare_level(h, 1, ref["level"])
    finally:
        hg.hg_destroy(h)


@pytest.mark.parametrize("name", ["uniform10k", "zipf20k", "stress", "weighted"])
def test_coarsen_level_parity(oracle_mod, name):
    hgr = medium_cases()[name]
    k = {"uniform10k": 2, "zipf20k": 8, "stress": 64, "weighted": 4}[name]
    factor = {"uniform10k": 160, "zipf20k": 20, "stress": 4, "weighted": 40}[name]
    check_one_level(oracle_mod, hgr, k, make_opt(seed=3, factor=factor))


def hub_hypergraph(oracle_mod, seed=71, n=200_000, m_base=150_000, hub_nets=45_000, sub_seed=3):
    """Random 2 + Geom(0.3) nets plus one hub in hub_nets extra 3-pin nets with
    two random other nodes each.  The hub is the smallest id of sub-round 0
    (so it is rated before any node can join it), and its candidate bound
    D = min(W, n) >= 135,000 is above what eight shared-memory parts hold, so
    its rating runs through the global hash table split over the grid."""
    hub = next(u for u in range(n) if oracle_mod.subround_clustering(sub_seed, 0, u, 16) == 0)
    base = synth.random_uniform(seed, n, m_base)
    a = synth.uniform_ints(seed + 1, hub_nets, 0, n // 2 - 1)
    b = synth.uniform_ints(seed + 2, hub_nets, n // 2, n - 1)
    a[a == hub] = (hub + 1) % (n // 2)
    extra = np.stack([np.full(hub_nets, hub, np.int32), a, b], axis=1).reshape(-1)
    off = np.concatenate([base.offsets,
                          base.p + 3 * np.arange(1, hub_nets + 1, dtype=np.int64)]).astype(np.int32)
    pins = np.concatenate([base.pins, extra]).astype(np.int32)
    w = np.concatenate([base.net_w, np.ones(hub_nets, np.int32)])
    return hub, synth.Hypergraph(n, m_base + hub_nets, off, pins, w, base.node_w.copy(), "hub")


@pytest.mark.parametrize("k", [2, 8])
def test_coarsen_hub_uses_global_hash_split(oracle_mod, k):
    hub, hgr = hub_hypergraph(oracle_mod)
    W = int(hgr.node_w.sum())
    ref = oracle_mod.coarsen(hgr, W, k, 16, 1000, 160, 3, 0)
    assert ref["rated_in"][hub] == 0 and ref["target"][hub] >= 0
    check_one_level(oracle_mod, hgr, k, make_opt(seed=3))


@pytest.mark.parametrize("name", ["single_net", "isolated", "identical", "heavy_node"])
def test_coarsen_tiny_cases(oracle_mod, name):
    hgr = tiny_cases()[name]
    check_one_level(oracle_mod, hgr, 1, make_opt(seed=5, S=2, factor=1))


def test_coarsen_small_threshold_and_subrounds(oracle_mod):
    hgr = synth.zipf_1m(8, n=6000)
    check_one_level(oracle_mod, hgr, 2, make_opt(seed=8, S=3, T=8, factor=10))


def test_fingerprint_collisions_resolved(oracle_mod):
    # 3-bit fingerprints: almost every coarse net collides with others of its
    # group; the exact comparison rounds must still give the oracle's nets
    hgr = synth.random_uniform(9, 3000, 6000, cap=6)
    check_one_level(oracle_mod, hgr, 2, make_opt(seed=9, factor=5, fp_bits=3))


def test_hierarchy_parity(oracle_mod):
    hgr = synth.zipf_1m(11, n=30_000)
    k, factor = 8, 10
    opt = make_opt(seed=11, factor=factor)
    vc = oracle_mod.multilevel(hgr, k, seed=11, factor=factor, max_passes=0)
    h = create(hgr, opt)
    try:
        while hg.hg_coarsen_level(h, k)[0] == hg.HG_OK:
            pass
        assert hg.hg_num_levels(h) == len(vc.levels)
        for lv in range(1, len(vc.levels)):
            compare_level(h, lv, vc.levels[lv])
            got = hg.hg_get_level(h, lv - 1, with_map=True)
            assert np.array_equal(got["map"], vc.maps[lv - 1])
    finally:
        hg.hg_destroy(h)


# ---------------------------------------------------------------- refinement

def test_initial_partition_and_projection(oracle_mod):
    hgr = synth.zipf_1m(12, n=8000)
    k = 8
    h = create(hgr, make_opt(seed=12, factor=10))
    try:
        hg.hg_coarsen_level(h, k)
        n1 = hg.hg_level_info(h, 1)[0]
        cpart = torch.empty(n1, dtype=torch.int32, device="cuda")
        hg.hg_initial_partition(h, 1, k, cpart)
        lvl1 = hg.hg_get_level(h, 1)
        ref = oracle_mod.initial_partition(lvl1["node_w"], k, 12)
        assert np.array_equal(cpart.cpu().numpy(), ref)
        fpart = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        hg.hg_project(h, 1, cpart, fpart)
        mp = hg.hg_get_level(h, 0, with_map=True)["map"]
        assert np.array_equal(fpart.cpu().numpy(), oracle_mod.project(mp, ref))
    finally:
        hg.hg_destroy(h)


@pytest.mark.parametrize("k,passes,name", [(2, 5, "uniform10k"), (8, 3, "zipf20k"), (64, 2, "stress"),
                                           (4, 5, "weighted"), (3, 1, "uniform10k")])
def test_lp_parity(oracle_mod, k, passes, name):
    hgr = medium_cases()[name]
    seed = 21
    part0 = oracle_mod.initial_partition(hgr.node_w, k, seed)
    ref = oracle_mod.lp_refine(hgr, k, part0, 30000, 16, seed, 0, passes)
    h = create(hgr, make_opt(seed=seed))
    try:
        dpart = dev(part0)
        obj, moves = hg.hg_lp_refine(h, 0, k, 30000, passes, dpart)
        got = dpart.cpu().numpy()
    finally:
        hg.hg_destroy(h)
    assert moves == ref["moves"]
    assert np.array_equal(got, ref["part"])
    assert obj == ref["objective"]


@pytest.mark.parametrize("n,k,eps", [(600_000, 2, 30000), (200_000, 32, 2_000_000_000)])
def test_lp_parity_long_directions(oracle_mod, n, k, eps):
    """Sub-rounds with more candidate moves in one direction than the pair
    selection sorts in shared memory (4096 for k <= 8, 1024 for k > 16): the
    sorted sequences and weight prefixes of that direction go through global
    memory, at offsets the pair block sums from the direction counts (k <= 16)
    or at the bucket offsets (larger k).  Only blocks 0 and 1 are used at the
    start, so every candidate move is between them (a move into an empty
    block has no positive gain)."""
    hgr = synth.random_uniform(61 + k, n, n)
    part0 = synth.uniform_ints(n + k, n, 0, 1)
    seed = 7
    _, mv = oracle_mod.lp_subround(hgr, k, part0, eps, 16, seed, 0, 0, 0)
    longest = int(np.bincount(mv["src"] * k + mv["dst"], minlength=k * k).max())
    assert longest > (4096 if k <= 8 else 1024)
    ref = oracle_mod.lp_refine(hgr, k, part0, eps, 16, seed, 0, 2)
    h = create(hgr, make_opt(seed=seed))
    try:
        dpart = dev(part0)
        obj, moves = hg.hg_lp_refine(h, 0, k, eps, 2, dpart)
        got = dpart.cpu().numpy()
    finally:
        hg.hg_destroy(h)
    assert moves == ref["moves"]
    assert np.array_equal(got, ref["part"])
    assert obj == ref["objective"]


def test_lp_large_slack_and_tight_balance(oracle_mod):
    hgr = synth.random_uniform(22, 4000, 4000, node_w=(1, 9))
    for eps in (0, 1_000_000):
        part0 = oracle_mod.initial_partition(hgr.node_w, 2, 22)
        ref = oracle_mod.lp_refine(hgr, 2, part0, eps, 16, 22, 0, 4)
        h = create(hgr, make_opt(seed=22))
        try:
            dpart = dev(part0)
            obj, moves = hg.hg_lp_refine(h, 0, 2, eps, 4, dpart)
            assert np.array_equal(dpart.cpu().numpy(), ref["part"])
            assert (obj, moves) == (ref["objective"], ref["moves"])
        finally:
            hg.hg_destroy(h)


@pytest.mark.parametrize("name,k,factor", [("uniform10k", 2, 160), ("zipf20k", 8, 10)])
def test_partition_vcycle_parity(oracle_mod, name, k, factor):
    hgr = medium_cases()[name]
    seed = 31
    vc = oracle_mod.multilevel(hgr, k, 30000, S=16, T=1000, factor=factor, seed=seed, max_passes=5)
    h = create(hgr, make_opt(seed=seed, factor=factor))
    try:
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        obj = hg.hg_partition(h, k, 30000, 5, part)
        assert hg.hg_num_levels(h) == len(vc.levels)
        assert np.array_equal(part.cpu().numpy(), vc.parts[0])
        assert obj == vc.objectives[0]
    finally:
        hg.hg_destroy(h)


def test_repeated_runs_identical():
    hgr = synth.zipf_1m(41, n=50_000)
    results = []
    for _ in range(2):
        h = create(hgr, make_opt(seed=41, factor=10))
        try:
            part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
            obj = hg.hg_partition(h, 8, 30000, 5, part)
            results.append((obj, part.cpu().numpy(), hg.hg_get_level(h, 1)["pins"]))
        finally:
            hg.hg_destroy(h)
    assert results[0][0] == results[1][0]
    assert np.array_equal(results[0][1], results[1][1])
    assert np.array_equal(results[0][2], results[1][2])


# ------------------------------------------------- gain recalculation (Sec. 6.3)

def random_moves(rng, part, k, count):
    nodes = rng.permutation(len(part))[:count].astype(np.int32)
    targets = np.array([(int(part[u]) + 1 + int(rng.integers(0, k - 1))) % k for u in nodes],
                       np.int32)
    return nodes, targets


@pytest.mark.parametrize("name,k,frac,level", [("zipf20k", 8, 0.1, 0), ("zipf20k", 8, 1.0, 0),
                                               ("zipf20k", 4, 0.3, 1), ("stress", 64, 0.2, 0),
                                               ("weighted", 2, 0.5, 0)])
def test_gain_recalculation_parity(oracle_mod, name, k, frac, level):
    hgr = medium_cases()[name]
    h = create(hgr, make_opt(factor=10))
    try:
        if level > 0:
            hg.hg_coarsen_level(h, k)
            got = hg.hg_get_level(h, level)
            lvl = oracle_mod.Level(len(got["node_w"]), len(got["net_w"]), got["offsets"],
                                   got["pins"], got["net_w"], got["node_w"])
        else:
            lvl = hgr
        rng = np.random.default_rng(k * 100 + level)
        part = rng.integers(0, k, size=lvl.n).astype(np.int32)
        nodes, targets = random_moves(rng, part, k, max(1, int(frac * lvl.n)))
        gains = torch.zeros(len(nodes), dtype=torch.int64, device="cuda")
        hg.hg_recalculate_gains(h, level, k, dev(part), dev(nodes), dev(targets), gains)
        want = oracle_mod.recalculate_gains(lvl, k, part, nodes, targets)
        assert np.array_equal(gains.cpu().numpy(), want)
        moved = part.copy()
        moved[nodes] = targets
        assert int(want.sum()) == (oracle_mod.objective(lvl, k, part)
                                   - oracle_mod.objective(lvl, k, moved))
    finally:
        hg.hg_destroy(h)


def test_gain_recalculation_rejects_bad_sequences():
    hgr = medium_cases()["uniform10k"]
    h = create(hgr, make_opt())
    try:
        part = dev(np.zeros(hgr.n, np.int32))
        gains = torch.zeros(2, dtype=torch.int64, device="cuda")
        for nodes, targets in (([0, 0], [1, 1]), ([1, 2], [0, 1]), ([1, 2], [1, 5])):
            with pytest.raises(hg.HgError) as ei:
                hg.hg_recalculate_gains(h, 0, 4, part, dev(nodes), dev(targets), gains)
            assert ei.value.status == hg.HG_ERR_INVALID
        # the handle stays usable
        hg.hg_recalculate_gains(h, 0, 4, part, dev([1, 2]), dev([1, 3]), gains)
    finally:
        hg.hg_destroy(h)


# ------------------------------------------------------ gain table (Sec. 6.2)

@pytest.mark.parametrize("name,k,frac", [("zipf20k", 8, 0.2), ("stress", 64, 0.1),
                                         ("weighted", 3, 1.0), ("uniform10k", 2, 0.5)])
def test_gain_table_build_and_moves(oracle_mod, name, k, frac):
    hgr = medium_cases()[name]
    h = create(hgr, make_opt())
    try:
        rng = np.random.default_rng(k + 5)
        part = rng.integers(0, k, size=hgr.n).astype(np.int32)
        dpart = dev(part)
        b = torch.zeros(hgr.n, dtype=torch.int64, device="cuda")
        p = torch.zeros((hgr.n, k), dtype=torch.int64, device="cuda")
        hg.hg_gain_table(h, 0, k, dpart, b, p)
        wb, wp = oracle_mod.gain_table(hgr, k, part)
        assert np.array_equal(b.cpu().numpy(), wb) and np.array_equal(p.cpu().numpy(), wp)
        # a set of moves applied at once with the update rules, then the moved
        # nodes' benefits recomputed: the table of the new partition
        nodes, targets = random_moves(rng, part, k, max(1, int(frac * hgr.n)))
        hg.hg_gain_table_move(h, 0, k, dpart, dev(nodes), dev(targets), b, p)
        moved = part.copy()
        moved[nodes] = targets
        assert np.array_equal(dpart.cpu().numpy(), moved)
        wb2, wp2 = oracle_mod.gain_table(hgr, k, moved)
        assert np.array_equal(b.cpu().numpy(), wb2)
        assert np.array_equal(p.cpu().numpy(), wp2)
    finally:
        hg.hg_destroy(h)


def test_gain_table_and_objective_reject_bad_block_ids():
    hgr = medium_cases()["uniform10k"]
    h = create(hgr, make_opt())
    try:
        part = np.zeros(hgr.n, np.int32)
        part[7] = 4  # k = 4: out of range
        dpart = dev(part)
        b = torch.zeros(hgr.n, dtype=torch.int64, device="cuda")
        p = torch.zeros((hgr.n, 4), dtype=torch.int64, device="cuda")
        for call in (lambda: hg.hg_gain_table(h, 0, 4, dpart, b, p),
                     lambda: hg.hg_objective(h, 0, 4, dpart),
                     lambda: hg.hg_pin_counts(h, 0, 4, dpart)):
            with pytest.raises(hg.HgError) as ei:
                call()
            assert ei.value.status == hg.HG_ERR_INVALID
        good = dev(np.zeros(hgr.n, np.int32))
        before = good.clone()
        with pytest.raises(hg.HgError):  # node 3 twice: nothing changes
            hg.hg_gain_table_move(h, 0, 4, good, dev([3, 3]), dev([1, 2]), b, p)
        assert torch.equal(good, before)
        assert hg.hg_objective(h, 0, 4, good) == 0
    finally:
        hg.hg_destroy(h)


def test_device_input_with_repeated_pins_rejected():
    """hg_create on device arrays rejects a node repeated inside a net, for
    small nets (warp match), mid-size nets (shared hash set) and nets above
    1024 pins (per-block node bitmap); the valid versions are accepted."""
    stream = torch.cuda.current_stream()
    n = 5000
    for size in (5, 300, 3000):
        pins = np.arange(size, dtype=np.int32)
        off = np.array([0, size, size + 2], np.int32)
        good = np.concatenate([pins, [0, 1]]).astype(np.int32)
        bad = good.copy()
        bad[size - 1] = bad[size // 2]  # a repeat inside net 0
        for arr, ok in ((good, True), (bad, False)):
            args = (dev(off), dev(arr), dev(np.ones(2, np.int32)), dev(np.ones(n, np.int32)))
            if ok:
                h = hg.hg_create(n, 2, *args, hg.HG_MEM_DEVICE, make_opt(), stream)
                hg.hg_destroy(h)
            else:
                with pytest.raises(hg.HgError) as ei:
                    hg.hg_create(n, 2, *args, hg.HG_MEM_DEVICE, make_opt(), stream)
                assert ei.value.status == hg.HG_ERR_INVALID


@pytest.mark.parametrize("repeat", [False, True])
def test_repeated_pin_in_a_big_net_of_a_huge_node_set(repeat):
    """With more than 14 million nodes the per-block node bitmaps of the
    big-net repeat check would exceed their budget, so the check falls back
    to per-block hash sets: a node repeated inside a 3000-pin net is still
    rejected, and the net without the repeat is accepted."""
    n = 15_000_000
    size = 3000
    pins = np.arange(0, n, n // size, dtype=np.int32)[:size].copy()
    if repeat:
        pins[-1] = pins[10]
    off = np.array([0, size, size + 2], np.int32)
    pins = np.concatenate([pins, [1, 2]]).astype(np.int32)
    stream = torch.cuda.current_stream()
    args = (dev(off), dev(pins), dev(np.ones(2, np.int32)), None)
    if not repeat:
        h = hg.hg_create(n, 2, *args, hg.HG_MEM_DEVICE, make_opt(), stream)
        hg.hg_destroy(h)
        return
    with pytest.raises(hg.HgError) as ei:
        hg.hg_create(n, 2, *args, hg.HG_MEM_DEVICE, make_opt(), stream)
    assert ei.value.status == hg.HG_ERR_INVALID


@pytest.mark.parametrize("size", ["mid", "large"])
@pytest.mark.parametrize("fault", ["out_of_range", "repeat_small", "repeat_big", "bad_weight",
                                   "decreasing_offsets", "none"])
def test_large_host_input_pins_checked_on_the_device(fault, size):
    """Host inputs above 65,536 pins have their pins checked on the device
    (above 4,194,304 pins their offsets and weights too): a pin out of range,
    a node repeated inside a net (small or large net), a weight of zero or an
    empty net is rejected with HG_ERR_INVALID and the next create succeeds."""
    hgr = (synth.random_uniform(61, 30_000, 40_000) if size == "mid"
           else synth.random_uniform(62, 600_000, 1_200_000))
    assert hgr.p > 1 << 16
    assert (hgr.p > 1 << 22) == (size == "large")
    off = np.concatenate([hgr.offsets, [hgr.p + 2000]]).astype(np.int32)
    big = np.arange(0, 4000, 2, dtype=np.int32)  # a 2000-pin net
    pins = np.concatenate([hgr.pins, big]).astype(np.int32)
    w = np.concatenate([hgr.net_w, [1]]).astype(np.int32)
    if fault == "bad_weight":
        w[hgr.m // 3] = 0
    elif fault == "decreasing_offsets":
        off[hgr.m // 2] = off[hgr.m // 2 + 1]  # an empty net
    elif fault == "out_of_range":
        pins[hgr.p // 2] = hgr.n
    elif fault == "repeat_small":
        e = 7
        b = hgr.offsets[e]
        pins[b + 1] = pins[b]
    elif fault == "repeat_big":
        pins[-1] = pins[-1000]
    stream = torch.cuda.current_stream()
    if fault == "none":
        h = hg.hg_create(hgr.n, hgr.m + 1, off, pins, w, hgr.node_w, hg.HG_MEM_HOST, make_opt(),
                         stream)
        hg.hg_destroy(h)
        return
    with pytest.raises(hg.HgError) as ei:
        hg.hg_create(hgr.n, hgr.m + 1, off, pins, w, hgr.node_w, hg.HG_MEM_HOST, make_opt(), stream)
    assert ei.value.status == hg.HG_ERR_INVALID
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     make_opt(), stream)
    hg.hg_destroy(h)
