"""hg_objective_noalloc (objective and block weights with no handle and no
device allocation) against the handle-based entry points hg_objective and
hg_pin_counts on the same inputs.  All values are integers, so the tolerance
is zero.  The file name keeps it last in collection, so the entry point is
also exercised after every other test has run in the same process."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_17679_gb300 import hg as mod
    return mod


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def test_sizes_beyond_the_scratch_are_rejected_on_the_host(hg):
    lib = hg.load()
    off = np.zeros(1, np.int32)
    part = np.zeros(4, np.int32)
    obj = hg.ctypes.c_int64(-7)
    for n, m, p, k, want in [(4, 0, 0, 65, hg.HG_ERR_UNSUPPORTED), (4, 0, 0, 0, hg.HG_ERR_INVALID),
                             (0, 0, 0, 2, hg.HG_ERR_INVALID), (4, -1, 0, 2, hg.HG_ERR_INVALID),
                             (4, 0, -1, 2, hg.HG_ERR_INVALID), (4, 0, 2**31, 2, hg.HG_ERR_INVALID)]:
        rc = lib.hg_objective_noalloc(n, m, p, hg._ptr(off), None, None, None, k, hg._ptr(part),
                                      None, hg.ctypes.byref(obj), None)
        assert rc == want, (n, m, p, k, rc)
    assert obj.value == -7  # nothing written on rejection


def _cases():
    return {
        "zipf20k_k8": (synth.zipf_1m(3, n=20_000), 8),
        "weighted_k64": (synth.random_uniform(5, 5000, 8000, node_w=(1, 50), net_w=(1, 1000)), 64),
        "zipf200k_k2": (synth.zipf_1m(7, n=200_000), 2),
    }


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(_cases()))
def test_matches_the_handle_entry_points_twice_in_a_row(hg, name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hgr, k = _cases()[name]
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     None, stream)
    try:
        rng = np.random.default_rng(11)
        part = _dev(rng.integers(0, k, size=hgr.n))
        want_obj = hg.hg_objective(h, 0, k, part)
        _, _, want_bw = hg.hg_pin_counts(h, 0, k, part)
    finally:
        hg.hg_destroy(h)
    off, pins, w, c = (_dev(a) for a in (hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w))
    for _ in range(2):
        obj, bw = hg.hg_objective_noalloc(hgr.n, hgr.m, len(hgr.pins), off, pins, w, c, k, part,
                                          stream)
        assert obj == want_obj
        assert np.array_equal(bw, want_bw)
    # unit weights (NULL arrays) against the same partition with unit weights
    ones = np.ones_like
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, ones(hgr.net_w), ones(hgr.node_w),
                     hg.HG_MEM_HOST, None, stream)
    try:
        want1 = hg.hg_objective(h, 0, k, part)
        _, _, want1_bw = hg.hg_pin_counts(h, 0, k, part)
    finally:
        hg.hg_destroy(h)
    obj1, bw1 = hg.hg_objective_noalloc(hgr.n, hgr.m, len(hgr.pins), off, pins, None, None, k, part,
                                        stream)
    assert obj1 == want1 and np.array_equal(bw1, want1_bw)


@pytest.mark.gpu
def test_bad_block_id_is_reported_and_the_next_call_is_clean(hg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hgr = synth.uniform_10k(1)
    k = 4
    stream = torch.cuda.current_stream()
    off, pins = _dev(hgr.offsets), _dev(hgr.pins)
    good = np.random.default_rng(3).integers(0, k, size=hgr.n).astype(np.int32)
    bad = good.copy()
    bad[hgr.n // 2] = k  # one block id out of range
    with pytest.raises(hg.HgError) as ei:
        hg.hg_objective_noalloc(hgr.n, hgr.m, len(hgr.pins), off, pins, None, None, k, _dev(bad),
                                stream)
    assert ei.value.status == hg.HG_ERR_INVALID
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, None, None, hg.HG_MEM_HOST, None, stream)
    try:
        dgood = _dev(good)
        want = hg.hg_objective(h, 0, k, dgood)
        _, _, want_bw = hg.hg_pin_counts(h, 0, k, dgood)
    finally:
        hg.hg_destroy(h)
    for _ in range(2):
        obj, bw = hg.hg_objective_noalloc(hgr.n, hgr.m, len(hgr.pins), off, pins, None, None, k,
                                          dgood, stream)
        assert obj == want and np.array_equal(bw, want_bw)
