"""hg_objective_noalloc (objective and block weights with no handle and no
device allocation), for callers that cannot allocate device memory, against
the handle-based entry points hg_objective and hg_pin_counts and against the
CPU oracle on the same inputs.  All values are integers, so the tolerance is
zero.  A warm call must leave the device's free memory, PyTorch's allocator
and the device's default memory pool exactly as they were.  The file name
keeps it last in collection, so the entry point is also exercised after every
other test has run in the same process."""
import ctypes
import gc

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


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _default_pool_used(rt):
    """Bytes in use in the current device's default stream-ordered pool, or None."""
    if rt is None:
        return None
    dev = ctypes.c_int(0)
    pool = ctypes.c_void_p()
    used = ctypes.c_uint64(0)
    if rt.cudaGetDevice(ctypes.byref(dev)) != 0:
        return None
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) != 0:
        return None
    attr_used_mem_current = 5  # cudaMemPoolAttrUsedMemCurrent
    if rt.cudaMemPoolGetAttribute(pool, attr_used_mem_current, ctypes.byref(used)) != 0:
        return None
    return used.value


def _memory_state(rt):
    gc.collect()  # settle frees of unreachable tensors before reading the counters
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), _default_pool_used(rt)


def _assert_nothing_allocated(before, after):
    """Free device memory, PyTorch's reserved memory and the default pool's
    used bytes unchanged, and PyTorch's allocated bytes not grown."""
    assert after[0] == before[0], ("free device memory", before, after)
    assert after[1] <= before[1], ("torch allocated", before, after)
    assert after[2] == before[2], ("torch reserved", before, after)
    assert after[3] == before[3], ("default pool used", before, after)


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
def test_matches_the_handle_entry_points_twice_in_a_row(hg, oracle_mod, name):
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
    hpart = part.cpu().numpy()
    assert want_obj == oracle_mod.objective(hgr, k, hpart)
    assert np.array_equal(want_bw, oracle_mod.block_weights(hgr, k, hpart))
    off, pins, w, c = (_dev(a) for a in (hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w))
    rt = _cudart()
    for i in range(2):
        before = _memory_state(rt)
        obj, bw = hg.hg_objective_noalloc(hgr.n, hgr.m, len(hgr.pins), off, pins, w, c, k, part,
                                          stream)
        after = _memory_state(rt)
        assert obj == want_obj
        assert np.array_equal(bw, want_bw)
        if i == 1:  # a warm call: no device memory taken from any allocator
            _assert_nothing_allocated(before, after)
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


@pytest.mark.gpu
@pytest.mark.parametrize("fault", ["offset_beyond_p", "pin_out_of_range"])
def test_bad_csr_on_the_device_is_reported_and_the_next_call_is_clean(hg, oracle_mod, fault):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hgr = synth.uniform_10k(2)
    k = 8
    stream = torch.cuda.current_stream()
    p = len(hgr.pins)
    off = np.array(hgr.offsets, np.int32)
    pins = np.array(hgr.pins, np.int32)
    if fault == "offset_beyond_p":
        off[-1] = p + 1  # the last net would end past the pins
    else:
        pins[p // 3] = hgr.n  # a pin naming a node that does not exist
    good = np.random.default_rng(5).integers(0, k, size=hgr.n).astype(np.int32)
    dgood = _dev(good)
    with pytest.raises(hg.HgError) as ei:
        hg.hg_objective_noalloc(hgr.n, hgr.m, p, _dev(off), _dev(pins), None, None, k, dgood,
                                stream)
    assert ei.value.status == hg.HG_ERR_INVALID
    want = oracle_mod.objective(
        type(hgr)(hgr.n, hgr.m, hgr.offsets, hgr.pins, np.ones(hgr.m, np.int32),
                  np.ones(hgr.n, np.int32)), k, good)
    want_bw = np.bincount(good, minlength=k).astype(np.int64)
    for _ in range(2):
        obj, bw = hg.hg_objective_noalloc(hgr.n, hgr.m, p, _dev(hgr.offsets), _dev(hgr.pins), None,
                                          None, k, dgood, stream)
        assert obj == want and np.array_equal(bw, want_bw)
