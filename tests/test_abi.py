"""The C-ABI library loads without a GPU, exports every entry point that
include/hg.h declares, and rejects malformed host inputs before touching the
device (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_17679_gb300 import build, hg
    build.build()
    return hg.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hg_create", "hg_coarsen_level", "hg_lp_refine", "hg_objective", "hg_project",
                     "hg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2303_17679_gb300 import hg
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(hg.exported_symbols()) == declared_functions()


def test_strerror_and_version(lib):
    from paper_2303_17679_gb300 import hg
    assert hg.hg_strerror(hg.HG_ERR_INVALID) == "invalid argument"
    assert "sm_103a" in hg.hg_version()


def _create(lib, n, m, off, pins, w=None, c=None):
    from paper_2303_17679_gb300 import hg
    h = ctypes.c_void_p()
    arr = lambda a: None if a is None else np.ascontiguousarray(a, np.int32)
    off, pins, w, c = arr(off), arr(pins), arr(w), arr(c)
    p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    rc = lib.hg_create(n, m, p(off), p(pins), p(w), p(c), hg.HG_MEM_HOST, None, None,
                       ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("case", [
    dict(n=3, m=1, off=[0, 0], pins=[]),                       # empty net
    dict(n=3, m=1, off=[0, 2], pins=[0, 3]),                   # pin out of range
    dict(n=3, m=1, off=[0, 3], pins=[0, 1, 1]),                # repeated pin
    dict(n=3, m=1, off=[1, 3], pins=[0, 1, 2]),                # offsets not starting at 0
    dict(n=3, m=2, off=[0, 2, 1], pins=[0, 1, 2]),             # decreasing offsets
    dict(n=3, m=1, off=[0, 2], pins=[0, 1], w=[0]),            # zero net weight
    dict(n=3, m=1, off=[0, 2], pins=[0, 1], c=[1, -1, 1]),     # negative node weight
    dict(n=2, m=1, off=[0, 2], pins=[0, 1], c=[2 ** 30, 2 ** 30]),  # total weight >= 2^31
    dict(n=0, m=0, off=[0], pins=[]),                          # no nodes
])
def test_malformed_host_input_rejected(lib, case):
    from paper_2303_17679_gb300 import hg
    rc, h = _create(lib, case["n"], case["m"], case["off"], case["pins"], case.get("w"),
                    case.get("c"))
    assert rc == hg.HG_ERR_INVALID
    assert not h.value


@pytest.mark.parametrize("fault", ["empty_net", "zero_weight", "heavy_nodes"])
def test_mid_sized_host_input_checked_before_any_device_work(lib, fault):
    """Host inputs of 65,536 to 4,194,304 pins have their offsets and weights
    checked on the caller's thread before anything touches the device, so a
    bad one is rejected on a host without a GPU."""
    from paper_2303_17679_gb300 import hg
    rng = np.random.default_rng(5)
    n, m, size = 50_000, 30_000, 4
    off = np.arange(0, size * m + 1, size, dtype=np.int32)
    pins = np.concatenate([rng.choice(n, size, replace=False) for _ in range(m)]).astype(np.int32)
    assert 1 << 16 < off[-1] <= 1 << 22
    w = np.ones(m, np.int32)
    c = np.ones(n, np.int32)
    if fault == "empty_net":
        off[m // 2] = off[m // 2 + 1]
    elif fault == "zero_weight":
        w[m // 3] = 0
    else:
        c[:] = 2 ** 20  # total node weight above 2^31
    rc, h = _create(lib, n, m, off, pins, w, c)
    assert rc == hg.HG_ERR_INVALID
    assert not h.value


def test_bad_options_rejected(lib):
    from paper_2303_17679_gb300 import hg
    o = hg.hg_default_options()
    assert (o.seed, o.subrounds, o.rating_max_net_size, o.contraction_limit_factor) == (1, 16, 1000, 160)
    for field, value in (("subrounds", 0), ("subrounds", 257), ("rating_max_net_size", 1),
                         ("contraction_limit_factor", 0), ("fingerprint_bits", 65)):
        bad = hg.hg_default_options()
        setattr(bad, field, value)
        h = ctypes.c_void_p()
        off = np.array([0, 2], np.int32)
        pins = np.array([0, 1], np.int32)
        rc = lib.hg_create(2, 1, ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(pins.ctypes.data),
                           None, None, hg.HG_MEM_HOST, ctypes.byref(bad), None, ctypes.byref(h))
        assert rc == hg.HG_ERR_INVALID


def test_launch_mapping_options_bounded(lib):
    """The tunable cutoffs default to 0 (built-in mapping) and are rejected
    above the capacity of the kernels' tables."""
    from paper_2303_17679_gb300 import hg
    o = hg.hg_default_options()
    assert all(getattr(o, f) == 0 for f in hg.hg_options.TUNABLE)
    for field, value in (("rate_warp_max_d", 257), ("rate_pair_max_d", 1025),
                         ("rate_quad_max_d", 2049), ("rate_block_max_d", 4097),
                         ("lp_block_min_deg", -1), ("rate_warp_max_d", -1)):
        bad = hg.hg_default_options()
        setattr(bad, field, value)
        h = ctypes.c_void_p()
        off = np.array([0, 2], np.int32)
        pins = np.array([0, 1], np.int32)
        rc = lib.hg_create(2, 1, ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(pins.ctypes.data),
                           None, None, hg.HG_MEM_HOST, ctypes.byref(bad), None, ctypes.byref(h))
        assert rc == hg.HG_ERR_INVALID, (field, value)


def test_null_handle_calls_are_rejected(lib):
    from paper_2303_17679_gb300 import hg
    assert lib.hg_destroy(None) == hg.HG_OK
    assert lib.hg_lp_refine(None, 0, 2, 0, 1, None, None, None) == hg.HG_ERR_INVALID
    assert lib.hg_objective(None, 0, 2, None, None) == hg.HG_ERR_INVALID
