"""The C-ABI library builds, loads and exports every declared symbol; host-side
logic (query compaction, input validation) behaves as documented.  No GPU."""
import ctypes
import os

import numpy as np
import pytest

from paper_2005_06727_gb300 import build as build_mod
from paper_2005_06727_gb300 import wmd


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return wmd.lib()


def test_every_declared_function_is_exported(lib):
    names = wmd.declared_functions()
    assert len(names) >= 10
    raw = ctypes.CDLL(wmd.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib):
    assert b"sm_103a" in lib.wmd_version()
    assert "arch=compute_103a,code=sm_103a" in " ".join(build_mod.ARCH)


def test_compact_query_drops_zero_weights_and_keeps_order(lib):
    ids, w = wmd.compact_query([7, 2, 9, 4], [0.25, 0.0, 0.5, 0.25], 10)
    assert ids.tolist() == [7, 9, 4]
    assert w.tolist() == [0.25, 0.5, 0.25]
    ids, w = wmd.compact_query([], [], 10)
    assert ids.size == 0


@pytest.mark.parametrize("ids,w,msg", [
    ([1, 1], [0.5, 0.5], "duplicate"),
    ([1, 10], [0.5, 0.5], "outside"),
    ([-1], [1.0], "outside"),
    ([1], [-0.5], "negative"),
    ([1], [float("nan")], "not finite"),
    ([1], [float("inf")], "not finite"),
])
def test_compact_query_rejects_bad_input(lib, ids, w, msg):
    with pytest.raises(wmd.WMDError) as e:
        wmd.compact_query(ids, w, 10)
    assert e.value.status == wmd.WMD_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_compact_query_zero_weight_duplicates_are_ignored(lib):
    ids, _ = wmd.compact_query([3, 3], [0.0, 1.0], 10)
    assert ids.tolist() == [3]


def test_compact_query_too_many_words(lib):
    n = wmd.MAX_VR + 1
    with pytest.raises(wmd.WMDError) as e:
        wmd.compact_query(np.arange(n), np.full(n, 1.0 / n), 1000)
    assert e.value.status == wmd.WMD_ERR_UNSUPPORTED


def _corpus_args():
    vecs = np.ones((4, 3), np.float32)
    row_ptr = np.array([0, 1, 1, 3, 3], np.int64)
    doc_idx = np.array([0, 0, 1], np.int32)
    val = np.array([0.5, 0.5, 1.0], np.float32)
    return vecs, row_ptr, doc_idx, val, 2


@pytest.mark.parametrize("mutate,msg", [
    (lambda a: a[1].__setitem__(4, 2), "end at nnz"),
    (lambda a: a[1].__setitem__(2, 0), "decreases"),
    (lambda a: a[2].__setitem__(0, 5), "outside [0, N)"),
    (lambda a: a[2].__setitem__(2, 0), "strictly increasing"),
    (lambda a: a[3].__setitem__(1, 0.0), "> 0"),
    (lambda a: a[3].__setitem__(1, np.nan), "> 0"),
    (lambda a: a[0].__setitem__((0, 0), np.inf), "non-finite"),
])
def test_corpus_load_validates_on_host(lib, mutate, msg):
    """Malformed inputs are rejected before anything touches a GPU."""
    args = list(_corpus_args())
    mutate(args)
    with pytest.raises(wmd.WMDError) as e:
        wmd.Corpus(*args)
    assert e.value.status == wmd.WMD_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(wmd, "_lib", None)
    monkeypatch.setattr(wmd, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(wmd.WMDError):
        wmd.lib()


def test_new_entry_points_validate_on_host(lib):
    """k nearest documents, the convergence-tested query and the dense
    comparator reject bad arguments before any CUDA call (the pointers below
    are never dereferenced)."""
    fake = ctypes.c_void_p(0x1000)
    bad, unsupported, ok = wmd.WMD_ERR_INVALID_ARG, wmd.WMD_ERR_UNSUPPORTED, wmd.WMD_OK
    # wmd_topk: 0 <= k <= min(N, 1024), non-NULL pointers, N below 2^31
    assert lib.wmd_topk(fake, 10, 11, fake, fake, None) == bad
    assert lib.wmd_topk(fake, 10, -1, fake, fake, None) == bad
    assert lib.wmd_topk(fake, 5000, 1025, fake, fake, None) == bad
    assert lib.wmd_topk(None, 10, 3, fake, fake, None) == bad
    assert lib.wmd_topk(fake, 10, 3, fake, None, None) == bad
    assert lib.wmd_topk(fake, 1 << 32, 3, fake, fake, None) == unsupported
    assert lib.wmd_topk(fake, 10, 0, None, None, None) == ok          # nothing to select
    # entry points that take a corpus refuse a NULL one
    assert lib.wmd_query_device_tol(None, fake, fake, 5, 10.0, 15, 1e-3, 0, fake, 1 << 20, fake,
                                    None, None) == bad
    assert lib.wmd_query_device_topk(None, fake, fake, 5, 10.0, 15, 0, fake, 1 << 20, fake, 3,
                                     fake, fake, None) == bad
    assert lib.wmd_query_dense(None, fake, fake, 5, 10.0, 15, fake, 1 << 20, fake, None) == bad
    assert lib.wmd_dense_load_c(None, fake, 1 << 20, None) == bad
    assert lib.wmd_dense_workspace_bytes(None, 5) == 0
    assert b"corpus" in lib.wmd_last_error()


def test_options_defaults_and_host_validation(lib):
    """wmd_options_default gives the documented defaults, and options out of
    range are refused before anything touches a GPU."""
    o = wmd.options()
    assert (o.device, o.use_graphs, o.cdist_kernel, o.wait_limit_cycles) == (0, 1, 0, 0)
    assert o.autotune_cache is None
    assert (o.server.max_batch, o.server.slots, o.server.mem_budget, o.server.max_pending) == \
        (64, 2, 8 << 30, 65536)
    args = _corpus_args()
    for kw, msg in [({"cdist_kernel": 5}, "cdist kernel"), ({"wait_limit_cycles": -1}, "wait"),
                    ({"slots": 0}, "server options"), ({"slots": 17}, "server options"),
                    ({"device": -1}, "device")]:
        with pytest.raises(wmd.WMDError) as e:
            wmd.Corpus(*args, **kw)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
        assert msg in str(e.value)
    with pytest.raises(TypeError):
        wmd.options(no_such_option=1)
    # a NULL corpus is refused by the setters and getters
    assert lib.wmd_corpus_set_wait_limit(None, 5) == wmd.WMD_ERR_INVALID_ARG
    assert lib.wmd_get_loop_variant(None, 30, 0) == -1


def test_measure_fp32_peak_rejects_null_output(lib):
    """wmd_measure_fp32_peak checks its output pointer before touching CUDA."""
    assert lib.wmd_measure_fp32_peak(0, 1, None) == wmd.WMD_ERR_INVALID_ARG


def test_partition_entry_points_on_null_corpus(lib):
    assert lib.wmd_get_loop_partition(None, 30, 0) == -1
    assert lib.wmd_set_loop_partition(None, 30, 0, 100) == wmd.WMD_ERR_INVALID_ARG


def test_loop_width_classes(lib):
    """wmd_loop_width (host only): v_r rounded up to the tile widths 8, 16,
    32, 48, 64, 96, 128, 192, 256, and 0 outside [1, WMD_MAX_VR]."""
    widths = (8, 16, 32, 48, 64, 96, 128, 192, 256)
    lo = 0
    for w in widths:
        for v_r in (lo + 1, (lo + 1 + w) // 2, w):
            assert wmd.loop_width(v_r) == w, (v_r, w)
        lo = w
    assert sorted({wmd.loop_width(v) for v in range(1, 257)}) == list(widths)
    assert wmd.loop_width(0) == 0 and wmd.loop_width(-3) == 0 and wmd.loop_width(257) == 0
    assert all(wmd.loop_variant_count(v) >= 1 for v in (1, 48, 49, 96, 97, 192, 193, 256))
