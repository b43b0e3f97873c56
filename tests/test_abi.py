"""The C-ABI library loads, exports every declared symbol, and its host-side
argument checks work without a GPU (no compute call is made here)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bt():
    from paper_2604_21117_gb300 import build_lib
    build_lib.build()
    from paper_2604_21117_gb300 import btree
    return btree


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bt_[a-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(bt):
    declared = _declared_functions()
    assert declared, "no declarations found"
    lib = ctypes.CDLL(bt.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert declared == set(bt.EXPORTED)


def test_status_strings(bt):
    for code in range(9):
        assert bt.bt_status_str(code)
    assert bt.bt_status_str(0) == "ok"


def test_build_rejects_bad_arguments_before_touching_the_gpu(bt):
    k = np.array([1, 2, 3], np.uint64)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_build(k, k, 12, stream=0)
    assert e.value.code == "BT_ERR_FANOUT"
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_build(np.array([1, 3, 2], np.uint64), k, 16, stream=0)
    assert e.value.code == "BT_ERR_UNSORTED"
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_build(np.array([1, 3, 3], np.uint64), k, 16, stream=0)
    assert e.value.code == "BT_ERR_DUPLICATE"
    with pytest.raises(ValueError):
        bt.bt_build(np.array([1, 2], np.int64), np.array([1, 2], np.int64), 16, stream=0)


def test_build_checks_32_byte_key_order_bytewise(bt):
    """32-byte keys are ordered by their bytes from the first on: 0x01 0x00..
    sorts after 0x00 0xff.. although its last byte is smaller."""
    a = np.zeros((2, 32), np.uint8)
    a[0, 0], a[0, 31] = 1, 0
    a[1, 0], a[1, 31] = 0, 255
    v = np.arange(2, dtype=np.uint64)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_build(a, v, 16, stream=0)
    assert e.value.code == "BT_ERR_UNSORTED"
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_build(np.stack([a[1], a[1]]), v, 16, stream=0)
    assert e.value.code == "BT_ERR_DUPLICATE"
    h = bt.bt_build(np.zeros((0, 32), np.uint8), np.zeros(0, np.uint64), 16, stream=0)
    info = bt.bt_tree_info(h)
    assert info.key_bytes == 32 and info.height == 0 and info.device_bytes == 0
    bt.bt_free(h)
    with pytest.raises(ValueError):
        bt.bt_build(np.zeros((3, 16), np.uint8), np.zeros(3, np.uint64), 16, stream=0)


def test_empty_tree_needs_no_device_memory(bt):
    h = bt.bt_build(np.empty(0, np.uint64), np.empty(0, np.uint64), 32, stream=0)
    info = bt.bt_tree_info(h)
    assert info.height == 0 and info.n == 0 and info.device_bytes == 0
    # nq = 0 is a no-op that succeeds without a device
    bt.bt_search_batch(h, 0, 0, 0, 0, 0, 0, stream=0)
    bt.bt_free(h)


def test_workspace_size_is_monotone_and_aligned(bt):
    h = bt.bt_build(np.empty(0, np.uint32), np.empty(0, np.uint32), 16, stream=0)
    prev = 0
    for nq in (1, 31, 32, 1000, 4096, 4097, 1 << 20):
        w = bt.bt_search_workspace_bytes(h, nq)
        assert w >= prev and w % 256 == 0 and w >= nq * (4 + 4)
        prev = w
    assert bt.bt_search_workspace_bytes(h, 0) == 0
    bt.bt_free(h)


def test_search_argument_errors(bt):
    h = bt.bt_build(np.empty(0, np.uint64), np.empty(0, np.uint64), 32, stream=0)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_search_batch(h, 0, 10, 0, 0, 0, 0, stream=0)  # null pointers
    assert e.value.code == "BT_ERR_ARG"
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_search_batch(h, 256, 10, 512, 768, 0, 0, stream=0)  # no workspace
    assert e.value.code == "BT_ERR_WORKSPACE"
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_search_batch(h, 256, 1 << 31, 512, 768, 1024, 1 << 40, stream=0)
    assert e.value.code == "BT_ERR_ARG"
    bt.bt_free(h)


def test_server_and_forest_argument_checks(bt):
    lib = bt._lib
    out = ctypes.c_void_p()
    # no trees / bad options are refused before any device work
    assert lib.bt_server_create(None, None, 0, None, ctypes.byref(out)) == 1
    assert lib.bt_forest_create(None, 0, ctypes.byref(out)) == 1
    assert lib.bt_forest_workspace_bytes(9) == 40
    assert lib.bt_tree_set_launch(None, 8, 0) == 1


def test_paper_node_bytes_follows_eq1(bt):
    """Eq. 1: N_size = 32 + 32 k_max + 32 (k_max + 1) / 4 = 40 m bytes for
    32-byte keys; integer keys keep the 32-byte header and 8-byte child
    addresses, padded to whole 32-byte chunks."""
    for m in (8, 16, 32, 64):
        kmax = m - 1
        assert bt.bt_paper_node_bytes(m, bt.BT_B32) == 32 + 32 * kmax + 32 * (kmax + 1) // 4 == 40 * m
        for w in (4, 8):
            raw = 32 + -(-(w * kmax) // 8) * 8 + 8 * m
            got = bt.bt_paper_node_bytes(m, w)
            assert got % 32 == 0 and raw <= got < raw + 32
    assert bt.bt_paper_node_bytes(2, bt.BT_U64) == 0 and bt.bt_paper_node_bytes(16, 16) == 0


def test_paper_layout_entry_points_check_arguments(bt):
    h = bt.bt_build(np.empty(0, np.uint64), np.empty(0, np.uint64), 16, stream=0)
    bt.bt_paper_layout_build(h, stream=0)  # empty tree: nothing to build
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_paper_search_batch(0, 256, 10, 512, 768, 1024, 1 << 20, stream=0)
    assert e.value.code == "BT_ERR_ARG"
    bt.bt_paper_search_batch(h, 0, 0, 0, 0, 0, 0, stream=0)  # nq = 0 is a no-op
    bt.bt_free(h)


def test_range_build_rejects_bad_arguments_before_touching_the_gpu(bt):
    import ctypes
    lib = bt._lib
    keys = np.arange(10, dtype=np.uint64)
    out = ctypes.c_void_p()
    for parts in (0, 65, 11):  # none, too many, more than keys
        assert lib.bt_range_build(keys.ctypes.data, keys.ctypes.data, 10, 8, 8, 16, parts, None,
                                  ctypes.byref(out)) == 1
    assert lib.bt_range_build(keys.ctypes.data, keys.ctypes.data, 10, 32, 8, 16, 2, None, ctypes.byref(out)) == 1
    assert lib.bt_range_workspace_bytes(None, 100) == 0
    assert lib.bt_range_part(None, 0) is None


def test_corun_caps_check_their_range(bt):
    # an empty tree is built without a device; the setter only stores the caps
    h = bt.bt_build(np.empty(0, np.uint64), np.empty(0, np.uint64), 32, stream=0)
    bt.bt_tree_set_corun(h, 3, 1)
    bt.bt_tree_set_corun(h, 0, 0)
    for d, p in ((33, 1), (3, 33)):
        with pytest.raises(bt.BTreeError) as e:
            bt.bt_tree_set_corun(h, d, p)
        assert e.value.code == "BT_ERR_ARG"
    assert bt._lib.bt_tree_set_corun(None, 3, 1) == 1
    bt.bt_free(h)
