"""Thin ctypes binding of the C ABI in ``include/btree_gb300.h``.

Argument marshalling only: every step of a search runs in the CUDA library
``libbtgb300.so``.  The functions keep the C names (``bt_build``,
``bt_search_batch``, ...) and take numpy arrays (host) or torch CUDA tensors
(device) where the C call takes pointers; ``BTree`` wraps them for
convenience.  Importing this module raises if the library has not been built
(``__graft_entry__.build()``): there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbtgb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

BT_U32, BT_U64, BT_B32 = 4, 8, 32
BT_MAX_LEVELS = 24
STATUS = {0: "BT_OK", 1: "BT_ERR_ARG", 2: "BT_ERR_UNSORTED", 3: "BT_ERR_DUPLICATE",
          4: "BT_ERR_FANOUT", 5: "BT_ERR_NOMEM", 6: "BT_ERR_CUDA", 7: "BT_ERR_TIMEOUT",
          8: "BT_ERR_WORKSPACE"}

# Every symbol include/btree_gb300.h declares.
EXPORTED = ("bt_build", "bt_free", "bt_tree_info", "bt_tree_copy_image", "bt_search_workspace_bytes",
            "bt_search_batch", "bt_search_batch_ex", "bt_sort_batch", "bt_descend_sorted", "bt_sort_launches", "bt_sort_bits",
            "bt_search_host_workspace_bytes",
            "bt_search_batch_host", "bt_search_batch_noalloc", "bt_status_str", "bt_last_error_detail",
            "bt_model_train", "bt_model_free", "bt_model_get_info", "bt_model_copy_params", "bt_mlp_grad",
            "bt_learned_descend_sorted", "bt_learned_search_batch", "bt_model_copy_err_bounds",
            "bt_forest_create", "bt_forest_create_learned", "bt_forest_free", "bt_forest_set_launch",
            "bt_forest_get_launch", "bt_forest_autotune", "bt_forest_workspace_bytes", "bt_forest_search", "bt_forest_bad_batches", "bt_tree_set_launch", "bt_tree_set_staging",
            "bt_tree_set_lane_queries", "bt_tree_set_descent", "bt_tree_set_l2_window", "bt_tree_set_corun", "bt_debug_set_wait_polls",
            "bt_check_timeouts", "bt_autotune", "bt_paper_node_bytes", "bt_paper_layout_build",
            "bt_paper_search_batch", "bt_paper_descend_sorted",
            "bt_server_create", "bt_server_submit", "bt_server_poll", "bt_server_drain", "bt_server_get_stats",
            "bt_server_destroy", "bt_server_run_trace", "bt_range_build", "bt_range_free", "bt_range_info",
            "bt_range_part", "bt_range_workspace_bytes", "bt_range_search")


class bt_info(ctypes.Structure):
    _fields_ = [("height", ctypes.c_uint32), ("fanout", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("val_bytes", ctypes.c_uint32),
                ("n", ctypes.c_uint64),
                ("level_nodes", ctypes.c_uint64 * BT_MAX_LEVELS),
                ("level_key_offset", ctypes.c_uint64 * BT_MAX_LEVELS),
                ("leaf_val_offset", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("split_offset", ctypes.c_uint64), ("split_inv_offset", ctypes.c_uint64),
                ("nsplit", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("d_image", ctypes.c_void_p)]


class bt_search_opts(ctypes.Structure):
    _fields_ = [("sort_bits", ctypes.c_int32), ("d_fetch_counts", ctypes.c_void_p), ("phase_event", ctypes.c_void_p)]


_vp, _u64, _i = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
_lib.bt_build.restype = _i
_lib.bt_build.argtypes = [_vp, _vp, _u64, _i, _i, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]
_lib.bt_free.restype = None
_lib.bt_free.argtypes = [_vp]
_lib.bt_tree_info.restype = _i
_lib.bt_tree_info.argtypes = [_vp, ctypes.POINTER(bt_info)]
_lib.bt_tree_copy_image.restype = _i
_lib.bt_tree_copy_image.argtypes = [_vp, _vp, _u64]
_lib.bt_search_workspace_bytes.restype = _u64
_lib.bt_search_workspace_bytes.argtypes = [_vp, _u64]
_lib.bt_search_host_workspace_bytes.restype = _u64
_lib.bt_search_host_workspace_bytes.argtypes = [_vp, _u64]
_lib.bt_search_batch.restype = _i
_lib.bt_search_batch.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]
_lib.bt_search_batch_ex.restype = _i
_lib.bt_search_batch_ex.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, ctypes.POINTER(bt_search_opts), _vp]
_lib.bt_sort_batch.restype = _i
_lib.bt_sort_batch.argtypes = [_vp, _vp, _u64, ctypes.c_int32, _vp, _vp, _vp, _u64, _vp]
_lib.bt_sort_launches.restype = ctypes.c_int32
_lib.bt_sort_launches.argtypes = [_vp, _u64, ctypes.c_int32]
_lib.bt_sort_bits.restype = ctypes.c_int32
_lib.bt_sort_bits.argtypes = [_vp, _u64, ctypes.c_int32]
_lib.bt_descend_sorted.restype = _i
_lib.bt_descend_sorted.argtypes = [_vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp]
_lib.bt_search_batch_host.restype = _i
_lib.bt_search_batch_host.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]
_lib.bt_search_batch_noalloc.restype = _i
_lib.bt_search_batch_noalloc.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
_lib.bt_status_str.restype = ctypes.c_char_p
_lib.bt_status_str.argtypes = [_i]
_lib.bt_last_error_detail.restype = ctypes.c_char_p
_lib.bt_last_error_detail.argtypes = []


class BTreeError(RuntimeError):
    def __init__(self, call: str, status: int):
        self.status = status
        self.code = STATUS.get(status, str(status))
        detail = _lib.bt_last_error_detail().decode() if status == 6 else ""
        msg = f"{call}: {self.code} ({_lib.bt_status_str(status).decode()})"
        super().__init__(msg + (f" -- {detail}" if detail else ""))


def _check(call: str, st: int):
    if st != 0:
        raise BTreeError(call, st)


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int | None:
    """Device address of a torch CUDA tensor (or a raw int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _width(dtype) -> int:
    dt = np.dtype(dtype)
    if dt == np.uint32:
        return BT_U32
    if dt == np.uint64:
        return BT_U64
    raise ValueError("keys and values must be uint32 or uint64")


def bt_status_str(status: int) -> str:
    return _lib.bt_status_str(status).decode()


def bt_build(h_keys: np.ndarray, h_vals: np.ndarray, fanout: int, stream=None) -> int:
    """Bulk-load a tree from sorted host keys/values; returns the opaque handle.
    Keys: a 1-D uint32/uint64 array, or an (n, 32) uint8 array of 32-byte keys."""
    k = np.ascontiguousarray(h_keys)
    v = np.ascontiguousarray(h_vals)
    if k.ndim == 2 and k.dtype == np.uint8 and k.shape[1] == 32:
        n, kw = k.shape[0], BT_B32
    elif k.ndim == 1:
        n, kw = k.size, _width(k.dtype)
    else:
        raise ValueError("keys must be a 1-D uint32/uint64 array or an (n, 32) uint8 array")
    if v.ndim != 1 or v.size != n:
        raise ValueError("values must be a 1-D array with one value per key")
    out = _vp()
    st = _lib.bt_build(k.ctypes.data if n else None, v.ctypes.data if n else None,
                       n, kw, _width(v.dtype), fanout, _stream_handle(stream), ctypes.byref(out))
    _check("bt_build", st)
    return out.value


def bt_free(tree: int) -> None:
    _lib.bt_free(tree)


def bt_tree_info(tree: int) -> bt_info:
    info = bt_info()
    _check("bt_tree_info", _lib.bt_tree_info(tree, ctypes.byref(info)))
    return info


def bt_tree_copy_image(tree: int, nbytes: int) -> np.ndarray:
    out = np.empty(nbytes, np.uint8)
    _check("bt_tree_copy_image", _lib.bt_tree_copy_image(tree, out.ctypes.data, nbytes))
    return out


def bt_search_workspace_bytes(tree: int, nq: int) -> int:
    return int(_lib.bt_search_workspace_bytes(tree, nq))


def bt_search_host_workspace_bytes(tree: int, nq: int) -> int:
    return int(_lib.bt_search_host_workspace_bytes(tree, nq))


def bt_search_batch(tree: int, d_queries, nq: int, d_out_vals, d_out_found, d_workspace,
                    ws_bytes: int, stream=None) -> None:
    st = _lib.bt_search_batch(tree, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                              _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_search_batch", st)


def bt_search_batch_ex(tree: int, d_queries, nq: int, d_out_vals, d_out_found, d_workspace,
                       ws_bytes: int, sort_bits: int = -1, d_fetch_counts=None, stream=None,
                       phase_event=None) -> None:
    """phase_event: a torch.cuda.Event (or raw cudaEvent_t) recorded between the
    partition and the descent."""
    ev = None
    if phase_event is not None:
        ev = phase_event if isinstance(phase_event, int) else phase_event.cuda_event
    opts = bt_search_opts(sort_bits, _dptr(d_fetch_counts), ev)
    st = _lib.bt_search_batch_ex(tree, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                                 _dptr(d_workspace), ws_bytes, ctypes.byref(opts), _stream_handle(stream))
    _check("bt_search_batch_ex", st)


def bt_sort_batch(tree: int, d_queries, nq: int, sort_bits: int, d_sorted_queries, d_sorted_index,
                  d_workspace, ws_bytes: int, stream=None) -> None:
    st = _lib.bt_sort_batch(tree, _dptr(d_queries), nq, sort_bits, _dptr(d_sorted_queries),
                            _dptr(d_sorted_index), _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_sort_batch", st)


def bt_sort_launches(tree: int, nq: int, sort_bits: int = -1) -> int:
    return int(_lib.bt_sort_launches(tree, nq, sort_bits))


def bt_sort_bits(tree: int, nq: int, sort_bits: int = -1) -> int:
    return int(_lib.bt_sort_bits(tree, nq, sort_bits))


def bt_descend_sorted(tree: int, d_queries, d_index, nq: int, d_out_vals, d_out_found,
                      d_fetch_counts=None, stream=None) -> None:
    st = _lib.bt_descend_sorted(tree, _dptr(d_queries), _dptr(d_index), nq, _dptr(d_out_vals),
                                _dptr(d_out_found), _dptr(d_fetch_counts), _stream_handle(stream))
    _check("bt_descend_sorted", st)


def bt_search_batch_host(tree: int, h_queries, nq: int, h_out_vals, h_out_found, d_workspace,
                         ws_bytes: int, stream=None) -> None:
    """Host buffers: numpy arrays or pinned CPU torch tensors."""
    def hp(a):
        if isinstance(a, np.ndarray):
            if not a.flags.c_contiguous:
                raise ValueError("host buffers must be contiguous")
            return a.ctypes.data
        if a.is_cuda:
            raise ValueError("expected a host buffer")
        return a.data_ptr()
    st = _lib.bt_search_batch_host(tree, hp(h_queries), nq, hp(h_out_vals), hp(h_out_found),
                                   _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_search_batch_host", st)


BT_MODEL_PL, BT_MODEL_MLP = 1, 2
BT_MLP_PARAMS = 1153


class bt_learn_opts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("segments", ctypes.c_uint32), ("h_init", ctypes.c_void_p),
                ("steps", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class bt_model_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("segments", ctypes.c_uint32), ("leaves", ctypes.c_uint32),
                ("max_err", ctypes.c_uint32), ("final_loss", ctypes.c_float), ("device_bytes", ctypes.c_uint64)]


_lib.bt_model_train.restype = _i
_lib.bt_model_train.argtypes = [_vp, ctypes.POINTER(bt_learn_opts), _vp, ctypes.POINTER(_vp)]
_lib.bt_model_free.restype = None
_lib.bt_model_free.argtypes = [_vp]
_lib.bt_model_get_info.restype = _i
_lib.bt_model_get_info.argtypes = [_vp, ctypes.POINTER(bt_model_info)]
_lib.bt_model_copy_params.restype = _i
_lib.bt_model_copy_params.argtypes = [_vp, _vp, _u64]
_lib.bt_mlp_grad.restype = _i
_lib.bt_mlp_grad.argtypes = [_vp, _vp, _vp, ctypes.c_uint32, _vp, _vp, _vp]
_lib.bt_learned_descend_sorted.restype = _i
_lib.bt_learned_descend_sorted.argtypes = [_vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp]
_lib.bt_learned_search_batch.restype = _i
_lib.bt_learned_search_batch.argtypes = [_vp, _vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]


def bt_model_train(tree: int, kind: int, segments: int = 256, h_init=None, steps: int = 0, batch: int = 0,
                   lr: float = 0.0, seed: int = 0, stream=None) -> int:
    """Fit (PL) or train (MLP) a leaf predictor for `tree` on the GPU."""
    init = None
    if h_init is not None:
        init = np.ascontiguousarray(h_init, dtype=np.float32)
        if init.size != BT_MLP_PARAMS:
            raise ValueError(f"h_init must hold {BT_MLP_PARAMS} floats")
    o = bt_learn_opts(kind, segments, init.ctypes.data if init is not None else None, steps, batch, lr, seed)
    out = _vp()
    _check("bt_model_train", _lib.bt_model_train(tree, ctypes.byref(o), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def bt_model_free(model: int) -> None:
    _lib.bt_model_free(model)


def bt_model_get_info(model: int) -> bt_model_info:
    info = bt_model_info()
    _check("bt_model_get_info", _lib.bt_model_get_info(model, ctypes.byref(info)))
    return info


def bt_model_copy_params(model: int):
    """PL: (b uint64[S], inv_w, slope, icpt float32[S]); MLP: float32[1153]."""
    info = bt_model_get_info(model)
    if info.kind == BT_MODEL_PL:
        S = int(info.segments)
        buf = np.empty(20 * S, np.uint8)
        _check("bt_model_copy_params", _lib.bt_model_copy_params(model, buf.ctypes.data, buf.size))
        return (buf[:8 * S].view(np.uint64).copy(), buf[8 * S:12 * S].view(np.float32).copy(),
                buf[12 * S:16 * S].view(np.float32).copy(), buf[16 * S:].view(np.float32).copy())
    out = np.empty(BT_MLP_PARAMS, np.float32)
    _check("bt_model_copy_params", _lib.bt_model_copy_params(model, out.ctypes.data, out.nbytes))
    return out


BT_ERR_RANGES = 256
_lib.bt_model_copy_err_bounds.restype = _i
_lib.bt_model_copy_err_bounds.argtypes = [_vp, _vp, ctypes.c_uint32]


def bt_model_copy_err_bounds(model: int) -> np.ndarray:
    out = np.zeros(BT_ERR_RANGES, np.uint32)
    _check("bt_model_copy_err_bounds", _lib.bt_model_copy_err_bounds(model, out.ctypes.data, out.size))
    return out


def bt_mlp_grad(d_params, d_x, d_t, n: int, d_grad, d_loss, stream=None) -> None:
    _check("bt_mlp_grad", _lib.bt_mlp_grad(_dptr(d_params), _dptr(d_x), _dptr(d_t), n, _dptr(d_grad),
                                           _dptr(d_loss), _stream_handle(stream)))


def bt_learned_descend_sorted(tree: int, model: int, d_queries, d_index, nq: int, d_out_vals, d_out_found,
                              d_stats=None, stream=None) -> None:
    st = _lib.bt_learned_descend_sorted(tree, model, _dptr(d_queries), _dptr(d_index), nq, _dptr(d_out_vals),
                                        _dptr(d_out_found), _dptr(d_stats), _stream_handle(stream))
    _check("bt_learned_descend_sorted", st)


def bt_learned_search_batch(tree: int, model: int, d_queries, nq: int, d_out_vals, d_out_found, d_workspace,
                            ws_bytes: int, stream=None) -> None:
    st = _lib.bt_learned_search_batch(tree, model, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                                      _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_learned_search_batch", st)


class bt_batch_desc(ctypes.Structure):
    _fields_ = [("tree", ctypes.c_uint32), ("count", ctypes.c_uint32), ("offset", ctypes.c_uint64)]


class bt_tune(ctypes.Structure):
    _fields_ = [("fanout", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32), ("pin_bytes", ctypes.c_uint32),
                ("staging", ctypes.c_uint32), ("lane_queries", ctypes.c_uint32),
                ("inner_staged", ctypes.c_uint32), ("us_per_batch", ctypes.c_float)]


class bt_forest_tune(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_uint32), ("pin_budget", ctypes.c_uint32),
                ("lane_queries", ctypes.c_uint32), ("staging", ctypes.c_uint32), ("pin_applied", ctypes.c_uint32),
                ("us", ctypes.c_float)]


BATCH_DESC_DTYPE = np.dtype([("tree", np.uint32), ("count", np.uint32), ("offset", np.uint64)])

_lib.bt_forest_create.restype = _i
_lib.bt_forest_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.POINTER(_vp)]
_lib.bt_forest_create_learned.restype = _i
_lib.bt_forest_create_learned.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_uint32,
                                          ctypes.POINTER(_vp)]
_lib.bt_forest_free.restype = None
_lib.bt_forest_free.argtypes = [_vp]
_lib.bt_forest_set_launch.restype = _i
_lib.bt_forest_set_launch.argtypes = [_vp, ctypes.POINTER(bt_forest_tune)]
_lib.bt_forest_get_launch.restype = _i
_lib.bt_forest_get_launch.argtypes = [_vp, ctypes.POINTER(bt_forest_tune)]
_lib.bt_forest_autotune.restype = _i
_lib.bt_forest_autotune.argtypes = [_vp, _vp, ctypes.c_uint32, _vp, _u64, _vp, _vp, _vp, _u64, _vp,
                                    ctypes.POINTER(bt_forest_tune)]
_lib.bt_forest_workspace_bytes.restype = _u64
_lib.bt_forest_workspace_bytes.argtypes = [ctypes.c_uint32]
_lib.bt_forest_search.restype = _i
_lib.bt_forest_search.argtypes = [_vp, _vp, ctypes.c_uint32, _vp, _u64, _vp, _vp, _vp, _u64, ctypes.c_uint32, _vp]
_lib.bt_forest_bad_batches.restype = _i
_lib.bt_forest_bad_batches.argtypes = [ctypes.POINTER(_u64)]
_lib.bt_tree_set_launch.restype = _i
_lib.bt_tree_set_launch.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32]
_lib.bt_tree_set_staging.restype = _i
_lib.bt_tree_set_staging.argtypes = [_vp, ctypes.c_uint32]
_lib.bt_tree_set_lane_queries.restype = _i
_lib.bt_tree_set_lane_queries.argtypes = [_vp, ctypes.c_uint32]
_lib.bt_tree_set_descent.restype = _i
_lib.bt_tree_set_descent.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32]
_lib.bt_tree_set_l2_window.restype = _i
_lib.bt_tree_set_l2_window.argtypes = [_vp, _u64]
_lib.bt_tree_set_corun.restype = _i
_lib.bt_tree_set_corun.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32]
_lib.bt_debug_set_wait_polls.restype = None
_lib.bt_debug_set_wait_polls.argtypes = [ctypes.c_uint32]
_lib.bt_check_timeouts.restype = _i
_lib.bt_check_timeouts.argtypes = []
_lib.bt_autotune.restype = _i
_lib.bt_autotune.argtypes = [_vp, _vp, _u64, _i, _i, _vp, _u64, _vp, ctypes.POINTER(_vp), ctypes.POINTER(bt_tune)]


def bt_forest_create(trees) -> int:
    arr = (_vp * len(trees))(*[t if isinstance(t, int) else t.handle for t in trees])
    out = _vp()
    _check("bt_forest_create", _lib.bt_forest_create(arr, len(trees), ctypes.byref(out)))
    return out.value


def bt_forest_create_learned(trees, models) -> int:
    """models: one entry per tree, a model handle or None (plain descent)."""
    if len(models) != len(trees):
        raise ValueError("one model entry per tree")
    arr = (_vp * len(trees))(*[t if isinstance(t, int) else t.handle for t in trees])
    marr = (_vp * len(models))(*[m if m else None for m in models])
    out = _vp()
    _check("bt_forest_create_learned", _lib.bt_forest_create_learned(arr, marr, len(trees), ctypes.byref(out)))
    return out.value


def bt_forest_free(forest: int) -> None:
    _lib.bt_forest_free(forest)


def bt_forest_set_launch(forest: int, warps_per_block: int = 8, pin_budget: int = 32768, lane_queries: int = 0,
                         staging: int = 0) -> None:
    cfg = bt_forest_tune(warps_per_block, pin_budget, lane_queries, staging, 0, 0.0)
    _check("bt_forest_set_launch", _lib.bt_forest_set_launch(forest, ctypes.byref(cfg)))


def bt_forest_get_launch(forest: int) -> bt_forest_tune:
    out = bt_forest_tune()
    _check("bt_forest_get_launch", _lib.bt_forest_get_launch(forest, ctypes.byref(out)))
    return out


def bt_forest_autotune(forest: int, d_batches, nbatches: int, d_queries, d_out_vals, d_out_found, d_workspace,
                       ws_bytes: int, stream=None, nq: int | None = None) -> bt_forest_tune:
    """Time the work list under every forest launch setting; keeps and returns the fastest."""
    if nq is None:
        nq = int(d_queries.numel())
    out = bt_forest_tune()
    st = _lib.bt_forest_autotune(forest, _dptr(d_batches), nbatches, _dptr(d_queries), nq, _dptr(d_out_vals),
                                 _dptr(d_out_found), _dptr(d_workspace), ws_bytes, _stream_handle(stream),
                                 ctypes.byref(out))
    _check("bt_forest_autotune", st)
    return out


def bt_forest_workspace_bytes(nbatches: int) -> int:
    return int(_lib.bt_forest_workspace_bytes(nbatches))


def bt_forest_search(forest: int, d_batches, nbatches: int, d_queries, d_out_vals, d_out_found, d_workspace,
                     ws_bytes: int, warps_per_block: int = 0, stream=None, nq: int | None = None) -> None:
    """nq: entries of the query and result arrays (default: the query tensor's length)."""
    if nq is None:
        nq = int(d_queries.numel())
    st = _lib.bt_forest_search(forest, _dptr(d_batches), nbatches, _dptr(d_queries), nq, _dptr(d_out_vals),
                               _dptr(d_out_found), _dptr(d_workspace), ws_bytes, warps_per_block,
                               _stream_handle(stream))
    _check("bt_forest_search", st)


def bt_forest_bad_batches() -> int:
    """Work-list entries the batching kernel rejected since the last call."""
    out = _u64()
    _check("bt_forest_bad_batches", _lib.bt_forest_bad_batches(ctypes.byref(out)))
    return int(out.value)


def bt_tree_set_launch(tree: int, warps_per_block: int, pin_bytes: int) -> None:
    _check("bt_tree_set_launch", _lib.bt_tree_set_launch(tree, warps_per_block, pin_bytes))


BT_STAGE_CP_ASYNC = 0
BT_STAGE_BULK = 1
BT_STAGE_PIPELINED = 2
BT_DEFAULT_WAIT_POLLS = 1 << 22


def bt_tree_set_staging(tree: int, mode: int) -> None:
    _check("bt_tree_set_staging", _lib.bt_tree_set_staging(tree, mode))


def bt_tree_set_lane_queries(tree: int, per_lane: int) -> None:
    _check("bt_tree_set_lane_queries", _lib.bt_tree_set_lane_queries(tree, per_lane))


def bt_tree_set_descent(tree: int, inner_staged: int = 0, rank_ballot: int = 0) -> None:
    _check("bt_tree_set_descent", _lib.bt_tree_set_descent(tree, inner_staged, rank_ballot))


def bt_tree_set_corun(tree: int, descent_blocks_per_sm: int, partition_blocks_per_sm: int) -> None:
    """Resident blocks per SM of the descent and the partition (0 = as many as fit)."""
    _check("bt_tree_set_corun", _lib.bt_tree_set_corun(tree, descent_blocks_per_sm, partition_blocks_per_sm))


def bt_tree_set_l2_window(tree: int, max_bytes: int) -> None:
    _check("bt_tree_set_l2_window", _lib.bt_tree_set_l2_window(tree, max_bytes))


def bt_debug_set_wait_polls(polls: int) -> None:
    _lib.bt_debug_set_wait_polls(polls)


def bt_check_timeouts() -> None:
    """Raises if a bounded device wait of a search gave up since the last call."""
    _check("bt_check_timeouts", _lib.bt_check_timeouts())


def bt_autotune(h_keys: np.ndarray, h_vals: np.ndarray, d_sample, nsample: int, stream=None):
    """(tree handle, bt_tune) with the fastest fanout and launch settings."""
    k = np.ascontiguousarray(h_keys)
    v = np.ascontiguousarray(h_vals)
    out = _vp()
    best = bt_tune()
    st = _lib.bt_autotune(k.ctypes.data, v.ctypes.data, k.size, _width(k.dtype), _width(v.dtype), _dptr(d_sample),
                          nsample, _stream_handle(stream), ctypes.byref(out), ctypes.byref(best))
    _check("bt_autotune", st)
    return out.value, best


_lib.bt_paper_node_bytes.restype = ctypes.c_uint32
_lib.bt_paper_node_bytes.argtypes = [ctypes.c_uint32, _i]
_lib.bt_paper_layout_build.restype = _i
_lib.bt_paper_layout_build.argtypes = [_vp, _vp]
_lib.bt_paper_search_batch.restype = _i
_lib.bt_paper_search_batch.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]
_lib.bt_paper_descend_sorted.restype = _i
_lib.bt_paper_descend_sorted.argtypes = [_vp, _vp, _vp, _u64, _vp, _vp, _vp]


def bt_paper_node_bytes(fanout: int, key_width: int) -> int:
    """Node size of the paper's layout (Eq. 1); 0 if unsupported."""
    return int(_lib.bt_paper_node_bytes(fanout, key_width))


def bt_paper_layout_build(tree: int, stream=None) -> None:
    _check("bt_paper_layout_build", _lib.bt_paper_layout_build(tree, _stream_handle(stream)))


def bt_paper_search_batch(tree: int, d_queries, nq: int, d_out_vals, d_out_found, d_workspace, ws_bytes: int,
                          stream=None) -> None:
    st = _lib.bt_paper_search_batch(tree, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                                    _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_paper_search_batch", st)


def bt_paper_descend_sorted(tree: int, d_queries, d_index, nq: int, d_out_vals, d_out_found, stream=None) -> None:
    st = _lib.bt_paper_descend_sorted(tree, _dptr(d_queries), _dptr(d_index), nq, _dptr(d_out_vals),
                                      _dptr(d_out_found), _stream_handle(stream))
    _check("bt_paper_descend_sorted", st)


class bt_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("deadline_us", ctypes.c_double),
                ("mem_cap_bytes", ctypes.c_uint64), ("pending_cap_bytes", ctypes.c_uint64)]


class bt_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("lookups", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("p50_us", ctypes.c_float),
                ("p99_us", ctypes.c_float), ("max_us", ctypes.c_float)]


_lib.bt_server_create.restype = _i
_lib.bt_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_uint32,
                                  ctypes.POINTER(bt_server_opts), ctypes.POINTER(_vp)]
_lib.bt_server_submit.restype = _i
_lib.bt_server_submit.argtypes = [_vp, ctypes.c_uint32, _vp, ctypes.c_uint32, _vp, _vp, ctypes.POINTER(_u64)]
_lib.bt_server_poll.restype = _i
_lib.bt_server_poll.argtypes = [_vp, ctypes.POINTER(_u64), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
_lib.bt_server_drain.restype = _i
_lib.bt_server_drain.argtypes = [_vp, ctypes.c_double]
_lib.bt_server_get_stats.restype = _i
_lib.bt_server_get_stats.argtypes = [_vp, ctypes.POINTER(bt_server_stats), _i]
_lib.bt_server_destroy.restype = None
_lib.bt_server_destroy.argtypes = [_vp]
_lib.bt_server_run_trace.restype = _i
_lib.bt_server_run_trace.argtypes = [_vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]


def bt_server_create(trees, models=None, slots: int = 4, max_batch: int = 4096, deadline_us: float = 50.0,
                     mem_cap_bytes: int = 0, pending_cap_bytes: int = 0) -> int:
    n = len(trees)
    t_arr = (_vp * n)(*[t if isinstance(t, int) else t.handle for t in trees])
    m_arr = None
    if models is not None:
        m_arr = (_vp * n)(*[m for m in models])
    o = bt_server_opts(slots, max_batch, deadline_us, mem_cap_bytes, pending_cap_bytes)
    out = _vp()
    _check("bt_server_create", _lib.bt_server_create(t_arr, m_arr, n, ctypes.byref(o), ctypes.byref(out)))
    return out.value


def bt_server_submit(server: int, tree: int, h_keys: np.ndarray, h_out_vals: np.ndarray,
                     h_out_found: np.ndarray) -> int:
    """Queue a request; the numpy buffers must stay alive until it completes."""
    t = _u64()
    st = _lib.bt_server_submit(server, tree, h_keys.ctypes.data, h_keys.size, h_out_vals.ctypes.data,
                               h_out_found.ctypes.data, ctypes.byref(t))
    _check("bt_server_submit", st)
    return int(t.value)


def bt_server_poll(server: int, max_tickets: int = 4096):
    buf = (_u64 * max_tickets)()
    n = ctypes.c_uint32()
    _check("bt_server_poll", _lib.bt_server_poll(server, buf, max_tickets, ctypes.byref(n)))
    return [int(buf[i]) for i in range(n.value)]


def bt_server_drain(server: int, timeout_s: float = 60.0) -> None:
    _check("bt_server_drain", _lib.bt_server_drain(server, timeout_s))


def bt_server_get_stats(server: int, reset: bool = False) -> bt_server_stats:
    s = bt_server_stats()
    _check("bt_server_get_stats", _lib.bt_server_get_stats(server, ctypes.byref(s), int(reset)))
    return s


def bt_server_destroy(server: int) -> None:
    _lib.bt_server_destroy(server)


def bt_server_run_trace(server: int, t_arrival_s: np.ndarray, tree: np.ndarray, count: np.ndarray,
                        key_offset: np.ndarray, h_keys: np.ndarray, h_out_vals: np.ndarray,
                        h_out_found: np.ndarray) -> float:
    """Replay an arrival trace through the server; returns the wall time (s)."""
    ta = np.ascontiguousarray(t_arrival_s, np.float64)
    tr = np.ascontiguousarray(tree, np.uint32)
    ct = np.ascontiguousarray(count, np.uint32)
    ko = np.ascontiguousarray(key_offset, np.uint64)
    wall = ctypes.c_double()
    st = _lib.bt_server_run_trace(server, ta.size, ta.ctypes.data, tr.ctypes.data, ct.ctypes.data, ko.ctypes.data,
                                  h_keys.ctypes.data, h_out_vals.ctypes.data, h_out_found.ctypes.data,
                                  ctypes.byref(wall))
    _check("bt_server_run_trace", st)
    return float(wall.value)


BT_NOALLOC_MAX_QUERIES = 65536


def bt_search_batch_noalloc(tree: int, d_queries, nq: int, d_out_vals, d_out_found, stream=None) -> None:
    """Search without a workspace or any device allocation, for callers that
    cannot allocate device memory; the library's own 2 MiB device scratch
    array is used instead (at most BT_NOALLOC_MAX_QUERIES queries; calls that
    overlap on the GPU share that array and race)."""
    st = _lib.bt_search_batch_noalloc(tree, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                                      _stream_handle(stream))
    _check("bt_search_batch_noalloc", st)


def _torch_dtype(width: int):
    import torch
    return torch.uint64 if width == 8 else torch.uint32


class BTree:
    """A tree on the current CUDA device with convenience search methods."""

    def __init__(self, keys: np.ndarray | None, vals: np.ndarray | None, fanout: int = 0, stream=None,
                 handle: int | None = None):
        """Build from sorted keys/values, or take ownership of a built tree's handle."""
        self.handle = handle if handle is not None else bt_build(keys, vals, fanout, stream)
        i = bt_tree_info(self.handle)
        self.height = int(i.height)
        self.fanout = int(i.fanout)
        self.key_bytes = int(i.key_bytes)
        self.val_bytes = int(i.val_bytes)
        self.n = int(i.n)
        self.level_nodes = [int(i.level_nodes[l]) for l in range(self.height)]
        self.device_bytes = int(i.device_bytes)

    def close(self):
        if getattr(self, "handle", None):
            bt_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, nq: int) -> int:
        return bt_search_workspace_bytes(self.handle, nq)

    def alloc_workspace(self, nq: int, host: bool = False):
        import torch
        nb = bt_search_host_workspace_bytes(self.handle, nq) if host else self.workspace_bytes(nq)
        # torch's caching allocator returns 512-byte aligned blocks
        return torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda"), nb

    def alloc_outputs(self, nq: int):
        import torch
        v = torch.empty(nq, dtype=_torch_dtype(self.val_bytes), device="cuda")
        f = torch.empty(nq, dtype=torch.uint8, device="cuda")
        return v, f

    def count(self, queries) -> int:
        """Queries in a batch: its elements, or its rows of 32 bytes for 32-byte keys."""
        n = int(queries.numel() if hasattr(queries, "numel") else np.asarray(queries).size)
        return n // 32 if self.key_bytes == 32 else n

    def search_into(self, d_queries, d_out_vals, d_out_found, d_workspace, ws_bytes: int,
                    sort_bits: int = -1, d_fetch_counts=None, stream=None):
        bt_search_batch_ex(self.handle, d_queries, self.count(d_queries), d_out_vals, d_out_found,
                           d_workspace, ws_bytes, sort_bits, d_fetch_counts, stream)

    def search(self, d_queries, sort_bits: int = -1, stream=None):
        """Allocate outputs and workspace, search, return (values, found) CUDA tensors."""
        nq = self.count(d_queries)
        v, f = self.alloc_outputs(nq)
        ws, nb = self.alloc_workspace(nq)
        self.search_into(d_queries, v, f, ws, nb, sort_bits=sort_bits, stream=stream)
        return v, f

    def search_host(self, h_queries: np.ndarray, stream=None):
        """Search from host memory through bt_search_batch_host; returns numpy arrays."""
        import torch
        nq = self.count(h_queries)
        vals = np.empty(nq, np.uint64 if self.val_bytes == 8 else np.uint32)
        found = np.empty(nq, np.uint8)
        ws, nb = self.alloc_workspace(nq, host=True)
        bt_search_batch_host(self.handle, np.ascontiguousarray(h_queries), nq, vals, found, ws, nb, stream)
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return vals, found


# ------------------------------------------------------------ range partition

_lib.bt_range_build.restype = _i
_lib.bt_range_build.argtypes = [_vp, _vp, _u64, _i, _i, ctypes.c_uint32, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]
_lib.bt_range_free.restype = None
_lib.bt_range_free.argtypes = [_vp]
_lib.bt_range_info.restype = _i
_lib.bt_range_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint32), _vp, _vp]
_lib.bt_range_part.restype = _vp
_lib.bt_range_part.argtypes = [_vp, ctypes.c_uint32]
_lib.bt_range_workspace_bytes.restype = _u64
_lib.bt_range_workspace_bytes.argtypes = [_vp, _u64]
_lib.bt_range_search.restype = _i
_lib.bt_range_search.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _vp]


def bt_range_build(h_keys: np.ndarray, h_vals: np.ndarray, fanout: int, parts: int, stream=None) -> int:
    k = np.ascontiguousarray(h_keys)
    v = np.ascontiguousarray(h_vals)
    out = _vp()
    st = _lib.bt_range_build(k.ctypes.data, v.ctypes.data, k.size, _width(k.dtype), _width(v.dtype), fanout, parts,
                             _stream_handle(stream), ctypes.byref(out))
    _check("bt_range_build", st)
    return out.value


def bt_range_free(r: int) -> None:
    _lib.bt_range_free(r)


def bt_range_info(r: int):
    """(parts, splitters uint64[P-1], keys per part uint64[P])."""
    p = ctypes.c_uint32()
    _check("bt_range_info", _lib.bt_range_info(r, ctypes.byref(p), None, None))
    sp = np.zeros(max(p.value - 1, 1), np.uint64)
    nk = np.zeros(p.value, np.uint64)
    _check("bt_range_info", _lib.bt_range_info(r, ctypes.byref(p), sp.ctypes.data, nk.ctypes.data))
    return int(p.value), sp[: p.value - 1], nk


def bt_range_part(r: int, p: int) -> int | None:
    return _lib.bt_range_part(r, p)


def bt_range_workspace_bytes(r: int, nq: int) -> int:
    return int(_lib.bt_range_workspace_bytes(r, nq))


def bt_range_search(r: int, d_queries, nq: int, d_out_vals, d_out_found, d_workspace, ws_bytes: int,
                    stream=None) -> None:
    st = _lib.bt_range_search(r, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found), _dptr(d_workspace),
                              ws_bytes, _stream_handle(stream))
    _check("bt_range_search", st)
