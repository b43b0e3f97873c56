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

BT_U32, BT_U64 = 4, 8
BT_MAX_LEVELS = 24
STATUS = {0: "BT_OK", 1: "BT_ERR_ARG", 2: "BT_ERR_UNSORTED", 3: "BT_ERR_DUPLICATE",
          4: "BT_ERR_FANOUT", 5: "BT_ERR_NOMEM", 6: "BT_ERR_CUDA", 7: "BT_ERR_TIMEOUT",
          8: "BT_ERR_WORKSPACE"}

# Every symbol include/btree_gb300.h declares.
EXPORTED = ("bt_build", "bt_free", "bt_tree_info", "bt_tree_copy_image", "bt_search_workspace_bytes",
            "bt_search_batch", "bt_search_batch_ex", "bt_sort_batch", "bt_descend_sorted", "bt_sort_passes", "bt_workspace_status",
            "bt_search_host_workspace_bytes",
            "bt_search_batch_host", "bt_search_batch_noalloc", "bt_status_str", "bt_last_error_detail")


class bt_info(ctypes.Structure):
    _fields_ = [("height", ctypes.c_uint32), ("fanout", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("val_bytes", ctypes.c_uint32),
                ("n", ctypes.c_uint64),
                ("level_nodes", ctypes.c_uint64 * BT_MAX_LEVELS),
                ("level_key_offset", ctypes.c_uint64 * BT_MAX_LEVELS),
                ("leaf_val_offset", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("d_image", ctypes.c_void_p)]


class bt_search_opts(ctypes.Structure):
    _fields_ = [("sort_bits", ctypes.c_int32), ("d_fetch_counts", ctypes.c_void_p)]


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
_lib.bt_sort_passes.restype = ctypes.c_int32
_lib.bt_sort_passes.argtypes = [_vp, _u64, ctypes.c_int32]
_lib.bt_workspace_status.restype = _i
_lib.bt_workspace_status.argtypes = [_vp, _vp, _u64]
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
    """Bulk-load a tree from sorted host keys/values; returns the opaque handle."""
    k = np.ascontiguousarray(h_keys)
    v = np.ascontiguousarray(h_vals)
    if k.shape != v.shape or k.ndim != 1:
        raise ValueError("keys and values must be 1-D arrays of equal length")
    out = _vp()
    st = _lib.bt_build(k.ctypes.data if k.size else None, v.ctypes.data if v.size else None,
                       k.size, _width(k.dtype), _width(v.dtype), fanout, _stream_handle(stream),
                       ctypes.byref(out))
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
                       ws_bytes: int, sort_bits: int = -1, d_fetch_counts=None, stream=None) -> None:
    opts = bt_search_opts(sort_bits, _dptr(d_fetch_counts))
    st = _lib.bt_search_batch_ex(tree, _dptr(d_queries), nq, _dptr(d_out_vals), _dptr(d_out_found),
                                 _dptr(d_workspace), ws_bytes, ctypes.byref(opts), _stream_handle(stream))
    _check("bt_search_batch_ex", st)


def bt_sort_batch(tree: int, d_queries, nq: int, sort_bits: int, d_sorted_queries, d_sorted_index,
                  d_workspace, ws_bytes: int, stream=None) -> None:
    st = _lib.bt_sort_batch(tree, _dptr(d_queries), nq, sort_bits, _dptr(d_sorted_queries),
                            _dptr(d_sorted_index), _dptr(d_workspace), ws_bytes, _stream_handle(stream))
    _check("bt_sort_batch", st)


def bt_sort_passes(tree: int, nq: int, sort_bits: int = -1) -> int:
    return int(_lib.bt_sort_passes(tree, nq, sort_bits))


def bt_workspace_status(tree: int, d_workspace, nq: int) -> int:
    """0 (BT_OK) or 7 (BT_ERR_TIMEOUT) for the last sort in this workspace."""
    st = int(_lib.bt_workspace_status(tree, _dptr(d_workspace), nq))
    if st not in (0, 7):
        _check("bt_workspace_status", st)
    return st


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

    def __init__(self, keys: np.ndarray, vals: np.ndarray, fanout: int, stream=None):
        self.handle = bt_build(keys, vals, fanout, stream)
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

    def search_into(self, d_queries, d_out_vals, d_out_found, d_workspace, ws_bytes: int,
                    sort_bits: int = -1, d_fetch_counts=None, stream=None):
        bt_search_batch_ex(self.handle, d_queries, int(d_queries.numel()), d_out_vals, d_out_found,
                           d_workspace, ws_bytes, sort_bits, d_fetch_counts, stream)

    def search(self, d_queries, sort_bits: int = -1, stream=None):
        """Allocate outputs and workspace, search, return (values, found) CUDA tensors."""
        nq = int(d_queries.numel())
        v, f = self.alloc_outputs(nq)
        ws, nb = self.alloc_workspace(nq)
        self.search_into(d_queries, v, f, ws, nb, sort_bits=sort_bits, stream=stream)
        return v, f

    def search_host(self, h_queries: np.ndarray, stream=None):
        """Search from host memory through bt_search_batch_host; returns numpy arrays."""
        import torch
        nq = int(h_queries.size)
        vals = np.empty(nq, np.uint64 if self.val_bytes == 8 else np.uint32)
        found = np.empty(nq, np.uint8)
        ws, nb = self.alloc_workspace(nq, host=True)
        bt_search_batch_host(self.handle, np.ascontiguousarray(h_queries), nq, vals, found, ws, nb, stream)
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return vals, found
