"""CPU oracle for B+ tree point search on fixed-width byte-string keys (the
paper's 32-byte keys) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  The tree (``btree_oracle_bytes.c``) is the same even
bulk load as the integer-key oracle, with keys compared byte by byte from the
first byte on (Sec. IV-E's per-byte comparators and their cascade, i.e.
lexicographic order).

Pinned by ``tests/test_oracle_bytes.py``: a Python dict (brute-force point
lookup), Python's own ``bytes`` ordering with ``bisect`` (leaf = the leaf
holding the lower bound), the integer-key oracle on big-endian encodings of
integers (where byte order and integer order agree), structural invariants,
and a planted little-endian compare that those pins must catch.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btree_oracle_bytes.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_bytes.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)


def compile_oracle(out_path: str = _LIB_PATH, defines: tuple[str, ...] = ()) -> str:
    """Compile btree_oracle_bytes.c with gcc into a shared library at out_path."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread"]
    cmd += [f"-D{d}" for d in defines]
    tmp = out_path + ".tmp"
    cmd += ["-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.btb_build.restype = ctypes.c_void_p
    lib.btb_build.argtypes = [_u8p, _u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.btb_free.restype = None
    lib.btb_free.argtypes = [ctypes.c_void_p]
    lib.btb_search.restype = None
    lib.btb_search.argtypes = [ctypes.c_void_p, _u8p, ctypes.c_uint64, _u64p, _u8p, _u64p, _i32p]
    lib.btb_search_mt.restype = ctypes.c_int
    lib.btb_search_mt.argtypes = [ctypes.c_void_p, _u8p, ctypes.c_uint64, _u64p, _u8p, ctypes.c_int]
    lib.btb_paths.restype = None
    lib.btb_paths.argtypes = [ctypes.c_void_p, _u8p, ctypes.c_uint64, _u64p]
    lib.btb_height.restype = ctypes.c_int
    lib.btb_height.argtypes = [ctypes.c_void_p]
    lib.btb_level_nodes.restype = ctypes.c_uint64
    lib.btb_level_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.btb_node_dump.restype = ctypes.c_int
    lib.btb_node_dump.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_int), _u8p, _u64p, _u64p]
    return lib


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the byte-key oracle (compiling it first if missing or stale)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            compile_oracle()
        _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def load_planted(define: str) -> ctypes.CDLL:
    """A copy compiled with one planted mistake (pin-strength tests)."""
    d = tempfile.mkdtemp(prefix="oracle_bytes_plant_")
    return load(compile_oracle(os.path.join(d, f"liboracle_bytes_{define}.so"), (define,)))


def _rows(a, kb: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8))
    if a.ndim != 2 or a.shape[1] != kb:
        raise ValueError(f"expected an (n, {kb}) uint8 array of keys")
    return a


class OracleBytesTree:
    """Pointer-based CPU B+ tree over kb-byte keys: bulk load, then one query
    at a time from the root."""

    def __init__(self, keys, vals, m: int, val_bits: int = 64, lib: ctypes.CDLL | None = None):
        self._lib = lib if lib is not None else load()
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8))
        self.kb = int(k.shape[1])
        self.m = int(m)
        self.val_bits = int(val_bits)
        v = np.ascontiguousarray(np.asarray(vals).astype(np.uint64, copy=False))
        assert v.size == k.shape[0]
        self.n = int(v.size)
        self._keep = (k, v)
        self._h = self._lib.btb_build(k.ctypes.data_as(_u8p), v.ctypes.data_as(_u64p), self.n, self.kb, self.m,
                                      self.val_bits)
        if not self._h:
            raise ValueError("byte-key oracle bulk load failed")
        self.miss = (1 << self.val_bits) - 1

    def close(self):
        if self._h:
            self._lib.btb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def height(self) -> int:
        return int(self._lib.btb_height(self._h))

    def level_nodes(self) -> list[int]:
        return [int(self._lib.btb_level_nodes(self._h, l)) for l in range(self.height)]

    def search(self, queries):
        """(values uint64, found uint8, leaf index uint64, slot int32)."""
        q = _rows(queries, self.kb)
        n = q.shape[0]
        vals = np.empty(n, np.uint64)
        found = np.empty(n, np.uint8)
        leaf = np.empty(n, np.uint64)
        slot = np.empty(n, np.int32)
        self._lib.btb_search(self._h, q.ctypes.data_as(_u8p), n, vals.ctypes.data_as(_u64p),
                             found.ctypes.data_as(_u8p), leaf.ctypes.data_as(_u64p), slot.ctypes.data_as(_i32p))
        return vals, found, leaf, slot

    def search_mt(self, queries, nthreads: int):
        q = _rows(queries, self.kb)
        n = q.shape[0]
        vals = np.empty(n, np.uint64)
        found = np.empty(n, np.uint8)
        if self._lib.btb_search_mt(self._h, q.ctypes.data_as(_u8p), n, vals.ctypes.data_as(_u64p),
                                   found.ctypes.data_as(_u8p), int(nthreads)) != 0:
            raise RuntimeError("oracle thread start failed")
        return vals, found

    def paths(self, queries) -> np.ndarray:
        q = _rows(queries, self.kb)
        h = self.height
        out = np.zeros((q.shape[0], max(h, 1)), np.uint64)
        if h:
            self._lib.btb_paths(self._h, q.ctypes.data_as(_u8p), q.shape[0], out.ctypes.data_as(_u64p))
        return out[:, :h]

    def node(self, level: int, index: int):
        """(is_leaf, keys as (k, kb) uint8, values or None, child indices or None)."""
        is_leaf = ctypes.c_int(0)
        keys = np.zeros((self.m, self.kb), np.uint8)
        vals = np.zeros(self.m, np.uint64)
        ch = np.zeros(self.m + 1, np.uint64)
        nk = self._lib.btb_node_dump(self._h, level, index, ctypes.byref(is_leaf), keys.ctypes.data_as(_u8p),
                                     vals.ctypes.data_as(_u64p), ch.ctypes.data_as(_u64p))
        if nk < 0:
            raise IndexError((level, index))
        if is_leaf.value:
            return True, keys[:nk].copy(), vals[:nk].copy(), None
        return False, keys[:nk].copy(), None, ch[:nk + 1].copy()


def dict_lookup(keys, vals, queries, val_bits: int = 64):
    """Point lookup by its plain definition: a Python dict from each key's
    bytes to its value.  Used only to pin the tree oracle."""
    k = np.asarray(keys, np.uint8)
    d = {bytes(k[i]): int(v) for i, v in enumerate(np.asarray(vals).tolist())}
    miss = (1 << val_bits) - 1
    qs = np.asarray(queries, np.uint8)
    out = np.empty(qs.shape[0], np.uint64)
    found = np.empty(qs.shape[0], np.uint8)
    for i in range(qs.shape[0]):
        v = d.get(bytes(qs[i]))
        out[i] = miss if v is None else v
        found[i] = v is not None
    return out, found
