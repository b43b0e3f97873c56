"""CPU oracle for batched B+ tree point search -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it.

The oracle is a pointer-based B+ tree in plain C (``btree_oracle.c``):
an even bulk load (the paper does not say how its trees were filled), then
one query at a time from the root, routing on "q <= separator" (Sec. IV-E)
and matching equal keys at the leaf, -1 (all-ones) for a miss (Sec. IV-D).

Every function here is pinned by ``tests/test_oracle.py`` against things
other than itself: ``numpy.searchsorted`` over the sorted keys (the exact
definition of a point lookup), brute force on tiny trees, the closed forms
of Sec. III (N_max, keys per height), structural invariants and hand-worked
fixtures under ``tests/golden/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btree_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)


def compile_oracle(out_path: str = _LIB_PATH, defines: tuple[str, ...] = ()) -> str:
    """Compile btree_oracle.c with gcc into a shared library at out_path."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread"]
    cmd += [f"-D{d}" for d in defines]
    tmp = out_path + ".tmp"
    cmd += ["-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.bto_build.restype = ctypes.c_void_p
    lib.bto_build.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
    lib.bto_free.restype = None
    lib.bto_free.argtypes = [ctypes.c_void_p]
    lib.bto_search.restype = None
    lib.bto_search.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, _u64p, _u8p, _u64p, _i32p]
    lib.bto_search_mt.restype = ctypes.c_int
    lib.bto_search_mt.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, _u64p, _u8p, ctypes.c_int]
    lib.bto_paths.restype = None
    lib.bto_paths.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, _u64p]
    lib.bto_height.restype = ctypes.c_int
    lib.bto_height.argtypes = [ctypes.c_void_p]
    lib.bto_level_nodes.restype = ctypes.c_uint64
    lib.bto_level_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.bto_node_dump.restype = ctypes.c_int
    lib.bto_node_dump.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_int), _u64p, _u64p, _u64p]
    lib.bto_touched.restype = ctypes.c_int
    lib.bto_touched.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, _u64p, _u64p]
    return lib


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the oracle library (compiling it first if it is missing or stale)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        if (not os.path.exists(_LIB_PATH)
                or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
            compile_oracle()
        _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def load_planted(define: str) -> ctypes.CDLL:
    """A copy of the oracle compiled with one planted mistake (pin-strength tests)."""
    d = tempfile.mkdtemp(prefix="oracle_plant_")
    p = compile_oracle(os.path.join(d, f"liboracle_{define}.so"), (define,))
    return load(p)


def _as_u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.uint64, copy=False))


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class OracleTree:
    """Pointer-based CPU B+ tree: bulk load, then one query at a time."""

    def __init__(self, keys, vals, m: int, val_bits: int = 64, lib: ctypes.CDLL | None = None):
        self._lib = lib if lib is not None else load()
        self.m = int(m)
        self.val_bits = int(val_bits)
        k = _as_u64(keys)
        v = _as_u64(vals)
        assert k.shape == v.shape
        self.n = int(k.size)
        self._h = self._lib.bto_build(_ptr(k, _u64p), _ptr(v, _u64p), self.n, self.m, self.val_bits)
        if not self._h:
            raise ValueError("oracle bulk load failed (bad fanout/value width or out of memory)")
        self.miss = (1 << self.val_bits) - 1

    def close(self):
        if self._h:
            self._lib.bto_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def height(self) -> int:
        return int(self._lib.bto_height(self._h))

    def level_nodes(self) -> list[int]:
        return [int(self._lib.bto_level_nodes(self._h, l)) for l in range(self.height)]

    def search(self, queries):
        """Return (values uint64, found uint8, leaf index uint64, slot int32)."""
        q = _as_u64(queries)
        n = q.size
        vals = np.empty(n, np.uint64)
        found = np.empty(n, np.uint8)
        leaf = np.empty(n, np.uint64)
        slot = np.empty(n, np.int32)
        self._lib.bto_search(self._h, _ptr(q, _u64p), n, _ptr(vals, _u64p),
                             _ptr(found, _u8p), _ptr(leaf, _u64p), _ptr(slot, _i32p))
        return vals, found, leaf, slot

    def search_mt(self, queries, nthreads: int):
        """The batch split evenly over nthreads threads (returns values, found)."""
        q = _as_u64(queries)
        n = q.size
        vals = np.empty(n, np.uint64)
        found = np.empty(n, np.uint8)
        rc = self._lib.bto_search_mt(self._h, _ptr(q, _u64p), n, _ptr(vals, _u64p),
                                     _ptr(found, _u8p), int(nthreads))
        if rc != 0:
            raise RuntimeError("oracle thread start failed")
        return vals, found

    def paths(self, queries) -> np.ndarray:
        """Index of the node visited at every level: shape (nq, height)."""
        q = _as_u64(queries)
        h = self.height
        out = np.zeros((q.size, max(h, 1)), np.uint64)
        if h:
            self._lib.bto_paths(self._h, _ptr(q, _u64p), q.size, _ptr(out, _u64p))
        return out[:, :h]

    def node(self, level: int, index: int):
        """(is_leaf, keys, values or None, child indices or None) of one node."""
        is_leaf = ctypes.c_int(0)
        keys = np.zeros(self.m, np.uint64)
        vals = np.zeros(self.m, np.uint64)
        ch = np.zeros(self.m + 1, np.uint64)
        nk = self._lib.bto_node_dump(self._h, level, index, ctypes.byref(is_leaf),
                                     _ptr(keys, _u64p), _ptr(vals, _u64p), _ptr(ch, _u64p))
        if nk < 0:
            raise IndexError((level, index))
        if is_leaf.value:
            return True, keys[:nk].copy(), vals[:nk].copy(), None
        return False, keys[:nk].copy(), None, ch[:nk + 1].copy()

    def touched(self, queries):
        """Distinct nodes per level on the batch's paths, and distinct 32-byte
        value sectors its hits read (leaf values laid out m slots per leaf)."""
        q = _as_u64(queries)
        h = self.height
        counts = np.zeros(max(h, 1), np.uint64)
        sectors = np.zeros(1, np.uint64)
        rc = self._lib.bto_touched(self._h, _ptr(q, _u64p), q.size, _ptr(counts, _u64p),
                                   _ptr(sectors, _u64p))
        if rc != 0:
            raise MemoryError("oracle touched-count allocation failed")
        return [int(c) for c in counts[:h]], int(sectors[0])


def reference_lookup(sorted_keys, vals, queries, val_bits: int = 64):
    """Point lookup by its plain definition: binary search (std::lower_bound)
    over the sorted key array.  Used only to pin the tree oracle."""
    k = _as_u64(sorted_keys)
    v = _as_u64(vals)
    q = _as_u64(queries)
    pos = np.searchsorted(k, q, side="left")
    inb = pos < k.size
    hit = np.zeros(q.size, bool)
    hit[inb] = k[pos[inb]] == q[inb]
    out = np.full(q.size, (1 << val_bits) - 1, np.uint64)
    out[hit] = v[pos[hit]]
    return out, hit.astype(np.uint8)
