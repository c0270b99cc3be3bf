"""Python side of the CPU oracle.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The product path (``paper_1712_09494_gb300``)
never does.  ``build()`` compiles ``oracle.cpp`` with the host C++ compiler;
everything else marshals numpy arrays into the C functions, whose header
comments cite the passage each follows.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle into oracle/_build/liboracle.so (plain -O2, one thread)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Model(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_int32), ("P", ctypes.c_int32),
        ("bits", ctypes.c_uint8 * 16),
        ("pc1", ctypes.c_uint8 * 8), ("pc2", ctypes.c_uint8 * 8),
        ("deg", ctypes.c_uint8 * (16 * 32)),
        ("tgt", ctypes.c_uint8 * (16 * 32 * 4)),
        ("lab", ctypes.c_uint8 * (16 * 32 * 4)),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P, U64, U32, VP = ctypes.POINTER, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.orc_new.restype = VP
        lib.orc_new.argtypes = [U64]
        lib.orc_free.argtypes = [VP]
        lib.orc_size.restype = U64
        lib.orc_size.argtypes = [VP]
        lib.orc_find_or_put.argtypes = [VP, VP, U64, VP]
        lib.orc_insert.argtypes = [VP, VP, VP, U64]
        lib.orc_lookup.argtypes = [VP, VP, U64, VP, VP]
        lib.orc_export.restype = U64
        lib.orc_export.argtypes = [VP, VP, VP, U64]
        lib.orc128_new.restype = VP
        lib.orc128_new.argtypes = [U64]
        lib.orc128_free.argtypes = [VP]
        lib.orc128_size.restype = U64
        lib.orc128_size.argtypes = [VP]
        lib.orc128_find_or_put.argtypes = [VP, VP, U64, VP]
        lib.orc128_lookup.argtypes = [VP, VP, U64, VP]
        lib.orc128_export.restype = U64
        lib.orc128_export.argtypes = [VP, VP, U64]
        lib.orclong_new.restype = VP
        lib.orclong_new.argtypes = [U32]
        lib.orclong_free.argtypes = [VP]
        lib.orclong_size.restype = U64
        lib.orclong_size.argtypes = [VP]
        lib.orclong_find_or_put.argtypes = [VP, VP, U64, VP]
        lib.orclong_lookup.argtypes = [VP, VP, U64, VP]
        lib.orclong_export.restype = U64
        lib.orclong_export.argtypes = [VP, VP, U64]
        lib.orc_successors.restype = U64
        lib.orc_successors.argtypes = [P(Model), U64, VP, U64]
        lib.orc_successors128.restype = U64
        lib.orc_successors128.argtypes = [P(Model), U64, U64, VP, U64]
        lib.orc_bfs128.restype = ctypes.c_int
        lib.orc_bfs128.argtypes = [P(Model), U64, U64, U64, U32, VP, VP, VP, U64, P(U32), P(U64)]
        lib.orc_bfs.restype = ctypes.c_int
        lib.orc_bfs.argtypes = [P(Model), U64, U64, U32, VP, VP, VP, U64, P(U32), P(U64)]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _u64(keys):
    return np.ascontiguousarray(np.asarray(keys).astype(np.uint64, copy=False))


class OracleTable128:
    """The plain set definition for 128-bit keys (std::unordered_set of word
    pairs, one thread).  Keys are (n, 2) uint64 arrays: column 0 the low
    word, column 1 the high word."""

    def __init__(self, reserve=0):
        self._lib = _load()
        self._h = self._lib.orc128_new(int(reserve))

    def close(self):
        if self._h:
            self._lib.orc128_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self):
        return int(self._lib.orc128_size(self._h))

    @staticmethod
    def _k(keys):
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64).reshape(-1, 2))
        return k

    def find_or_put(self, keys):
        k = self._k(keys)
        out = np.empty(len(k), dtype=np.uint8)
        self._lib.orc128_find_or_put(self._h, _ptr(k), len(k), _ptr(out))
        return out

    def lookup(self, keys):
        k = self._k(keys)
        found = np.empty(len(k), dtype=np.uint8)
        self._lib.orc128_lookup(self._h, _ptr(k), len(k), _ptr(found))
        return found

    def export(self):
        n = self.size()
        out = np.empty((max(n, 1), 2), dtype=np.uint64)
        got = int(self._lib.orc128_export(self._h, _ptr(out), n))
        return out[:got]


class OracleTableLong:
    """The plain set definition for keys of ``words`` 64-bit words (an
    ordered std::set of word vectors, one thread).  Keys are (n, words)
    uint64 arrays, one key per row."""

    def __init__(self, words):
        self._lib = _load()
        self.words = int(words)
        if self.words < 1:
            raise ValueError("words must be >= 1")
        self._h = self._lib.orclong_new(self.words)

    def close(self):
        if self._h:
            self._lib.orclong_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self):
        return int(self._lib.orclong_size(self._h))

    def _k(self, keys):
        return np.ascontiguousarray(np.asarray(keys).astype(np.uint64, copy=False).reshape(-1, self.words))

    def find_or_put(self, keys):
        k = self._k(keys)
        out = np.empty(len(k), dtype=np.uint8)
        self._lib.orclong_find_or_put(self._h, _ptr(k), len(k), _ptr(out))
        return out

    def lookup(self, keys):
        k = self._k(keys)
        found = np.empty(len(k), dtype=np.uint8)
        self._lib.orclong_lookup(self._h, _ptr(k), len(k), _ptr(found))
        return found

    def export(self):
        n = self.size()
        out = np.empty((max(n, 1), self.words), dtype=np.uint64)
        got = int(self._lib.orclong_export(self._h, _ptr(out), n))
        return out[:got]


class OracleTable:
    """The plain set/map definition (std::unordered_map, one thread)."""

    def __init__(self, reserve=0):
        self._lib = _load()
        self._h = self._lib.orc_new(int(reserve))

    def close(self):
        if self._h:
            self._lib.orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self):
        return int(self._lib.orc_size(self._h))

    def find_or_put(self, keys):
        k = _u64(keys)
        out = np.empty(len(k), dtype=np.uint8)
        self._lib.orc_find_or_put(self._h, _ptr(k), len(k), _ptr(out))
        return out

    def insert(self, keys, values=None):
        k = _u64(keys)
        v = None if values is None else np.ascontiguousarray(np.asarray(values, dtype=np.uint32))
        self._lib.orc_insert(self._h, _ptr(k), _ptr(v), len(k))

    def lookup(self, keys):
        k = _u64(keys)
        found = np.empty(len(k), dtype=np.uint8)
        vals = np.empty(len(k), dtype=np.uint32)
        self._lib.orc_lookup(self._h, _ptr(k), len(k), _ptr(found), _ptr(vals))
        return found, vals

    def export(self):
        n = self.size()
        keys = np.empty(n, dtype=np.uint64)
        vals = np.empty(n, dtype=np.uint32)
        self._lib.orc_export(self._h, _ptr(keys), _ptr(vals), n)
        order = np.argsort(keys, kind="stable")
        return keys[order], vals[order]


def to_ctypes_model(m):
    """Marshal a workloads.statespace.Model into the oracle's struct."""
    s = Model()
    s.C, s.P = int(m.C), int(m.P)
    ctypes.memmove(s.bits, np.ascontiguousarray(m.bits, dtype=np.uint8).ctypes.data, 16)
    c1, c2 = m.pair_arrays()
    ctypes.memmove(s.pc1, c1.ctypes.data, 8)
    ctypes.memmove(s.pc2, c2.ctypes.data, 8)
    ctypes.memmove(s.deg, np.ascontiguousarray(m.deg, dtype=np.uint8).ctypes.data, 16 * 32)
    ctypes.memmove(s.tgt, np.ascontiguousarray(m.tgt, dtype=np.uint8).ctypes.data, 16 * 32 * 4)
    ctypes.memmove(s.lab, np.ascontiguousarray(m.lab, dtype=np.uint8).ctypes.data, 16 * 32 * 4)
    return s


def successors(model, s):
    lib = _load()
    cm = to_ctypes_model(model)
    cap = 256
    out = np.empty(cap, dtype=np.uint64)
    n = lib.orc_successors(ctypes.byref(cm), int(s), _ptr(out), cap)
    if n > cap:
        out = np.empty(int(n), dtype=np.uint64)
        n = lib.orc_successors(ctypes.byref(cm), int(s), _ptr(out), int(n))
    return out[:n]


def successors128(model, s):
    """Successors of a state wider than 64 bits (a Python int): (n, 2)
    uint64 array of (low word, high word)."""
    lib = _load()
    cm = to_ctypes_model(model)
    s = int(s)
    lo, hi = s & (2 ** 64 - 1), s >> 64
    cap = 256
    out = np.empty((cap, 2), dtype=np.uint64)
    n = lib.orc_successors128(ctypes.byref(cm), lo, hi, _ptr(out), cap)
    if n > cap:
        out = np.empty((int(n), 2), dtype=np.uint64)
        n = lib.orc_successors128(ctypes.byref(cm), lo, hi, _ptr(out), int(n))
    return out[:n]


class BfsResult:
    def __init__(self, rc, level_sizes, level_succ, states, total):
        self.rc = rc
        self.level_sizes = level_sizes
        self.level_succ = level_succ
        self.states = states
        self.total = total

    def level(self, d):
        off = int(self.level_sizes[:d].sum())
        return self.states[off:off + int(self.level_sizes[d])]


def bfs(model, max_states=1 << 24, max_levels=4096, keep_states=True, s0=0, wide=False):
    """BFS over the model's reachable states (Section 3.2's open/closed sets).
    wide=True: states as 128-bit vectors, (n, 2) uint64 arrays of (low
    word, high word) -- for models wider than 64 bits."""
    lib = _load()
    cm = to_ctypes_model(model)
    sizes = np.zeros(max_levels, dtype=np.uint64)
    succ = np.zeros(max_levels, dtype=np.uint64)
    cap = int(max_states) + 1 if keep_states else 0
    states = (np.empty((cap, 2) if wide else cap, dtype=np.uint64)) if keep_states else None
    nlev = ctypes.c_uint32(0)
    total = ctypes.c_uint64(0)
    if wide:
        rc = lib.orc_bfs128(ctypes.byref(cm), int(s0) & (2 ** 64 - 1), int(s0) >> 64, int(max_states),
                            int(max_levels), _ptr(sizes), _ptr(succ), _ptr(states), cap, ctypes.byref(nlev),
                            ctypes.byref(total))
    else:
        rc = lib.orc_bfs(ctypes.byref(cm), int(s0), int(max_states), int(max_levels), _ptr(sizes),
                         _ptr(succ), _ptr(states), cap, ctypes.byref(nlev), ctypes.byref(total))
    n = nlev.value
    st = states[:min(int(total.value), cap)] if keep_states else None
    return BfsResult(rc, sizes[:n].astype(np.int64), succ[:n].astype(np.int64), st, int(total.value))
