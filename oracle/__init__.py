"""CPU oracle for the PFAC scan -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package. The product library never calls it and
shares no code with it (the C source here is compiled on its own by gcc).

Functions (all follow the paper's statement of the problem, Sections II-B and
II-C; see ``pfac_oracle.c`` for the exact definitions):

* ``naive(patterns, text, i0, i1)`` -- the definition: every pattern compared
  at every start position. Slow; used as the pin and on sampled positions.
* ``Trie(patterns)`` + ``Trie.scan(text, ...)`` -- the PFAC walk over a plain
  pointer trie (one walk per start position, stop at the first mismatch).

Both return ``(ids int32[n], count, lookups)`` where ``ids[i]`` is the id of
the longest pattern occurring at start position i (-1 if none), ``count`` the
number of (position, pattern) occurrences and ``lookups`` the number of trie
transitions attempted.

The all-matches form, ``naive_all`` and ``Trie.scan_all``, returns every
occurrence as ``(pos int64[m], id int32[m], length int32[m])`` ordered by
position, then the longer pattern first.
"""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes as _C
import os
import subprocess
from typing import List, Sequence, Tuple, Union

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfac_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                           "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = _C.CDLL(build())
    P = _C.c_void_p
    i64, i32 = _C.c_int64, _C.c_int32
    lib.oracle_naive.argtypes = [P, P, i32, P, i64, i64, i64, P, P, P]
    lib.oracle_naive.restype = _C.c_int
    lib.otrie_new.argtypes = []
    lib.otrie_new.restype = P
    lib.otrie_free.argtypes = [P]
    lib.otrie_free.restype = None
    lib.otrie_insert.argtypes = [P, P, i64, i32]
    lib.otrie_insert.restype = _C.c_int
    for f in ("otrie_nodes", "otrie_edges", "otrie_dups", "otrie_max_len"):
        getattr(lib, f).argtypes = [P]
        getattr(lib, f).restype = i64
    lib.otrie_degrees.argtypes = [P, P]
    lib.otrie_degrees.restype = None
    lib.oracle_pfac.argtypes = [P, P, i64, i64, i64, P, P, P]
    lib.oracle_pfac.restype = None
    lib.oracle_naive_all.argtypes = [P, P, i32, P, i64, i64, i64, P, P, P, i64, P]
    lib.oracle_naive_all.restype = _C.c_int
    lib.oracle_pfac_all.argtypes = [P, P, i64, i64, i64, P, P, P, i64, P]
    lib.oracle_pfac_all.restype = _C.c_int
    _lib = lib
    return lib


def _pack(patterns) -> Tuple[np.ndarray, np.ndarray]:
    if hasattr(patterns, "data") and hasattr(patterns, "off"):
        return (np.ascontiguousarray(patterns.data, dtype=np.uint8),
                np.ascontiguousarray(patterns.off, dtype=np.int64))
    pats: List[bytes] = [bytes(p) for p in patterns]
    off = np.zeros(len(pats) + 1, dtype=np.int64)
    np.cumsum([len(p) for p in pats], out=off[1:])
    data = np.frombuffer(b"".join(pats) or b"\0", dtype=np.uint8).copy()
    return data, off


def _text(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        return np.frombuffer(bytes(text) or b"\0", dtype=np.uint8)[:len(text)]
    return np.ascontiguousarray(text, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


def naive(patterns, text, i0: int = 0, i1: int = None):
    """The definition, over start positions [i0, i1)."""
    lib = _load()
    data, off = _pack(patterns)
    t = _text(text)
    n = len(t)
    i1 = n if i1 is None else i1
    ids = np.empty(max(i1 - i0, 0), dtype=np.int32)
    cnt = _C.c_int64(0)
    look = _C.c_int64(0)
    rc = lib.oracle_naive(data.ctypes.data, off.ctypes.data, len(off) - 1,
                          _ptr(t), n, i0, i1, _ptr(ids),
                          _C.byref(cnt), _C.byref(look))
    if rc != 0:
        raise ValueError("empty pattern")
    return ids, cnt.value, look.value


def _all_calls(call):
    """Run an all-matches oracle call twice: count, then fill."""
    n = _C.c_int64(0)
    if call(None, None, None, 0, _C.byref(n)) != 0:
        raise ValueError("empty pattern or out of memory")
    m = n.value
    pos = np.empty(m, dtype=np.int64)
    ids = np.empty(m, dtype=np.int32)
    lens = np.empty(m, dtype=np.int32)
    if m and call(pos.ctypes.data, ids.ctypes.data, lens.ctypes.data, m, _C.byref(n)) != 0:
        raise ValueError("out of memory")
    return pos, ids, lens


def naive_all(patterns, text, i0: int = 0, i1: int = None):
    """Every occurrence by the definition, over start positions [i0, i1)."""
    lib = _load()
    data, off = _pack(patterns)
    t = _text(text)
    n = len(t)
    i1 = n if i1 is None else i1
    return _all_calls(lambda p, d, l, cap, nn: lib.oracle_naive_all(
        data.ctypes.data, off.ctypes.data, len(off) - 1, _ptr(t), n, i0, i1, p, d, l, cap, nn))


class Trie:
    """Plain pointer trie (insertion order ids; duplicates keep the first)."""

    def __init__(self, patterns):
        self._lib = _load()
        self._h = self._lib.otrie_new()
        if not self._h:
            raise MemoryError("otrie_new")
        data, off = _pack(patterns)
        for j in range(len(off) - 1):
            a, b = int(off[j]), int(off[j + 1])
            rc = self._lib.otrie_insert(self._h, data.ctypes.data + a, b - a, j)
            if rc < 0:
                raise ValueError(f"pattern {j}: empty or out of memory")

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.otrie_free(h)

    @property
    def n_nodes(self) -> int:
        return self._lib.otrie_nodes(self._h)

    @property
    def n_edges(self) -> int:
        return self._lib.otrie_edges(self._h)

    @property
    def dups(self) -> int:
        return self._lib.otrie_dups(self._h)

    @property
    def max_len(self) -> int:
        return self._lib.otrie_max_len(self._h)

    def degrees(self) -> np.ndarray:
        deg = np.empty(self.n_nodes, dtype=np.int32)
        self._lib.otrie_degrees(self._h, deg.ctypes.data)
        return deg

    def scan(self, text, i0: int = 0, i1: int = None, threads: int = 1):
        """PFAC walk over start positions [i0, i1), split over ``threads``
        contiguous ranges (ctypes releases the GIL during each call)."""
        t = _text(text)
        n = len(t)
        i1 = n if i1 is None else i1
        m = max(i1 - i0, 0)
        ids = np.empty(m, dtype=np.int32)
        threads = max(1, min(threads, m // 4096 + 1))
        bounds = [i0 + (m * k) // threads for k in range(threads + 1)]

        def part(k):
            a, b = bounds[k], bounds[k + 1]
            cnt = _C.c_int64(0)
            look = _C.c_int64(0)
            self._lib.oracle_pfac(self._h, _ptr(t), n, a, b,
                                  ids.ctypes.data + 4 * (a - i0) if m else None,
                                  _C.byref(cnt), _C.byref(look))
            return cnt.value, look.value

        if threads == 1:
            res = [part(0)]
        else:
            with _cf.ThreadPoolExecutor(threads) as ex:
                res = list(ex.map(part, range(threads)))
        return ids, sum(r[0] for r in res), sum(r[1] for r in res)

    def scan_all(self, text, i0: int = 0, i1: int = None, threads: int = 1):
        """Every occurrence by the PFAC walk over start positions [i0, i1),
        split over ``threads`` contiguous ranges."""
        t = _text(text)
        n = len(t)
        i1 = n if i1 is None else i1
        m = max(i1 - i0, 0)
        threads = max(1, min(threads, m // 4096 + 1))
        bounds = [i0 + (m * k) // threads for k in range(threads + 1)]

        def part(k):
            a, b = bounds[k], bounds[k + 1]
            return _all_calls(lambda p, d, l, cap, nn: self._lib.oracle_pfac_all(
                self._h, _ptr(t), n, a, b, p, d, l, cap, nn))

        if threads == 1:
            res = [part(0)]
        else:
            with _cf.ThreadPoolExecutor(threads) as ex:
                res = list(ex.map(part, range(threads)))
        return tuple(np.concatenate([r[j] for r in res]) for j in range(3))

    def scan_batch(self, text, offsets, threads: int = 1):
        """Scan each text text[offsets[k]:offsets[k+1]] on its own (no match
        crosses a text boundary). Returns (ids concatenated, counts[ntexts],
        lookups)."""
        t = _text(text)
        off = np.asarray(offsets, dtype=np.int64)
        ids = np.empty(len(t), dtype=np.int32)
        counts = np.zeros(len(off) - 1, dtype=np.int64)
        look = 0
        for k in range(len(off) - 1):
            a, b = int(off[k]), int(off[k + 1])
            i, c, l = self.scan(t[a:b], threads=threads)
            ids[a:b] = i
            counts[k] = c
            look += l
        return ids, counts, look
