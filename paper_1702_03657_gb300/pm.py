"""Thin ctypes binding of libpm (include/pm.h), same names as the C ABI.

Argument marshalling only: torch tensors give device pointers and streams;
every step of a scan runs in libpm's CUDA kernels. There is no CPU fallback:
if libpm.so is missing or a call fails, a ``PMError`` is raised.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

PM_OK = 0
PM_ERR_INVAL = -1
PM_ERR_NOMEM = -2
PM_ERR_EMPTY_PATTERN = -3
PM_ERR_PATTERN_TOO_LONG = -4
PM_ERR_CUDA = -5
PM_ERR_TIMEOUT = -6
PM_ERR_BOUNDS = -7
PM_ERR_BUSY = -8
PM_ERR_NOT_FOUND = -9
PM_ERR_HOST_ONLY = -10
PM_MAX_PATTERN_LEN = 4096
PM_STATIC_MAX_LEN = 1 << 20
PM_SCHED_AUTO = 0
PM_SCHED_STATIC = 1
PM_SCHED_DYNAMIC = 2
PM_CHUNK_TILES = 32

# every symbol include/pm.h declares (checked by the tests)
EXPORTS = (
    "pm_build", "pm_build_host", "pm_free", "pm_stats", "pm_export_csr",
    "pm_get_config", "pm_set_config", "pm_scan", "pm_scan_batch", "pm_scan_ex",
    "pm_scan_host", "pm_scan_host_static", "pm_device_error", "pm_strerror", "pm_last_error",
    "pm_last_error_msg", "pm_server_create", "pm_submit", "pm_poll", "pm_wait",
    "pm_server_get_stats", "pm_server_destroy", "pm_server_replay", "pm_replay_plain",
    "pm_scan_all", "pm_scan_all_work_bytes", "pm_scan_walks", "pm_scan_range",
    "pm_scan_all_host",
    "pm_scanner_open", "pm_scanner_push", "pm_scanner_finish", "pm_scanner_close",
)


class PMError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {code} ({msg})")


class pm_result(C.Structure):
    _fields_ = [("ids", C.c_void_p), ("count", C.c_void_p)]


class pm_trie_stats(C.Structure):
    _fields_ = [
        ("n_patterns", C.c_uint64), ("n_duplicates", C.c_uint64),
        ("n_nodes", C.c_uint64), ("nnz", C.c_uint64),
        ("min_len", C.c_uint32), ("max_len", C.c_uint32),
        ("alphabet", C.c_uint32), ("dense_k_max", C.c_uint32),
        ("crs_elements", C.c_uint64), ("csr_bytes", C.c_uint64),
        ("dense256_bytes", C.c_uint64), ("bitmap36_bytes", C.c_uint64),
        ("device_bytes", C.c_uint64), ("deep_bytes", C.c_uint64),
        ("deep_k", C.c_uint32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pm_server_config(C.Structure):
    _fields_ = [("arena_bytes", C.c_uint64), ("max_inflight", C.c_uint32),
                ("max_batch", C.c_uint32), ("max_batch_bytes", C.c_uint64),
                ("max_queue", C.c_uint32)]


class pm_server_stats(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in (
        "submitted", "completed", "batches", "bytes", "max_batch_seen",
        "max_inflight_seen", "admission_waits")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pm_config(C.Structure):
    _fields_ = [(f, C.c_int32) for f in (
        "threads", "tile", "dense_k", "filter_bits", "row_search",
        "ctas_per_sm", "stages", "checked", "positions", "deep", "layout",
        "wait_clocks", "light_max", "schedule")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    @staticmethod
    def from_dict(d):
        c = pm_config()
        for f, _ in pm_config._fields_:
            setattr(c, f, int(d[f]))
        return c


_lib = None


def load(path: Optional[str] = None):
    """Load libpm.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise PMError(PM_ERR_CUDA, "load", f"{path} missing: run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32
    sig = {
        "pm_build": ([P, P, u32, P, P], C.c_int),
        "pm_build_host": ([P, P, u32, P, P], C.c_int),
        "pm_free": ([P], None),
        "pm_stats": ([P, P], C.c_int),
        "pm_export_csr": ([P, P, P, P, P], C.c_int),
        "pm_get_config": ([P, P], C.c_int),
        "pm_set_config": ([P, P], C.c_int),
        "pm_scan": ([P, P, u64, pm_result, P], C.c_int),
        "pm_scan_batch": ([P, P, P, u32, P, P, P], C.c_int),
        "pm_scan_ex": ([P, P, P, u32, u64, P, P, P, P, P], C.c_int),
        "pm_scan_host": ([P, P, u64, P, P], C.c_int),
        "pm_scan_host_static": ([P, P, u64, P, P, P], C.c_int),
        "pm_device_error": ([P], C.c_int),
        "pm_strerror": ([C.c_int], C.c_char_p),
        "pm_last_error": ([], C.c_int),
        "pm_last_error_msg": ([], C.c_char_p),
        "pm_server_create": ([P, P, P], C.c_int),
        "pm_submit": ([P, P, u64, pm_result, P], C.c_int),
        "pm_poll": ([P, u64, P], C.c_int),
        "pm_wait": ([P, u64, u32], C.c_int),
        "pm_server_get_stats": ([P, P], C.c_int),
        "pm_server_destroy": ([P], C.c_int),
        "pm_server_replay": ([P, u32, P, P, P, P, P, P, P], C.c_int),
        "pm_replay_plain": ([P, u32, P, P, P, P, P, P, P, P, P], C.c_int),
        "pm_scan_all": ([P, P, u64, pm_result, P, u64, P, u64, P], C.c_int),
        "pm_scan_all_work_bytes": ([u64], u64),
        "pm_scan_walks": ([P, P, u64, P, P, P, P, P], C.c_int),
        "pm_scan_range": ([P, P, u64, u64, u64, pm_result, P], C.c_int),
        "pm_scan_all_host": ([P, P, u64, P, u64, P], C.c_int),
        "pm_scanner_open": ([P, P], C.c_int),
        "pm_scanner_push": ([P, P, u64, P, P, P, P], C.c_int),
        "pm_scanner_finish": ([P, P, P, P, P], C.c_int),
        "pm_scanner_close": ([P], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != PM_OK:
        msg = _lib.pm_last_error_msg().decode(errors="replace")
        raise PMError(rc, where, msg or _lib.pm_strerror(rc).decode())


def _pattern_arrays(patterns):
    """(keepalive, ptr array, lengths) for a PatternSet or a list of bytes."""
    if hasattr(patterns, "data") and hasattr(patterns, "off"):
        data = np.ascontiguousarray(patterns.data, dtype=np.uint8)
        off = np.asarray(patterns.off, dtype=np.int64)
    else:
        pats = [bytes(p) for p in patterns]
        off = np.zeros(len(pats) + 1, dtype=np.int64)
        np.cumsum([len(p) for p in pats], out=off[1:])
        data = np.frombuffer(b"".join(pats) + b"\0", dtype=np.uint8).copy()
    n = len(off) - 1
    if data.size == 0:
        data = np.zeros(1, np.uint8)
    base = data.ctypes.data
    ptrs = (C.c_void_p * max(n, 1))(*[base + int(o) for o in off[:-1]])
    lens = np.ascontiguousarray(np.diff(off), dtype=np.uint32)
    return (data, ptrs, lens), ptrs, lens, n


class Trie:
    """Owns a pm_trie handle; freed with pm_free."""

    def __init__(self, handle, footprint):
        self.handle = handle
        self.footprint = footprint

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.pm_free(h)

    @property
    def _as_parameter_(self):
        return self.handle


def pm_build(patterns, host_only: bool = False) -> Trie:
    lib = load()
    keep, ptrs, lens, n = _pattern_arrays(patterns)
    h = C.c_void_p()
    fp = C.c_uint64()
    fn = lib.pm_build_host if host_only else lib.pm_build
    _check(fn(ptrs, lens.ctypes.data if n else None, n, C.byref(h), C.byref(fp)),
           "pm_build_host" if host_only else "pm_build")
    return Trie(h.value, fp.value)


def pm_build_host(patterns) -> Trie:
    return pm_build(patterns, host_only=True)


def pm_free(trie: Trie):
    h, trie.handle = trie.handle, None
    if h:
        load().pm_free(h)


def pm_stats(trie: Trie) -> dict:
    s = pm_trie_stats()
    _check(load().pm_stats(trie.handle, C.byref(s)), "pm_stats")
    return s.as_dict()


def pm_export_csr(trie: Trie):
    st = pm_stats(trie)
    n, nnz = st["n_nodes"], st["nnz"]
    row_ptr = np.empty(n + 1, np.uint32)
    col = np.empty(max(nnz, 1), np.uint8)
    nxt = np.empty(max(nnz, 1), np.int32)
    fin = np.empty(n, np.int32)
    _check(load().pm_export_csr(trie.handle, row_ptr.ctypes.data, col.ctypes.data,
                                nxt.ctypes.data, fin.ctypes.data), "pm_export_csr")
    return row_ptr, col[:nnz], nxt[:nnz], fin


def pm_get_config(trie: Trie) -> dict:
    c = pm_config()
    _check(load().pm_get_config(trie.handle, C.byref(c)), "pm_get_config")
    return c.as_dict()


def pm_set_config(trie: Trie, cfg: dict):
    c = pm_config.from_dict(cfg)
    _check(load().pm_set_config(trie.handle, C.byref(c)), "pm_set_config")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise PMError(PM_ERR_INVAL, name, "must be a CUDA tensor")
    if not t.is_contiguous():
        raise PMError(PM_ERR_INVAL, name, "must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise PMError(PM_ERR_INVAL, name, f"dtype {t.dtype}, expected {dtype}")
    return t.data_ptr() if t.numel() else None


def _offsets_ptr(offsets):
    if offsets.element_size() != 8:
        raise PMError(PM_ERR_INVAL, "offsets", "must be 64-bit (int64 or uint64)")
    return _dptr(offsets, None, "offsets")


def pm_scan(trie: Trie, text, ids, count, stream=None, length: Optional[int] = None):
    """Scan one device text (uint8 tensor) into ids (int32[len]) and count
    (int64[1]) on `stream` (default: torch's current stream)."""
    import torch
    n = text.numel() if length is None else length
    out = pm_result(_dptr(ids, torch.int32, "ids"), _dptr(count, torch.int64, "count"))
    _check(load().pm_scan(trie.handle, _dptr(text, torch.uint8, "text"), n, out,
                          _stream_ptr(stream)), "pm_scan")


def pm_scan_range(trie: Trie, text, start: int, end: int, limit: int, ids, count,
                  stream=None):
    """Scan start positions [start, end) of a device text (uint8 tensor of at
    least `limit` bytes) whose walks may read up to `limit`; ids
    (int32[end - start]) and count (int64[1])."""
    import torch
    if limit > text.numel():
        raise PMError(PM_ERR_INVAL, "pm_scan_range", "limit beyond the text tensor")
    out = pm_result(_dptr(ids, torch.int32, "ids"), _dptr(count, torch.int64, "count"))
    _check(load().pm_scan_range(trie.handle, _dptr(text, torch.uint8, "text"), start, end,
                                limit, out, _stream_ptr(stream)), "pm_scan_range")


def pm_scan_walks(trie: Trie, text, ids, count, walks, cfg: Optional[dict] = None,
                  stream=None, length: Optional[int] = None):
    """pm_scan that also counts the walks queued into `walks` (int64[1])."""
    import torch
    n = text.numel() if length is None else length
    c = pm_config.from_dict(cfg) if cfg is not None else None
    _check(load().pm_scan_walks(trie.handle, _dptr(text, torch.uint8, "text"), n,
                                _dptr(ids, torch.int32, "ids"), _dptr(count, torch.int64, "count"),
                                _dptr(walks, torch.int64, "walks"),
                                C.byref(c) if c is not None else None, _stream_ptr(stream)),
           "pm_scan_walks")


PM_MATCH_BYTES = 16  # pm_match: u64 pos, i32 id, i32 len


def pm_scan_all_work_bytes(length: int) -> int:
    return int(load().pm_scan_all_work_bytes(length))


def pm_scan_all(trie: Trie, text, ids, count, matches, work, stream=None,
                length: Optional[int] = None):
    """pm_scan plus every occurrence: `matches` is an int64 CUDA tensor of
    shape [capacity, 2] holding pm_match records (see decode_matches);
    `work` a uint8 CUDA tensor of at least pm_scan_all_work_bytes(len)
    bytes (torch allocations are 256-byte aligned)."""
    import torch
    n = text.numel() if length is None else length
    if matches.dtype != torch.int64 or matches.dim() != 2 or matches.shape[1] != 2:
        raise PMError(PM_ERR_INVAL, "matches", "must be an int64 tensor of shape [capacity, 2]")
    out = pm_result(_dptr(ids, torch.int32, "ids"), _dptr(count, torch.int64, "count"))
    _check(load().pm_scan_all(trie.handle, _dptr(text, torch.uint8, "text"), n, out,
                              _dptr(matches, torch.int64, "matches"), matches.shape[0],
                              _dptr(work, torch.uint8, "work"), work.numel(),
                              _stream_ptr(stream)), "pm_scan_all")


def pm_scan_all_host(trie: Trie, text: np.ndarray, matches: np.ndarray) -> int:
    """Every occurrence in a host text (uint8 numpy, ideally pinned), listed
    into `matches` (a C-contiguous int64 numpy array of shape [capacity, 2]
    holding pm_match records, see decode_matches); returns the total count
    (the list stops after `capacity` records)."""
    if text.dtype != np.uint8 or not text.flags.c_contiguous:
        raise PMError(PM_ERR_INVAL, "pm_scan_all_host", "text must be C-contiguous uint8")
    if matches.dtype != np.int64 or matches.ndim != 2 or matches.shape[1] != 2 or \
            not matches.flags.c_contiguous or not matches.flags.writeable:
        raise PMError(PM_ERR_INVAL, "pm_scan_all_host",
                      "matches must be a writeable C-contiguous int64 array [capacity, 2]")
    cnt = C.c_uint64()
    _check(load().pm_scan_all_host(trie.handle, text.ctypes.data if text.size else None,
                                   text.size, matches.ctypes.data if matches.size else None,
                                   matches.shape[0], C.byref(cnt)), "pm_scan_all_host")
    return cnt.value


def decode_matches(matches, m: int):
    """(pos int64[m], id int32[m], length int32[m]) from the first m pm_match
    records of an int64 [capacity, 2] tensor."""
    a = matches[:m]
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    hi = a[:, 1].view(np.uint64)
    return (a[:, 0].copy(), (hi & 0xFFFFFFFF).astype(np.uint32).view(np.int32),
            (hi >> 32).astype(np.uint32).view(np.int32))


class Scanner:
    """A stream of chunks scanned as one text (pm_scanner_*): each push
    returns how many ids it wrote (the positions it resolved, in order)."""

    def __init__(self, trie: Trie):
        h = C.c_void_p()
        _check(load().pm_scanner_open(trie.handle, C.byref(h)), "pm_scanner_open")
        self.handle = h.value
        self.trie = trie  # keeps the trie alive

    def push(self, chunk, ids, count, stream=None, length: Optional[int] = None) -> int:
        import torch
        n = chunk.numel() if length is None else length
        k = C.c_uint64()
        _check(_lib.pm_scanner_push(self.handle, _dptr(chunk, torch.uint8, "chunk"), n,
                                    _dptr(ids, torch.int32, "ids"),
                                    _dptr(count, torch.int64, "count"), C.byref(k),
                                    _stream_ptr(stream)), "pm_scanner_push")
        return k.value

    def finish(self, ids, count, stream=None) -> int:
        import torch
        k = C.c_uint64()
        _check(_lib.pm_scanner_finish(self.handle, _dptr(ids, torch.int32, "ids"),
                                      _dptr(count, torch.int64, "count"), C.byref(k),
                                      _stream_ptr(stream)), "pm_scanner_finish")
        return k.value

    def close(self):
        h, self.handle = self.handle, None
        if h:
            _check(_lib.pm_scanner_close(h), "pm_scanner_close")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pm_scanner_open(trie: Trie) -> Scanner:
    return Scanner(trie)


def pm_scan_batch(trie: Trie, texts, offsets, ids, counts, stream=None):
    import torch
    ntexts = offsets.numel() - 1
    _check(load().pm_scan_batch(
        trie.handle, _dptr(texts, torch.uint8, "texts"),
        _offsets_ptr(offsets),
        ntexts, _dptr(ids, torch.int32, "ids"), _dptr(counts, torch.int64, "counts"),
        _stream_ptr(stream)), "pm_scan_batch")


def pm_scan_ex(trie: Trie, texts, offsets, ids, counts, lookups=None,
               cfg: Optional[dict] = None, stream=None, length: Optional[int] = None):
    import torch
    ntexts = offsets.numel() - 1 if offsets is not None else 1
    n = texts.numel() if length is None else length
    c = pm_config.from_dict(cfg) if cfg is not None else None
    _check(load().pm_scan_ex(
        trie.handle, _dptr(texts, torch.uint8, "texts"),
        _offsets_ptr(offsets) if offsets is not None else None,
        ntexts, n, _dptr(ids, torch.int32, "ids"), _dptr(counts, torch.int64, "counts"),
        _dptr(lookups, None, "lookups") if lookups is not None else None,
        C.byref(c) if c is not None else None, _stream_ptr(stream)), "pm_scan_ex")


def _host_arrays(text: np.ndarray, ids: np.ndarray, where: str):
    """Checks a host text (uint8) and id buffer (int32): both C-contiguous,
    ids at least as long as the text (the C ABI reads and writes them as
    flat arrays)."""
    if text.dtype != np.uint8 or ids.dtype != np.int32:
        raise PMError(PM_ERR_INVAL, where, "text must be uint8 and ids int32")
    if not (text.flags.c_contiguous and ids.flags.c_contiguous):
        raise PMError(PM_ERR_INVAL, where, "text and ids must be C-contiguous")
    if not ids.flags.writeable:
        raise PMError(PM_ERR_INVAL, where, "ids must be writeable")
    if ids.size < text.size:
        raise PMError(PM_ERR_INVAL, where, "ids shorter than the text")


def pm_scan_host(trie: Trie, text: np.ndarray, ids: np.ndarray) -> int:
    """Scan a host text (uint8 numpy, ideally pinned) into host ids (int32);
    returns the count."""
    _host_arrays(text, ids, "pm_scan_host")
    cnt = C.c_int64()
    _check(load().pm_scan_host(trie.handle, text.ctypes.data if text.size else None,
                               text.size, ids.ctypes.data if ids.size else None,
                               C.byref(cnt)), "pm_scan_host")
    return cnt.value


def pm_scan_host_static(trie: Trie, text: np.ndarray, ids: np.ndarray, stream=None) -> int:
    """pm_scan_host without any device allocation (text <= PM_STATIC_MAX_LEN
    bytes, staged in libpm's static device array); returns the count."""
    _host_arrays(text, ids, "pm_scan_host_static")
    cnt = C.c_int64()
    _check(load().pm_scan_host_static(trie.handle, text.ctypes.data if text.size else None,
                                      text.size, ids.ctypes.data if ids.size else None,
                                      C.byref(cnt), _stream_ptr(stream)), "pm_scan_host_static")
    return cnt.value


class Server:
    """Owns a pm_server handle (destroyed with pm_server_destroy)."""

    def __init__(self, handle, trie):
        self.handle = handle
        self.trie = trie  # the trie must outlive the server

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.pm_server_destroy(h)


def pm_server_create(trie: Trie, arena_bytes=0, max_inflight=0, max_batch=0,
                     max_batch_bytes=0, max_queue=0) -> Server:
    cfg = pm_server_config(arena_bytes, max_inflight, max_batch, max_batch_bytes, max_queue)
    h = C.c_void_p()
    _check(load().pm_server_create(trie.handle, C.byref(cfg), C.byref(h)), "pm_server_create")
    return Server(h.value, trie)


def pm_submit(srv: Server, h_text: np.ndarray, ids, count) -> int:
    """Queue a host text (numpy uint8, kept alive and unchanged by the caller
    until done) with device outputs ids (int32[len]) and count (int64[1])."""
    import torch
    rid = C.c_uint64()
    out = pm_result(_dptr(ids, torch.int32, "ids"), _dptr(count, torch.int64, "count"))
    _check(load().pm_submit(srv.handle, h_text.ctypes.data if h_text.size else None,
                            h_text.size, out, C.byref(rid)), "pm_submit")
    return rid.value


def pm_poll(srv: Server, req_id: int) -> bool:
    done = C.c_int()
    _check(load().pm_poll(srv.handle, req_id, C.byref(done)), "pm_poll")
    return bool(done.value)


def pm_wait(srv: Server, req_id: int, timeout_ms: int = 10000):
    _check(load().pm_wait(srv.handle, req_id, timeout_ms), "pm_wait")


def pm_server_get_stats(srv: Server) -> dict:
    st = pm_server_stats()
    _check(load().pm_server_get_stats(srv.handle, C.byref(st)), "pm_server_get_stats")
    return st.as_dict()


def pm_server_destroy(srv: Server):
    h, srv.handle = srv.handle, None
    if h:
        _check(load().pm_server_destroy(h), "pm_server_destroy")


def _ptr_array(ptrs):
    return (C.c_void_p * max(len(ptrs), 1))(*ptrs)


def pm_server_replay(srv: Server, h_ptrs, lens, arrival_ns, id_ptrs, count_ptrs):
    """Native trace replay; returns (latency_ns array, wall_ns)."""
    n = len(lens)
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    lat = np.zeros(n, dtype=np.uint64)
    wall = C.c_uint64()
    _check(load().pm_server_replay(srv.handle, n, _ptr_array(h_ptrs), lens.ctypes.data,
                                   arr.ctypes.data, _ptr_array(id_ptrs),
                                   _ptr_array(count_ptrs), lat.ctypes.data, C.byref(wall)),
           "pm_server_replay")
    return lat, wall.value


def pm_replay_plain(trie: Trie, h_ptrs, lens, arrival_ns, text_ptrs, id_ptrs, count_ptrs,
                    stream=None):
    n = len(lens)
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    lat = np.zeros(n, dtype=np.uint64)
    wall = C.c_uint64()
    _check(load().pm_replay_plain(trie.handle, n, _ptr_array(h_ptrs), lens.ctypes.data,
                                  arr.ctypes.data, _ptr_array(text_ptrs), _ptr_array(id_ptrs),
                                  _ptr_array(count_ptrs), lat.ctypes.data, C.byref(wall),
                                  _stream_ptr(stream)), "pm_replay_plain")
    return lat, wall.value


def pm_device_error() -> int:
    code = C.c_int()
    _check(load().pm_device_error(C.byref(code)), "pm_device_error")
    return code.value


def pm_strerror(code: int) -> str:
    return load().pm_strerror(code).decode()


def pm_last_error() -> int:
    return load().pm_last_error()
