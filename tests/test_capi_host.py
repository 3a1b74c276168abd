"""The C ABI without a GPU: library load, exported symbols, host-side trie
construction and CRS compression checked against the oracle and the paper's
storage formulas (Section III, Section V)."""
import re

import numpy as np
import pytest

import oracle
from paper_1702_03657_gb300 import build as B
from paper_1702_03657_gb300 import pm
from paper_1702_03657_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pm.load()


def header_symbols():
    src = open(B.INCLUDE + "/pm.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert "pm_build" in syms and "pm_scan" in syms and "pm_scan_batch" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(pm.EXPORTS) == syms


def test_strerror_and_last_error(lib):
    for code in range(0, -11, -1):
        assert pm.pm_strerror(code) not in ("", "unknown error")
    with pytest.raises(pm.PMError) as e:
        pm.pm_build_host([b"ab", b""])
    assert e.value.code == pm.PM_ERR_EMPTY_PATTERN
    assert pm.pm_last_error() == pm.PM_ERR_EMPTY_PATTERN
    with pytest.raises(pm.PMError) as e:
        pm.pm_build_host([b"x" * (pm.PM_MAX_PATTERN_LEN + 1)])
    assert e.value.code == pm.PM_ERR_PATTERN_TOO_LONG


def csr_walk(row_ptr, col, nxt, fin, text):
    """Pure-Python PFAC walk over exported CRS arrays (tiny inputs)."""
    best_ids, count = [], 0
    for i in range(len(text)):
        v, best, j = 0, -1, i
        while j < len(text):
            r0, r1 = int(row_ptr[v]), int(row_ptr[v + 1])
            hit = [e for e in range(r0, r1) if col[e] == text[j]]
            if not hit:
                break
            v = int(nxt[hit[0]])
            j += 1
            if fin[v] >= 0:
                count += 1
                best = int(fin[v])
        best_ids.append(best)
    return best_ids, count


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi", [
    (0, 2, 20, 1, 7), (1, 4, 60, 2, 9), (2, 26, 80, 3, 12), (3, 256, 100, 1, 6)])
def test_crs_against_oracle(lib, seed, alphabet, npat, lo, hi):
    wl = W.random_case(seed, npat, 3000, alphabet, lo, hi)
    pats = wl.patterns.as_list() + [wl.patterns.get(0)]     # one duplicate
    t = pm.pm_build_host(pats)
    st = pm.pm_stats(t)
    ot = oracle.Trie(pats)
    n, nnz = st["n_nodes"], st["nnz"]
    # trie shape equals the oracle's independent pointer trie
    assert n == ot.n_nodes and nnz == ot.n_edges == n - 1
    assert st["n_patterns"] == len(set(pats)) and st["n_duplicates"] == 1
    assert st["max_len"] == max(map(len, pats)) and st["min_len"] == min(map(len, pats))
    # storage formulas: CRS element count 2nnz+n+1 (Section III); 36-byte
    # bitmapped node and 256-wide state table (Section V)
    assert st["crs_elements"] == 2 * nnz + n + 1
    assert st["csr_bytes"] == 4 * (n + 1) + nnz + 4 * nnz + 4 * n
    assert st["dense256_bytes"] == 256 * 4 * n
    assert st["bitmap36_bytes"] == 36 * n
    row_ptr, col, nxt, fin = pm.pm_export_csr(t)
    # CRS invariants
    assert row_ptr[0] == 0 and row_ptr[-1] == nnz
    assert np.all(np.diff(row_ptr.astype(np.int64)) >= 0)
    for v in range(n):
        r = col[row_ptr[v]:row_ptr[v + 1]].astype(int)
        assert np.all(np.diff(r) > 0)
    # BFS numbering: the e-th non-zero in row order leads to node e+1
    assert np.array_equal(nxt, np.arange(1, nnz + 1))
    assert sorted(np.diff(row_ptr.astype(np.int64)).tolist()) == sorted(ot.degrees().tolist())
    assert int((fin >= 0).sum()) == len(set(pats))
    # walking the exported CRS gives the oracle's answer
    text = wl.text.tobytes()[:600]
    ids, cnt = csr_walk(row_ptr, col, nxt, fin, text)
    o_ids, o_cnt, _ = ot.scan(text)
    assert ids == o_ids.tolist() and cnt == o_cnt


def test_classes_and_dense_levels(lib):
    t = pm.pm_build_host([b"ACGTACGTAC", b"ACGGA" * 3, b"TTTTTTTT"])
    st = pm.pm_stats(t)
    assert st["alphabet"] == 5           # A, C, G, T + any other byte
    assert 0 <= st["dense_k_max"] <= st["min_len"]
    t = pm.pm_build_host([bytes([b]) * 3 for b in range(256)])
    st = pm.pm_stats(t)
    assert st["alphabet"] == 256 and st["dense_k_max"] < st["min_len"]


def _deep_words(cb, d):
    w = -(-(1 << (cb * d)) // 32)
    return w + (w & 1)


def test_deep_level_selection(lib):
    """Byte classes: U used classes take cb = ceil(log2 U) bits; the packed
    filter's depth F is at most the shortest pattern and 20 // cb, the deep
    level's depth D at most the shortest pattern and 26 // cb; the deep level
    is a bitmap with a rank word per 32 packed codes (8 bytes). The byte
    alphabet has no deep level."""
    rng = np.random.Generator(np.random.MT19937(1))

    def pats(alpha, lo, hi, n):
        return [rng.choice(list(alpha), size=int(rng.integers(lo, hi + 1))).astype(np.uint8).tobytes()
                for _ in range(n)]
    # 4 letters (cb = 2), shortest 12: F = 10, D = 12
    st = pm.pm_stats(pm.pm_build_host(pats(b"ACGT", 12, 24, 500)))
    assert (st["alphabet"], st["dense_k_max"], st["deep_k"]) == (5, 10, 12)
    assert st["deep_bytes"] == 8 * _deep_words(2, 12)
    # 3 letters (cb = 2), shortest 14: F = 10, D = 13 (26 bits)
    st = pm.pm_stats(pm.pm_build_host(pats(b"xyz", 14, 20, 300)))
    assert (st["dense_k_max"], st["deep_k"]) == (10, 13)
    assert st["deep_bytes"] == 8 * _deep_words(2, 13)
    # 26 letters (cb = 5), shortest 8: F = 4, D = 5
    st = pm.pm_stats(pm.pm_build_host(pats(b"abcdefghijklmnopqrstuvwxyz", 8, 16, 500)))
    assert (st["dense_k_max"], st["deep_k"]) == (4, 5)
    assert st["deep_bytes"] == 8 * _deep_words(5, 5)
    # shortest pattern below the cb limits: F = D = shortest
    st = pm.pm_stats(pm.pm_build_host(pats(b"ACGT", 6, 12, 200)))
    assert (st["dense_k_max"], st["deep_k"]) == (6, 6)
    # two letters (cb = 1), shortest 30: F = 20, D = 26
    st = pm.pm_stats(pm.pm_build_host(pats(b"ab", 30, 40, 100)))
    assert (st["dense_k_max"], st["deep_k"]) == (20, 26)
    # the byte alphabet: none
    st = pm.pm_stats(pm.pm_build_host([bytes(range(256))] + pats(bytes(range(256)), 20, 30, 50)))
    assert st["alphabet"] == 256 and st["deep_k"] == 0


def test_empty_set_and_host_only_scan(lib):
    t = pm.pm_build_host([])
    st = pm.pm_stats(t)
    assert st["n_nodes"] == 1 and st["nnz"] == 0 and st["n_patterns"] == 0
    import ctypes as C
    res = pm.pm_result(None, None)
    rc = lib.pm_scan(t.handle, None, 0, res, None)
    assert rc == pm.PM_ERR_INVAL or rc == pm.PM_ERR_HOST_ONLY
    cnt = C.c_int64()
    rc = lib.pm_scan_ex(t.handle, None, None, 1, 0, None, C.addressof(cnt), None, None, None)
    assert rc == pm.PM_ERR_HOST_ONLY


def test_config_validation(lib):
    t = pm.pm_build_host([b"hello", b"world"])
    cfg = pm.pm_get_config(t)
    assert 128 <= cfg["threads"] <= 1024 and cfg["threads"] % 32 == 0
    assert cfg["tile"] % (32 * cfg["positions"]) == 0
    assert cfg["deep"] == 1                         # byte classes with a deep level
    pm.pm_set_config(t, cfg)
    for bad in ({"threads": 100}, {"threads": 1056}, {"tile": 1000}, {"dense_k": -1},
                {"stages": 9}, {"dense_k": 99}, {"filter_bits": 16}, {"deep": 2},
                {"positions": 5}, {"positions": 8, "tile": 128}, {"wait_clocks": -1},
                {"light_max": -1}, {"schedule": 3}, {"schedule": -1}, {"positions": 16}):
        c = dict(cfg, **bad)
        with pytest.raises(pm.PMError) as e:
            pm.pm_set_config(t, c)
        assert e.value.code == pm.PM_ERR_INVAL
    tb = pm.pm_build_host([bytes([b, (b + 1) % 256, 7]) for b in range(256)])
    cb = pm.pm_get_config(tb)
    assert pm.pm_stats(tb)["alphabet"] == 256 and cb["deep"] == 0
    # sixteen positions a lane: the default at the byte alphabet's Bloom
    # level (dense_k 2), refused at the other levels
    assert cb["dense_k"] == 2 and cb["positions"] == 16
    for bad in ({"deep": 1}, {"filter_bits": 12}, {"dense_k": 1}, {"positions": 16, "tile": 256}):
        with pytest.raises(pm.PMError):
            pm.pm_set_config(tb, dict(cb, **bad))
    pm.pm_set_config(tb, dict(cb, dense_k=1, positions=8))


def test_scan_all_host_side(lib):
    """Workspace sizing (one u32 per 1024 positions, 256-byte aligned, and a
    bit per position in u32 words, together 256-byte aligned, plus two u64
    per 1024 tiles) and the errors that need no GPU."""
    def r256(x):
        return (x + 255) // 256 * 256
    for n in (0, 1, 31, 32, 33, 1024, 1025, 1024 * 1024, 1024 * 1024 + 1, 1 << 30):
        tiles = -(-n // 1024)
        blocks = -(-tiles // 1024)
        counts_and_bits = r256(r256(4 * tiles) + 4 * -(-n // 32))
        assert pm.pm_scan_all_work_bytes(n) == counts_and_bits + 2 * r256(8 * blocks)
    import ctypes as C
    t = pm.pm_build_host([b"abc"])
    res = pm.pm_result(None, None)
    assert lib.pm_scan_all(None, None, 0, res, None, 0, None, 0, None) == pm.PM_ERR_INVAL
    cnt = C.c_int64()
    res = pm.pm_result(None, C.addressof(cnt))
    assert lib.pm_scan_all(t.handle, None, 0, res, None, 0, None, 0, None) == pm.PM_ERR_HOST_ONLY
    assert lib.pm_scan_all(t.handle, None, 5, res, None, 0, None, 0, None) == pm.PM_ERR_INVAL


def test_scan_all_host_errors(lib):
    import ctypes as C
    t = pm.pm_build_host([b"abc"])
    cnt = C.c_uint64()
    assert lib.pm_scan_all_host(None, None, 0, None, 0, C.byref(cnt)) == pm.PM_ERR_INVAL
    assert lib.pm_scan_all_host(t.handle, None, 0, None, 0, C.byref(cnt)) == pm.PM_ERR_HOST_ONLY
    with pytest.raises(pm.PMError):
        pm.pm_scan_all_host(t, np.zeros(8, np.uint8)[::2], np.zeros((4, 2), np.int64))
    with pytest.raises(pm.PMError):
        pm.pm_scan_all_host(t, np.zeros(8, np.uint8), np.zeros((4, 3), np.int64))


def test_scan_range_host_side(lib):
    import ctypes as C
    t = pm.pm_build_host([b"abc"])
    cnt = C.c_int64()
    res = pm.pm_result(None, C.addressof(cnt))
    assert lib.pm_scan_range(t.handle, None, 5, 3, 10, res, None) == pm.PM_ERR_INVAL
    assert lib.pm_scan_range(t.handle, None, 0, 10, 5, res, None) == pm.PM_ERR_INVAL
    assert lib.pm_scan_range(t.handle, None, 0, 4, 4, res, None) == pm.PM_ERR_INVAL
    assert lib.pm_scan_range(t.handle, None, 3, 3, 3, res, None) == pm.PM_ERR_HOST_ONLY
    assert lib.pm_scan_range(None, None, 3, 3, 3, res, None) == pm.PM_ERR_INVAL


def test_scanner_host_side(lib):
    import ctypes as C
    t = pm.pm_build_host([b"abc"])
    h = C.c_void_p()
    assert lib.pm_scanner_open(t.handle, C.byref(h)) == pm.PM_ERR_HOST_ONLY
    assert lib.pm_scanner_open(None, C.byref(h)) == pm.PM_ERR_INVAL
    assert lib.pm_scanner_push(None, None, 0, None, None, None, None) == pm.PM_ERR_INVAL
    assert lib.pm_scanner_finish(None, None, None, None, None) == pm.PM_ERR_INVAL
    assert lib.pm_scanner_close(None) == pm.PM_OK


def test_autotune_candidates_host(lib):
    """The autotuner's candidates are valid configurations (the library
    accepts each), distinct, span positions per lane, row search, tile and
    CTA size, keep the deep level on where the trie has one, and leave the
    handle's configuration as it was."""
    from paper_1702_03657_gb300 import tune
    rng = np.random.Generator(np.random.MT19937(4))
    pats = [rng.choice(list(b"ACGT"), size=int(rng.integers(14, 21))).astype(np.uint8).tobytes()
            for _ in range(400)]
    t = pm.pm_build_host(pats)
    base = pm.pm_get_config(t)
    for total in (1 << 30, 1 << 16):
        cands = tune.candidates(t, total)
        assert len(cands) >= 20
        assert pm.pm_get_config(t) == base
        seen = set()
        for c in cands:
            pm.pm_set_config(t, c)
            assert c["deep"] == 1 and c["layout"] == 0
            seen.add(tuple(sorted(c.items())))
        assert len(seen) == len(cands)
        for knob in ("positions", "row_search", "tile", "threads", "stages"):
            assert len({c[knob] for c in cands}) >= 2, knob
        if total <= (1 << 16):
            assert min(c["threads"] for c in cands) <= 256
        pm.pm_set_config(t, base)


def test_binding_checks_arguments(lib):
    """The binding refuses host tensors, wrong dtypes, non-contiguous views
    and malformed match buffers before calling into the library."""
    torch = pytest.importorskip("torch")
    t = pm.pm_build_host([b"abc"])
    text = torch.zeros(16, dtype=torch.uint8)
    ids = torch.zeros(16, dtype=torch.int32)
    cnt = torch.zeros(1, dtype=torch.int64)
    for call in (lambda: pm.pm_scan(t, text, ids, cnt),
                 lambda: pm.pm_scan_batch(t, text, torch.zeros(2, dtype=torch.int64), ids, cnt),
                 lambda: pm.pm_scan_all(t, text, ids, cnt, torch.zeros((4, 2), dtype=torch.int64),
                                        torch.zeros(1024, dtype=torch.uint8)),
                 lambda: pm.pm_scan_all(t, text, ids, cnt, torch.zeros(8, dtype=torch.int64),
                                        torch.zeros(1024, dtype=torch.uint8)),
                 lambda: pm.pm_scan_walks(t, text, ids, cnt, cnt)):
        with pytest.raises(pm.PMError) as e:
            call()
        assert e.value.code == pm.PM_ERR_INVAL
    with pytest.raises(pm.PMError):
        pm._dptr(torch.zeros(4, dtype=torch.float32), torch.int32, "ids")
    with pytest.raises(pm.PMError):
        pm._offsets_ptr(torch.zeros(3, dtype=torch.int32))
    # host-buffer entry points: C-contiguous uint8 text, int32 ids
    text_h = np.zeros(64, np.uint8)
    ids_h = np.zeros(64, np.int32)
    for f in (pm.pm_scan_host, pm.pm_scan_host_static):
        for a, b in ((text_h[::2], ids_h[:32]), (text_h, ids_h[::2]),
                     (text_h.astype(np.int8), ids_h), (text_h, ids_h[:10])):
            with pytest.raises(pm.PMError) as e:
                f(t, a, b)
            assert e.value.code == pm.PM_ERR_INVAL


def test_header_constants_match_binding(lib):
    """The binding's copies of pm.h's constants and error codes are the
    header's."""
    src = open(B.INCLUDE + "/pm.h").read()
    defs = {}
    for name, val in re.findall(r"#define[ \t]+(PM_[A-Z_]+)[ \t]+([^\n/]+)", src):
        v = val.strip().replace("ull", "").rstrip("u")
        defs[name] = int(eval(v))
    for name, val in defs.items():
        assert getattr(pm, name) == val, name
    assert "PM_STATIC_MAX_LEN" in defs and "PM_ERR_HOST_ONLY" in defs


def test_server_rejects_host_only_trie(lib):
    t = pm.pm_build_host([b"abc", b"abd"])
    with pytest.raises(pm.PMError) as e:
        pm.pm_server_create(t)
    assert e.value.code == pm.PM_ERR_HOST_ONLY
