"""Pins for the CPU oracle (no GPU).

The oracle is pinned to things other than itself: hand-worked fixtures
(tests/golden), a closed form, special cases that reduce to a library routine
(bytes.find, dict membership), an independent pure-Python brute force on tiny
inputs, and invariants of the trie. Both oracle functions (the definition and
the PFAC pointer-trie walk) must meet every pin.
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_1702_03657_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixtures():
    out = []
    for f in sorted(glob.glob(os.path.join(GOLDEN, "*.json"))):
        with open(f) as fh:
            c = json.load(fh)
        c["patterns"] = [bytes.fromhex(p) for p in c["patterns"]]
        c["text"] = bytes.fromhex(c["text"])
        out.append(pytest.param(c, id=os.path.basename(f)[:-5]))
    return out


def py_brute(pats, text):
    """Independent brute force in pure Python (tiny inputs only): for each
    start position, the longest pattern that text[i:] starts with, the number
    of patterns it starts with, and the depth of the deepest trie prefix."""
    first = {}
    for j, p in enumerate(pats):
        first.setdefault(bytes(p), j)
    lens = sorted({len(p) for p in first}, reverse=True)
    prefixes = {p[:k] for p in first for k in range(1, len(p) + 1)}
    ids, count, look = [], 0, 0
    n = len(text)
    for i in range(n):
        best = -1
        for L in lens:
            s = text[i:i + L]
            if len(s) == L and s in first:
                count += 1
                if best == -1:
                    best = first[s]
        ids.append(best)
        d = 0
        while i + d < n and text[i:i + d + 1] in prefixes:
            d += 1
        look += d + (1 if i + d < n else 0)
    return ids, count, look


def occurrences(p: bytes, text: bytes):
    """All (overlapping) start positions of p in text, by bytes.find."""
    out, s = [], text.find(p)
    while s >= 0:
        out.append(s)
        s = text.find(p, s + 1)
    return out


def both(pats, text):
    a = oracle.naive(pats, text)
    t = oracle.Trie(pats)
    b = t.scan(text)
    return a, b


def both_all(pats, text):
    """The all-matches form by the definition and by the walk, as lists of
    [position, id, length]."""
    out = []
    for pos, ids, lens in (oracle.naive_all(pats, text), oracle.Trie(pats).scan_all(text)):
        out.append([[int(a), int(b), int(c)] for a, b, c in zip(pos, ids, lens)])
    return out


@pytest.mark.parametrize("case", _fixtures())
def test_golden(case):
    a, b = both(case["patterns"], case["text"])
    for ids, cnt, look in (a, b):
        assert ids.tolist() == case["ids"]
        assert cnt == case["count"]
        assert look == case["lookups"]
    for got in both_all(case["patterns"], case["text"]):
        assert got == case["matches"]
        assert len(got) == case["count"]


@pytest.mark.parametrize("m,n", [(1, 1), (3, 4), (5, 3), (7, 40)])
def test_all_matches_closed_form_unary(m, n):
    """P = {a, ..., a^m}, T = a^n: at position i the patterns a^L with
    L = min(m, n-i) down to 1 occur, a^L having id L-1."""
    pats = [b"a" * k for k in range(1, m + 1)]
    exp = [[i, L - 1, L] for i in range(n) for L in range(min(m, n - i), 0, -1)]
    for got in both_all(pats, b"a" * n):
        assert got == exp


def py_brute_all(pats, text):
    """Every occurrence by slicing, in plain Python: distinct patterns keep
    their first index; per position the longer pattern first."""
    first = {}
    for j, p in enumerate(pats):
        first.setdefault(p, j)
    out = []
    for i in range(len(text)):
        hits = sorted((p for p in first if text[i:i + len(p)] == p), key=len, reverse=True)
        out.extend([i, first[p], len(p)] for p in hits)
    return out


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi", [
    (0, 2, 12, 1, 6), (1, 3, 30, 1, 5), (3, 26, 50, 1, 4), (5, 256, 50, 1, 3),
])
def test_all_matches_against_python_brute_force(seed, alphabet, npat, lo, hi):
    wl = W.random_case(seed, npat, 1200, alphabet, lo, hi, plant_rate=0.08)
    pats = wl.patterns.as_list()
    pats = pats + [pats[0], pats[len(pats) // 2][:1]]
    text = wl.text.tobytes()
    exp = py_brute_all(pats, text)
    for got in both_all(pats, text):
        assert got == exp


def test_all_matches_agree_with_scan():
    """The longest-first list starts every matched position with ids[i], has
    count entries, and each entry is an occurrence; thread splits agree."""
    wl = W.random_case(8, 200, 30000, 3, 1, 9, plant_rate=0.1)
    t = oracle.Trie(wl.patterns)
    ids, cnt, _ = t.scan(wl.text)
    pos, mid, lens = t.scan_all(wl.text)
    assert len(pos) == cnt
    assert np.all(np.diff(pos) >= 0)
    text = wl.text.tobytes()
    pats = wl.patterns.as_list()
    firsts = np.r_[True, pos[1:] != pos[:-1]]
    assert np.array_equal(mid[firsts], ids[pos[firsts]])
    assert np.array_equal(np.unique(pos), np.flatnonzero(ids >= 0))
    same = ~firsts
    assert np.all(lens[same] < lens[np.flatnonzero(same) - 1])
    for a, b, c in zip(pos[::97], mid[::97], lens[::97]):
        assert len(pats[b]) == c and text[a:a + c] == pats[b]
    p4 = t.scan_all(wl.text, threads=4)
    assert all(np.array_equal(x, y) for x, y in zip((pos, mid, lens), p4))


@pytest.mark.parametrize("m,n", [(1, 1), (3, 4), (5, 3), (7, 40), (40, 7)])
def test_closed_form_unary(m, n):
    """P = {a, aa, ..., a^m}, T = a^n: every pattern that fits occurs, so
    count = sum_i min(m, n-i) and ids[i] = min(m, n-i) - 1 (a^k has id k-1);
    the walk from i reaches depth min(m, n-i) and attempts one more lookup
    only when it stopped at a leaf before the text's end."""
    pats = [b"a" * k for k in range(1, m + 1)]
    text = b"a" * n
    exp_ids = [min(m, n - i) - 1 for i in range(n)]
    exp_cnt = sum(min(m, n - i) for i in range(n))
    exp_look = sum(min(m, n - i) + (1 if m < n - i else 0) for i in range(n))
    for ids, cnt, look in both(pats, text):
        assert ids.tolist() == exp_ids
        assert cnt == exp_cnt
        assert look == exp_look


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_single_pattern_is_find(seed):
    rng = np.random.Generator(np.random.MT19937(seed))
    text = bytes(rng.integers(97, 100, size=3000, dtype=np.uint8))
    p = bytes(rng.integers(97, 100, size=int(rng.integers(1, 6)), dtype=np.uint8))
    occ = occurrences(p, text)
    exp = np.full(len(text), -1)
    exp[occ] = 0
    for ids, cnt, _ in both([p], text):
        assert np.array_equal(ids, exp)
        assert cnt == len(occ)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equal_length_is_set_membership(seed):
    rng = np.random.Generator(np.random.MT19937(seed))
    k = int(rng.integers(2, 5))
    pats = [bytes(rng.integers(97, 101, size=k, dtype=np.uint8)) for _ in range(30)]
    first = {}
    for j, p in enumerate(pats):
        first.setdefault(p, j)
    text = bytes(rng.integers(97, 101, size=2000, dtype=np.uint8))
    exp = [first.get(text[i:i + k], -1) if i + k <= len(text) else -1
           for i in range(len(text))]
    for ids, cnt, _ in both(pats, text):
        assert ids.tolist() == exp
        assert cnt == sum(e >= 0 for e in exp)


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi", [
    (0, 2, 12, 1, 6), (1, 3, 30, 1, 5), (2, 4, 50, 1, 8),
    (3, 26, 50, 1, 4), (4, 5, 40, 2, 9), (5, 256, 50, 1, 3),
])
def test_against_python_brute_force(seed, alphabet, npat, lo, hi):
    wl = W.random_case(seed, npat, 1500, alphabet, lo, hi, plant_rate=0.08)
    pats = wl.patterns.as_list()
    # a few duplicates and prefixes of existing patterns
    pats = pats + [pats[0], pats[len(pats) // 2][:1]]
    text = wl.text.tobytes()
    exp_ids, exp_cnt, exp_look = py_brute(pats, text)
    for ids, cnt, look in both(pats, text):
        assert ids.tolist() == exp_ids
        assert cnt == exp_cnt
        assert look == exp_look


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_invariants(seed):
    wl = W.random_case(seed, 60, 5000, 4, 1, 7, plant_rate=0.1)
    pats = wl.patterns.as_list()
    text = wl.text.tobytes()
    t = oracle.Trie(pats)
    ids, cnt, look = t.scan(text)
    # total matches = sum over patterns of their occurrence counts
    assert cnt == sum(len(occurrences(p, text)) for p in set(pats))
    # a reported id occurs at its position, and nothing longer does
    for i in np.flatnonzero(ids >= 0):
        p = pats[ids[i]]
        assert text[i:i + len(p)] == p
        assert not any(len(q) > len(p) and text[i:i + len(q)] == q for q in pats)
    assert cnt >= int((ids >= 0).sum())
    # trie shape: one node per distinct non-empty prefix plus the root;
    # a tree has one edge fewer than nodes, and the edges are the out-degrees
    prefixes = {p[:k] for p in pats for k in range(1, len(p) + 1)}
    assert t.n_nodes == 1 + len(prefixes)
    assert t.n_edges == t.n_nodes - 1
    assert int(t.degrees().sum()) == t.n_edges
    assert t.n_nodes - 1 <= sum(len(p) for p in set(pats))
    # every lookup is either a successful step or the walk's last attempt
    assert look >= len(text)


def test_thread_split_and_ranges():
    wl = W.random_case(7, 40, 20000, 3, 1, 6)
    t = oracle.Trie(wl.patterns)
    ids1, c1, l1 = t.scan(wl.text)
    ids4, c4, l4 = t.scan(wl.text, threads=4)
    assert np.array_equal(ids1, ids4) and c1 == c4 and l1 == l4
    a, b = 1234, 17000
    ids_r, _, _ = t.scan(wl.text, a, b)
    assert np.array_equal(ids_r, ids1[a:b])
    nv, _, _ = oracle.naive(wl.patterns, wl.text, a, a + 500)
    assert np.array_equal(nv, ids1[a:a + 500])


def test_batch_no_cross_boundary():
    pats = [b"abc", b"bc", b"c"]
    text = b"ab" + b"cabc"          # texts "ab" and "cabc"
    offsets = [0, 2, 6]
    t = oracle.Trie(pats)
    ids, counts, _ = t.scan_batch(np.frombuffer(text, np.uint8), offsets)
    # in the first text "ab" nothing matches ("abc" would cross the boundary)
    assert ids.tolist() == [-1, -1, 2, 0, 1, 2]
    assert counts.tolist() == [0, 4]


def test_empty_pattern_rejected():
    with pytest.raises(ValueError):
        oracle.naive([b"a", b""], b"abc")
    with pytest.raises(ValueError):
        oracle.Trie([b""])


MUTATIONS = [
    # the deepest final node must win: keep the first (shallowest) instead
    ("best = t->nodes[v].final_id;", "if (best < 0) best = t->nodes[v].final_id;"),
    # a walk that reached a final node must be counted
    ("                ++cnt;\n                best =", "                best ="),
    # the definition must count a repeated pattern once
    ("                if (dup) continue;\n                ++cnt;", "                ++cnt;"),
    # the definition must prefer the longer pattern
    ("if (L > best_len)", "if (best < 0)"),
    # no lookup is attempted once the text has ended
    ("look += deepest + (i + deepest < len ? 1 : 0);", "look += deepest + 1;"),
    ("            ++look;                       /* one lookup", "            /* one lookup"),
]


def _load_mutant(tmp_path, src):
    import ctypes as C
    import subprocess
    c = tmp_path / "m.c"
    so = tmp_path / "m.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared",
                           "-o", str(so), str(c)])
    lib = C.CDLL(str(so))
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    lib.oracle_naive.argtypes = [P, P, i32, P, i64, i64, i64, P, P, P]
    lib.otrie_new.restype = P
    lib.otrie_insert.argtypes = [P, P, i64, i32]
    lib.oracle_pfac.argtypes = [P, P, i64, i64, i64, P, P, P]
    return lib


def _run_mutant(lib, pats, text):
    import ctypes as C
    data, off = oracle._pack(pats)
    t = np.frombuffer(text + b"\0", np.uint8)
    n = len(text)
    res = []
    ids = np.empty(max(n, 1), np.int32)
    cnt, look = C.c_int64(), C.c_int64()
    lib.oracle_naive(data.ctypes.data, off.ctypes.data, len(off) - 1,
                     t.ctypes.data, n, 0, n, ids.ctypes.data,
                     C.byref(cnt), C.byref(look))
    res.append((ids[:n].tolist(), cnt.value, look.value))
    h = lib.otrie_new()
    for j in range(len(off) - 1):
        lib.otrie_insert(h, data.ctypes.data + int(off[j]), int(off[j + 1] - off[j]), j)
    lib.oracle_pfac(h, t.ctypes.data, n, 0, n, ids.ctypes.data,
                    C.byref(cnt), C.byref(look))
    res.append((ids[:n].tolist(), cnt.value, look.value))
    return res


MUTATIONS_ALL = [
    # the walk lists its finals deepest first, not in walk order
    ("for (int32_t a = nf - 1; a >= 0; --a, ++k)", "for (int32_t a = 0; a < nf; ++a, ++k)"),
    # a final's length is the bytes matched from the start
    ("fl[nf] = (int32_t)(j - i);", "fl[nf] = (int32_t)(j - i - 1);"),
    # the definition sorts each position's patterns longest first
    ("off[hit[a - 1] + 1] - off[hit[a - 1]] < L", "off[hit[a - 1] + 1] - off[hit[a - 1]] > L"),
    # the definition lists a repeated pattern once
    ("            if (dup) continue;\n            /* insert", "            /* insert"),
]


@pytest.mark.parametrize("k", range(len(MUTATIONS_ALL)))
def test_all_matches_mutations_are_caught(tmp_path, k):
    """A slip planted in a copy of the all-matches oracle (on the CPU) makes
    at least one hand-worked fixture's match list differ."""
    import ctypes as C
    src = open(oracle._SRC).read()
    old, new = MUTATIONS_ALL[k]
    assert src.count(old) == 1, old
    lib = _load_mutant(tmp_path, src.replace(old, new))
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    lib.oracle_naive_all.argtypes = [P, P, i32, P, i64, i64, i64, P, P, P, i64, P]
    lib.oracle_pfac_all.argtypes = [P, P, i64, i64, i64, P, P, P, i64, P]
    caught = False
    for c in _fixtures():
        case = c.values[0]
        data, off = oracle._pack(case["patterns"])
        text = bytes.fromhex(case["text"]) if isinstance(case["text"], str) else case["text"]
        t = np.frombuffer(text + b"\0", np.uint8)
        n = len(text)
        cap = 64
        pos, mid, lens = (np.zeros(cap, np.int64), np.zeros(cap, np.int32),
                          np.zeros(cap, np.int32))
        m = C.c_int64()
        lib.oracle_naive_all(data.ctypes.data, off.ctypes.data, len(off) - 1, t.ctypes.data,
                             n, 0, n, pos.ctypes.data, mid.ctypes.data, lens.ctypes.data,
                             cap, C.byref(m))
        got = [[int(a), int(b), int(c)] for a, b, c in
               zip(pos[:m.value], mid[:m.value], lens[:m.value])]
        caught |= got != case["matches"]
        h = lib.otrie_new()
        for j in range(len(off) - 1):
            lib.otrie_insert(h, data.ctypes.data + int(off[j]), int(off[j + 1] - off[j]), j)
        lib.oracle_pfac_all(h, t.ctypes.data, n, 0, n, pos.ctypes.data, mid.ctypes.data,
                            lens.ctypes.data, cap, C.byref(m))
        got = [[int(a), int(b), int(c)] for a, b, c in
               zip(pos[:m.value], mid[:m.value], lens[:m.value])]
        caught |= got != case["matches"]
    assert caught, f"all-matches mutation {k} not caught"


@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_mutations_are_caught(tmp_path, k):
    """A plausible slip planted in a copy of the oracle (on the CPU) makes at
    least one hand-worked fixture fail, so the pins are sensitive to it."""
    src = open(oracle._SRC).read()
    old, new = MUTATIONS[k]
    assert src.count(old) == 1, old
    lib = _load_mutant(tmp_path, src.replace(old, new))
    caught = False
    for c in _fixtures():
        case = c.values[0]
        exp = (case["ids"], case["count"], case["lookups"])
        for got in _run_mutant(lib, case["patterns"], case["text"]):
            caught |= got != exp
    assert caught, f"mutation {k} not caught"


def test_property_definition_equals_walk():
    """Random small pattern sets and texts (property-based): the definition
    and the walk agree on ids, count, lookups and the all-matches list, and
    both equal the plain-Python brute force."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    alpha = st.sampled_from([b"ab", b"abc", b"\x00\xff", b"acgt"])

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(alpha.flatmap(lambda a: st.tuples(
        st.lists(st.binary(min_size=1, max_size=6).map(
            lambda b: bytes(a[x % len(a)] for x in b)), min_size=1, max_size=12),
        st.binary(max_size=80).map(lambda b: bytes(a[x % len(a)] for x in b)))))
    def check(case):
        pats, text = case
        exp_ids, exp_cnt, exp_look = py_brute(pats, text)
        for ids, cnt, look in both(pats, text):
            assert ids.tolist() == exp_ids and cnt == exp_cnt and look == exp_look
        exp_all = py_brute_all(pats, text)
        for got in both_all(pats, text):
            assert got == exp_all

    check()
