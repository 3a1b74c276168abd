"""All-matches listing (pm_scan_all) on the GPU against the oracle.

Integer output, so bit-exact: every (position, pattern id, length) record,
in the oracle's order (position ascending, longer pattern first), the total
count, and the longest-match ids.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1702_03657_gb300 import pm
from paper_1702_03657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03657_gb300 import build as B
    B.build()
    pm.load()
    yield
    torch.cuda.synchronize()
    assert pm.pm_device_error() == 0


def gpu_all(trie, text: np.ndarray, capacity=None):
    n = len(text)
    tv = torch.from_numpy(np.array(text, dtype=np.uint8)).cuda() if n else \
        torch.zeros(1, dtype=torch.uint8, device="cuda")
    ids = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    cap = capacity if capacity is not None else max(n * 4, 16)
    m = torch.full((max(cap, 1), 2), -9, dtype=torch.int64, device="cuda")
    work = torch.empty(max(pm.pm_scan_all_work_bytes(n), 1), dtype=torch.uint8, device="cuda")
    pm.pm_scan_all(trie, tv, ids, cnt, m[:cap] if cap else m[:0], work, length=n)
    torch.cuda.synchronize()
    c = int(cnt.item())
    got = pm.decode_matches(m, min(c, cap))
    return ids[:n].cpu().numpy(), c, got


def assert_all_same(got, exp):
    for g, e, name in zip(got, exp, ("pos", "id", "len")):
        assert len(g) == len(e), f"{name}: {len(g)} vs {len(e)}"
        bad = np.flatnonzero(g != e)
        assert bad.size == 0, f"{name}: first mismatch at {bad[:5]}"


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi,n", [
    (0, 2, 20, 1, 7, 30_001), (1, 4, 300, 2, 12, 65_537), (2, 26, 300, 3, 16, 100_000),
    (3, 256, 500, 1, 8, 99_999), (4, 4, 2000, 12, 24, 150_001),
])
def test_all_matches_small(seed, alphabet, npat, lo, hi, n):
    wl = W.random_case(seed, npat, n, alphabet, lo, hi, plant_rate=0.05)
    t = pm.pm_build(wl.patterns)
    ot = oracle.Trie(wl.patterns)
    exp = ot.scan_all(wl.text)
    o_ids, o_cnt, _ = ot.scan(wl.text)
    ids, cnt, got = gpu_all(t, wl.text)
    assert cnt == o_cnt == len(exp[0])
    assert np.array_equal(ids, o_ids)
    assert_all_same(got, exp)


def test_nested_patterns_and_edges():
    pats = [b"a" * k for k in range(1, 40)] + [b"ab", b"b"]
    text = np.frombuffer(b"a" * 5000 + b"ab" + b"x" * 3 + b"a" * 70, np.uint8)
    t = pm.pm_build(pats)
    exp = oracle.Trie(pats).scan_all(text)
    ids, cnt, got = gpu_all(t, text, capacity=len(exp[0]))
    assert cnt == len(exp[0])
    assert_all_same(got, exp)
    # a list cut at the capacity keeps the order's first entries
    for cap in (0, 1, 7, 1000, cnt - 1):
        _, cnt2, got2 = gpu_all(t, text, capacity=cap)
        assert cnt2 == cnt
        assert_all_same(got2, tuple(e[:cap] for e in exp))
    # empty text, and a text without matches
    _, c0, g0 = gpu_all(t, np.zeros(0, np.uint8))
    assert c0 == 0 and len(g0[0]) == 0
    _, c1, g1 = gpu_all(t, np.frombuffer(b"xyz" * 999, np.uint8))
    assert c1 == 0 and len(g1[0]) == 0


def test_workspace_checks():
    t = pm.pm_build([b"abc"])
    n = 10_000
    tv = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    m = torch.empty((16, 2), dtype=torch.int64, device="cuda")
    need = pm.pm_scan_all_work_bytes(n)
    small = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_scan_all(t, tv, ids, cnt, m, small)
    assert e.value.code == pm.PM_ERR_INVAL
    big = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_scan_all(t, tv, ids, cnt, m, big[1:])   # not 256-byte aligned
    assert e.value.code == pm.PM_ERR_INVAL


def test_paper_scale_reduced_all():
    """6 MiB (two blocks of 4096 tiles) of the paper-scale workload."""
    wl = W.paper_scale(1, text_bytes=6 * W.MiB + 13)
    t = pm.pm_build(wl.patterns)
    ot = oracle.Trie(wl.patterns)
    exp = ot.scan_all(wl.text, threads=8)
    ids, cnt, got = gpu_all(t, wl.text, capacity=len(exp[0]) + 10)
    assert cnt == len(exp[0])
    assert_all_same(got, exp)


def test_acgt_reduced_all():
    """Dense matches: 4 MiB of the ACGT workload (about one position in a
    hundred starts a pattern, most 32-position words hold one), every record
    against the oracle's list; then the same through pm_scan_all_host."""
    wl = W.acgt(2, text_bytes=4 * W.MiB + 29, n_patterns=100_000)
    t = pm.pm_build(wl.patterns)
    exp = oracle.Trie(wl.patterns).scan_all(wl.text, threads=8)
    assert len(exp[0]) > 20_000
    ids, cnt, got = gpu_all(t, wl.text, capacity=len(exp[0]) + 10)
    assert cnt == len(exp[0])
    assert_all_same(got, exp)
    # a capacity that cuts the list inside a dense tile
    ids, cnt, got = gpu_all(t, wl.text, capacity=len(exp[0]) // 2 + 3)
    assert cnt == len(exp[0])
    assert_all_same(got, tuple(e[:len(exp[0]) // 2 + 3] for e in exp))


def check_list_properties(pats, text, ids, cnt, got):
    pos, mid, lens = got
    assert len(pos) == cnt
    assert np.all(np.diff(pos) >= 0)
    first = np.r_[True, pos[1:] != pos[:-1]] if len(pos) else np.zeros(0, bool)
    assert np.array_equal(np.unique(pos), np.flatnonzero(ids >= 0))
    assert np.array_equal(mid[first], ids[pos[first]])
    assert np.all(lens[~first] < lens[np.flatnonzero(~first) - 1])
    for a, b, c in zip(pos, mid, lens):
        p = pats.get(int(b))
        assert len(p) == c and bytes(text[a:a + c]) == p


def test_paper_scale_full_size_all():
    """The benchmark's 256 MiB workload: every record checked against the
    text and the pattern list, the ids against the oracle on sampled
    windows, and the records of those windows against the oracle's."""
    wl = W.paper_scale(0)
    t = pm.pm_build(wl.patterns)
    ids, cnt, got = gpu_all(t, wl.text, capacity=1 << 16)
    check_list_properties(wl.patterns, wl.text, ids, cnt, got)
    ot = oracle.Trie(wl.patterns)
    rng = np.random.Generator(np.random.MT19937(5))
    for a in list(rng.integers(0, len(wl.text) - 70_000, 6)) + [len(wl.text) - 70_000]:
        a, b = int(a), int(a) + 70_000
        o_ids, _, _ = ot.scan(wl.text, a, b)
        assert np.array_equal(ids[a:b], o_ids)
        e = ot.scan_all(wl.text, a, b)
        sel = (got[0] >= a) & (got[0] < b)
        assert_all_same(tuple(g[sel] for g in got), e)


def test_scan_all_host_chunks_and_capacity():
    """pm_scan_all_host: a host text longer than one 32 MiB chunk, with
    occurrences straddling the chunk boundary, listed in host memory exactly
    as the oracle lists them (positions are the whole text's); a capacity
    below the count keeps the list's first entries and reports the total;
    a list that outgrows the initial device buffers (dense ACGT) too."""
    pats = W.paper_scale(0, text_bytes=16, n_patterns=2000).patterns
    rng = np.random.Generator(np.random.MT19937(9))
    n = 40 * W.MiB + 77
    text = rng.integers(0, 256, size=n, dtype=np.uint8)
    W._plant_bernoulli(rng, text, pats, 1.0 / 4096)
    p = np.frombuffer(pats.get(int(np.argmax(pats.lengths()))), np.uint8)
    cut = 32 * W.MiB
    text[cut - len(p) // 2: cut - len(p) // 2 + len(p)] = p
    t = pm.pm_build(pats)
    h_text = torch.from_numpy(text).pin_memory().numpy()
    ot = oracle.Trie(pats)
    e_pos, e_id, e_len = ot.scan_all(text, threads=8)
    assert len(e_pos) > 5000 and np.any((e_pos < cut) & (e_pos + e_len > cut))
    m = np.full((len(e_pos) + 10, 2), -9, dtype=np.int64)
    total = pm.pm_scan_all_host(t, h_text, m)
    assert total == len(e_pos)
    g_pos, g_id, g_len = pm.decode_matches(m, total)
    assert np.array_equal(g_pos, e_pos) and np.array_equal(g_id, e_id) and np.array_equal(g_len, e_len)
    small = np.full((100, 2), -9, dtype=np.int64)
    assert pm.pm_scan_all_host(t, h_text, small) == len(e_pos)
    s_pos, s_id, s_len = pm.decode_matches(small, 100)
    assert np.array_equal(s_pos, e_pos[:100]) and np.array_equal(s_id, e_id[:100])
    # dense listing: more occurrences per chunk than the initial list buffers
    wl = W.acgt(3, text_bytes=12 * W.MiB + 5, n_patterns=20000, plant_rate=0.02)
    ta = pm.pm_build(wl.patterns)
    a_pos, a_id, a_len = oracle.Trie(wl.patterns).scan_all(wl.text, threads=8)
    assert len(a_pos) > (1 << 17)
    ma = np.zeros((len(a_pos), 2), dtype=np.int64)
    assert pm.pm_scan_all_host(ta, wl.text, ma) == len(a_pos)
    g_pos, g_id, g_len = pm.decode_matches(ma, len(a_pos))
    assert np.array_equal(g_pos, a_pos) and np.array_equal(g_id, a_id) and np.array_equal(g_len, a_len)
    assert pm.pm_scan_all_host(ta, wl.text[:0], ma) == 0
