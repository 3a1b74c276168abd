"""Streams of chunks (pm_scanner_*): a text pushed in arbitrary chunks gives
exactly the ids and count of one scan of the whole text (Section II-B's
overlap rule), checked against the oracle."""
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


def stream_scan(sc, text, sizes, max_len):
    """Push text in chunks of the given sizes (cycled), then finish; returns
    the concatenated ids and the summed count."""
    d = torch.from_numpy(np.array(text, dtype=np.uint8)).cuda() if len(text) else \
        torch.zeros(1, dtype=torch.uint8, device="cuda")
    ids_all, total, a, k = [], 0, 0, 0
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    while a < len(text):
        c = min(sizes[k % len(sizes)], len(text) - a)
        k += 1
        buf = torch.full((c + max_len,), -9, dtype=torch.int32, device="cuda")
        chunk = d[a:a + c]
        n = sc.push(chunk, buf, cnt, length=c)
        torch.cuda.synchronize()
        ids_all.append(buf[:n].cpu().numpy())
        total += int(cnt.item())
        a += c
    buf = torch.full((max_len + 1,), -9, dtype=torch.int32, device="cuda")
    n = sc.finish(buf, cnt)
    torch.cuda.synchronize()
    ids_all.append(buf[:n].cpu().numpy())
    total += int(cnt.item())
    return np.concatenate(ids_all) if ids_all else np.zeros(0, np.int32), total


@pytest.mark.parametrize("sizes", [
    [1 << 20], [100_000, 7, 0, 63, 64, 65, 1, 5000], [1], [3, 200, 17], [64 * 1024 + 3],
])
def test_chunks_equal_one_scan(sizes):
    wl = W.paper_scale(2, text_bytes=(2 << 20) + 11, n_patterns=3000)
    # plants straddling every 64 KiB boundary
    p = np.frombuffer(wl.patterns.get(5), np.uint8)
    text = wl.text.copy()
    for cut in range(1 << 16, len(text) - 100, 1 << 16):
        text[cut - len(p) // 2: cut - len(p) // 2 + len(p)] = p
    ot = oracle.Trie(wl.patterns)
    o_ids, o_cnt, _ = ot.scan(text, threads=8)
    t = pm.pm_build(wl.patterns)
    sc = pm.pm_scanner_open(t)
    ids, cnt = stream_scan(sc, text[:200_000] if sizes == [1] else text, sizes,
                           pm.pm_stats(t)["max_len"])
    if sizes == [1]:
        o_ids, o_cnt, _ = ot.scan(text[:200_000])
    assert cnt == o_cnt
    assert np.array_equal(ids, o_ids)
    sc.close()


def test_long_patterns_short_chunks_and_reuse():
    """max_len 4096 (carry of 4095 bytes) with chunks shorter than the carry,
    a single-byte trie (no carry), and a scanner reused after finish."""
    rng = np.random.Generator(np.random.MT19937(7))
    text = rng.integers(0, 4, size=60_000, dtype=np.uint8) + ord("a")
    pats = [bytes(text[1000:1000 + 4096]), bytes(text[30_000:30_010]), b"ab", b"abcd"]
    t = pm.pm_build(pats)
    o_ids, o_cnt, _ = oracle.Trie(pats).scan(text)
    sc = pm.pm_scanner_open(t)
    for sizes in ([1000, 3, 4095, 4096, 4097, 77], [50_000, 9], [10]):
        ids, cnt = stream_scan(sc, text, sizes, 4096)
        assert cnt == o_cnt and np.array_equal(ids, o_ids)
    sc.close()
    t1 = pm.pm_build([b"a", b"c"])
    o_ids, o_cnt, _ = oracle.Trie([b"a", b"c"]).scan(text)
    sc = pm.pm_scanner_open(t1)
    ids, cnt = stream_scan(sc, text, [333, 1], 1)
    assert cnt == o_cnt and np.array_equal(ids, o_ids)
    # an empty stream
    ids, cnt = stream_scan(sc, np.zeros(0, np.uint8), [5], 1)
    assert cnt == 0 and ids.size == 0
    sc.close()


def test_acgt_deep_level_stream():
    wl = W.acgt(3, text_bytes=3 << 20, n_patterns=20_000)
    t = pm.pm_build(wl.patterns)
    assert pm.pm_stats(t)["deep_k"] > 0
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=8)
    sc = pm.pm_scanner_open(t)
    ids, cnt = stream_scan(sc, wl.text, [777_777, 31, 1 << 20], 32)
    assert cnt == o_cnt and np.array_equal(ids, o_ids)
    sc.close()


def test_chunks_above_the_copy_limit():
    """Chunks over 16 MiB are scanned in place (held positions on a small
    copy, the chunk's own in the chunk); mixed with copied chunks."""
    wl = W.paper_scale(4, text_bytes=(40 << 20) + 5, n_patterns=2000)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=16)
    sc = pm.pm_scanner_open(t)
    ids, cnt = stream_scan(sc, wl.text, [(17 << 20) + 3, 5, 16 << 20, (20 << 20)],
                           pm.pm_stats(t)["max_len"])
    assert cnt == o_cnt and np.array_equal(ids, o_ids)
    sc.close()
