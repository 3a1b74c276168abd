"""GPU parity on a text longer than 2^32 bytes.

A walk's start position travels through the scan as 40 bits (the low 32 in
one word of its ring entry, bits 32..39 in another), and a tile's distance to
its text's end is clipped to 32 bits. Both only matter past 2^32 bytes, so
this test scans a text of 2^32 + 1 MiB + 77 bytes in the benchmark's launch
configuration and compares with the CPU oracle (Section II-C: one walk per
start position; the ids and the count are exact integers, compared
bit-exactly).

The text is one pad byte repeated up to 2^32 - 1 MiB, then 2 MiB + 77 bytes
drawn over the patterns' alphabet with plants: across 2^32 itself, across
tile boundaries just above it, and in the last 64 bytes.

* Byte-class trie ('a'..'z', pad byte 0 on no trie edge): the oracle scans
  every position (in 256 MiB pieces on the host cores) and every id and the
  total count are compared.
* Byte-alphabet trie (the paper-scale pattern shape): the oracle's walk over
  a 4 GiB run of one byte value is slow, so it scans the varied region plus
  the longest pattern's length of pad before it, and one window of the
  constant run. Every position i below (start of the varied region) - max_len
  reads exactly max_len pad bytes, the same bytes as the window's first
  position, so its id and its number of occurrences equal that position's;
  the GPU ids there are checked against that value on the device, and the
  count against the window's per-position count times their number plus the
  oracle's count of the rest.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1702_03657_gb300 import pm
from paper_1702_03657_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HOST_THREADS = max(1, min(16, os.cpu_count() or 1))
BASE = 1 << 32
N = BASE + W.MiB + 77
VARIED = BASE - W.MiB          # start of the varied region


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


def make_text(pats: W.PatternSet, alphabet: np.ndarray, pad: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.MT19937(seed))
    text = np.full(N, pad, dtype=np.uint8)
    text[VARIED:] = alphabet[rng.integers(0, len(alphabet), size=N - VARIED)]
    W._plant_bernoulli(rng, text[VARIED:], pats, 1.0 / 512)
    lens = pats.lengths()

    def plant(at, j):
        p = np.frombuffer(pats.get(j), np.uint8)
        if 0 <= at and at + len(p) <= N:
            text[at:at + len(p)] = p

    j = int(np.argmax(lens))
    plant(BASE - int(lens[j]) // 2, j)            # across 2^32
    for tile in (1024, 2048):                     # across tile ends above 2^32
        for k in range(1, 9):
            plant(BASE + k * tile - 3, int(rng.integers(0, pats.n)))
    short = int(np.argmin(lens))
    plant(N - int(lens[short]), short)            # ends at the last byte
    plant(N - 64, int(rng.integers(0, pats.n)))   # in the last 64 bytes
    return text


def scan_large(trie, text):
    tv = torch.from_numpy(text).to("cuda")
    ids = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    pm.pm_scan(trie, tv, ids, cnt)
    torch.cuda.synchronize()
    del tv
    return ids, int(cnt.item())


def test_byte_classes_every_position():
    wl = W.tiny(0, text_bytes=16)
    alpha = np.arange(ord("a"), ord("z") + 1, dtype=np.uint8)
    text = make_text(wl.patterns, alpha, 0, 41)
    t = pm.pm_build(wl.patterns)
    assert pm.pm_stats(t)["alphabet"] < 256
    ids, cnt = scan_large(t, text)
    ot = oracle.Trie(wl.patterns)
    piece = 256 * W.MiB
    total = 0
    for a in range(0, N, piece):
        b = min(N, a + piece)
        o_ids, o_cnt, _ = ot.scan(text, a, b, threads=HOST_THREADS)
        g = ids[a:b].cpu().numpy()
        bad = np.flatnonzero(g != o_ids)
        assert bad.size == 0, f"{bad.size} mismatches from {a}, first at {a + bad[:5]}"
        total += o_cnt
    assert cnt == total
    assert int((ids[BASE:] >= 0).sum().item()) > 1000   # matches past 2^32


def test_byte_alphabet_past_2_32():
    wl = W.paper_scale(0, text_bytes=16, n_patterns=4000)
    text = make_text(wl.patterns, np.arange(256, dtype=np.uint8), 0x5A, 42)
    t = pm.pm_build(wl.patterns)
    st = pm.pm_stats(t)
    assert st["alphabet"] == 256
    L = int(st["max_len"])
    ids, cnt = scan_large(t, text)
    ot = oracle.Trie(wl.patterns)
    lo = VARIED - L                      # positions below lo read only pad bytes
    w_ids, w_cnt, _ = ot.scan(text, 0, 4096, threads=HOST_THREADS)
    assert np.all(w_ids == w_ids[0]) and w_cnt % 4096 == 0
    per_pos = w_cnt // 4096
    assert int((ids[:lo] != int(w_ids[0])).sum().item()) == 0
    o_ids, o_cnt, _ = ot.scan(text, lo, N, threads=HOST_THREADS)
    g = ids[lo:].cpu().numpy()
    bad = np.flatnonzero(g != o_ids)
    assert bad.size == 0, f"{bad.size} mismatches, first at {lo + bad[:5]}"
    assert cnt == per_pos * lo + o_cnt
    assert int((ids[BASE:] >= 0).sum().item()) > 1000
