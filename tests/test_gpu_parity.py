"""GPU parity: the CUDA scan through the C ABI against the CPU oracle.

Integer work, so the bar is bit-exact: every ids[i] and every count equal
the oracle's on the same seeded input. Every test compares every position,
the full-size workloads included (in the launch configuration the benchmark
times). A text longer than 2^32 bytes checks the start positions past 32
bits (test_gpu_large.py).
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03657_gb300 import build as B
    B.build()
    pm.load()
    torch.cuda.init()
    yield
    torch.cuda.synchronize()
    assert pm.pm_device_error() == 0


def dev(a, dtype=torch.uint8):
    t = torch.from_numpy(np.array(a, copy=True))  # a writable copy
    return t.to("cuda")


def gpu_scan(trie, text: np.ndarray, cfg=None, lookups=False, offset=0):
    """Scan through pm_scan (or pm_scan_ex with a config / lookup counter).
    `offset` shifts the text inside its buffer to test unaligned pointers."""
    n = len(text)
    buf = torch.zeros(n + offset + 16, dtype=torch.uint8, device="cuda")
    if n:
        buf[offset:offset + n] = dev(text)
    tv = buf[offset:offset + n]
    ids = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    if cfg is None and not lookups:
        pm.pm_scan(trie, tv, ids, cnt, length=n)
        look = None
    else:
        lk = torch.zeros(1, dtype=torch.int64, device="cuda") if lookups else None
        pm.pm_scan_ex(trie, tv, None, ids, cnt, lookups=lk, cfg=cfg, length=n)
        look = int(lk.item()) if lookups else None
    torch.cuda.synchronize()
    return ids.cpu().numpy(), int(cnt.item()), look


def assert_same(ids, cnt, o_ids, o_cnt):
    bad = np.flatnonzero(ids != o_ids)
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: " \
                          f"gpu {ids[bad[:5]]} oracle {o_ids[bad[:5]]}"
    assert cnt == o_cnt


def small_cfg(trie, **kw):
    """A small persistent-kernel configuration (the light form off)."""
    c = pm.pm_get_config(trie)
    c.update(threads=128, tile=256, stages=2, positions=4, light_max=0)
    c.update(kw)
    return c


def no_deep(cfg):
    """cfg without the deep level: sixteen positions a lane need it (or the
    byte alphabet), so such a configuration goes to eight."""
    return dict(cfg, deep=0, positions=min(cfg["positions"], 8))


def persistent(trie, **kw):
    """The handle's configuration with the light form off."""
    return dict(pm.pm_get_config(trie), light_max=0, **kw)


def light(trie, **kw):
    """The handle's configuration with the light form for every length."""
    return dict(pm.pm_get_config(trie), light_max=1 << 30, **kw)


# --------------------------------------------------------------------------


def test_golden_fixtures():
    import glob
    import json
    for f in sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json"))):
        c = json.load(open(f))
        pats = [bytes.fromhex(p) for p in c["patterns"]]
        text = np.frombuffer(bytes.fromhex(c["text"]), np.uint8)
        t = pm.pm_build(pats)
        ids, cnt, look = gpu_scan(t, text, lookups=True)
        assert ids.tolist() == c["ids"], f
        assert cnt == c["count"], f
        assert look == c["lookups"], f
        for cfg in (None, persistent(t), light(t)):
            ids2, cnt2, _ = gpu_scan(t, text, cfg=cfg)
            assert ids2.tolist() == c["ids"] and cnt2 == c["count"], f


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi,n", [
    (0, 2, 20, 1, 7, 50_001), (1, 3, 60, 1, 9, 70_003), (2, 4, 200, 2, 12, 65_537),
    (3, 26, 300, 3, 16, 100_000), (4, 256, 500, 1, 8, 99_999), (5, 5, 100, 4, 30, 33_333),
])
def test_random_small_all_positions(seed, alphabet, npat, lo, hi, n):
    wl = W.random_case(seed, npat, n, alphabet, lo, hi, plant_rate=0.05)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, o_look = oracle.Trie(wl.patterns).scan(wl.text)
    ids, cnt, _ = gpu_scan(t, wl.text)                         # default config
    assert_same(ids, cnt, o_ids, o_cnt)
    ids, cnt, look = gpu_scan(t, wl.text, cfg=small_cfg(t), lookups=True)
    assert_same(ids, cnt, o_ids, o_cnt)
    assert look == o_look


def test_config_sweep():
    """Every launch configuration gives the same bits."""
    for wl in (W.random_case(11, 400, 40_000 + 77, 4, 3, 14, plant_rate=0.05),
               W.paper_scale(3, text_bytes=300_000 + 9, n_patterns=3000)):
        t = pm.pm_build(wl.patterns)
        st = pm.pm_stats(t)
        o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text)
        base = pm.pm_get_config(t)
        tried = 0
        for threads in (128, 256, 1024):
            for tile in (128, 1024, 8192):
                for k in sorted({0, 1, st["dense_k_max"]}):
                    for bits in (8, 16, 32):
                        for rs in (0, 1):
                            c = dict(base, threads=threads, tile=tile, dense_k=k,
                                     filter_bits=bits, row_search=rs, light_max=0,
                                     stages=2 + (tile == 128) * 2,
                                     checked=int(threads == 256),
                                     positions=(4, 8, 16)[(rs + threads // 128 + tile // 1024) % 3])
                            try:
                                pm.pm_set_config(t, c)
                            except pm.PMError:
                                continue  # e.g. no filter of that width at this k
                            ids, cnt, _ = gpu_scan(t, wl.text, cfg=c)
                            assert_same(ids, cnt, o_ids, o_cnt)
                            tried += 1
        assert tried >= 20
    assert pm.pm_device_error() == 0


def test_unaligned_and_ragged():
    wl = W.random_case(12, 200, 30_011, 26, 2, 20)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text)
    for off in (1, 3, 8, 15):
        for cfg in (persistent(t), light(t)):
            ids, cnt, _ = gpu_scan(t, wl.text, cfg=cfg, offset=off)
            assert_same(ids, cnt, o_ids, o_cnt)
    # ids pointer not 16-byte aligned
    tv = dev(wl.text)
    big = torch.zeros(len(wl.text) + 1, dtype=torch.int32, device="cuda")
    ids = big[1:]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pm.pm_scan(t, tv, ids, cnt)
    torch.cuda.synchronize()
    assert_same(ids.cpu().numpy(), int(cnt.item()), o_ids, o_cnt)
    # lengths around tile and halo boundaries
    c = small_cfg(t)
    for n in (0, 1, 2, 3, 4, 5, 15, 16, 17, 1023, 1024, 1025, 1024 + 19, 2048, 4097):
        o_ids2, o_cnt2, _ = oracle.Trie(wl.patterns).scan(wl.text[:n])
        ids, cnt, _ = gpu_scan(t, wl.text[:n], cfg=c)
        assert_same(ids, cnt, o_ids2, o_cnt2)


def test_degenerate_pattern_sets():
    rng = np.random.Generator(np.random.MT19937(5))
    text = rng.integers(0, 256, size=20_000, dtype=np.uint8)
    text[100:108] = np.frombuffer(b"\x00\x00\xff\xffabcd", np.uint8)
    cases = [
        [],                                              # nothing matches
        [bytes([b]) for b in range(256)],                # every byte, k = 1
        [b"\x00", b"\x00\x00", b"\xff\xff", b"abcd"],    # NUL and 0xFF
        [bytes(text[500:500 + 4096])],                    # longest allowed
        [b"a" * k for k in range(1, 40)],                 # nested prefixes
        [bytes(text[7:9]), bytes(text[7:9])],             # duplicates
    ]
    for pats in cases:
        t = pm.pm_build(pats)
        o_ids, o_cnt, o_look = oracle.Trie(pats).scan(text)
        for cfg in (None, small_cfg(t)):
            ids, cnt, _ = gpu_scan(t, text, cfg=cfg)
            assert_same(ids, cnt, o_ids, o_cnt)
        _, _, look = gpu_scan(t, text, lookups=True)
        assert look == o_look


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi,deep_k", [
    (20, 4, 3000, 12, 24, 12), (21, 3, 800, 14, 20, 13), (22, 26, 2000, 8, 16, 5),
    (23, 200, 2000, 4, 10, 3), (24, 128, 2000, 3, 9, 3), (25, 64, 1500, 5, 9, 4),
])
def test_deep_level(seed, alphabet, npat, lo, hi, deep_k):
    """Byte-class tries get a packed-class filter in shared memory and a deep
    level in L2 (depth D at most the shortest pattern). With the deep level
    on and off, every filter depth, four and eight positions per lane,
    checked and counting lookups, and with bytes outside the patterns'
    alphabet in the text, the bits equal the oracle's; a batch of short texts
    (shorter than the deep level's depth) too."""
    wl = W.random_case(seed, npat, 150_001, alphabet, lo, hi, plant_rate=0.05)
    rng = np.random.Generator(np.random.MT19937(seed))
    text = wl.text.copy()
    other = rng.random(len(text)) < 0.002           # bytes on no trie edge
    text[other] = ord("Z") if alphabet <= 26 else 255
    t = pm.pm_build(wl.patterns)
    st = pm.pm_stats(t)
    assert st["deep_k"] == deep_k
    assert st["deep_bytes"] > 0
    cfg = pm.pm_get_config(t)
    assert cfg["deep"] == 1
    ot = oracle.Trie(wl.patterns)
    o_ids, o_cnt, o_look = ot.scan(text)
    assert o_cnt > 0
    for c in (None, no_deep(cfg), dict(cfg, checked=1), small_cfg(t),
              small_cfg(t, deep=0, dense_k=1), dict(cfg, tile=128, stages=4, positions=4),
              dict(cfg, positions=4), small_cfg(t, dense_k=0)):
        ids, cnt, _ = gpu_scan(t, text, cfg=c)
        assert_same(ids, cnt, o_ids, o_cnt)
    _, _, look = gpu_scan(t, text, lookups=True)
    assert look == o_look
    # batch: texts around the deep level's depth
    pieces, a = [], 0
    for n in [0, 1, deep_k - 1, deep_k, deep_k + 1, 3, 100, 5000, deep_k + 3, 2]:
        pieces.append(text[a:a + n])
        a += n + 7
    data, off = W.concat(pieces)
    bw = W.Workload("deep_batch", seed, wl.patterns, data, off)
    b_ids, b_counts, _ = ot.scan_batch(data, off)
    for c in (None, small_cfg(t), no_deep(cfg)):
        ids, counts = batch_gpu(t, bw, c)
        assert np.array_equal(ids, b_ids) and np.array_equal(counts, b_counts)


@pytest.mark.parametrize("seed,alphabet,npat,lo,hi,n", [
    (40, 2, 30, 1, 9, 9_001), (41, 4, 3000, 14, 24, 40_000), (42, 26, 300, 3, 16, 65_536),
    (43, 256, 800, 1, 8, 20_003), (44, 200, 1500, 4, 10, 33_333), (45, 256, 3000, 8, 40, 64_000),
])
def test_light_form_equals_persistent(seed, alphabet, npat, lo, hi, n):
    """The light launch form for short texts (small CTAs, filters read from
    L2, walks in place) and the persistent kernel give the oracle's bits:
    byte alphabets with exact and Bloom filters, byte classes with and
    without a deep level, checked, counting and unaligned."""
    wl = W.random_case(seed, npat, n, alphabet, lo, hi, plant_rate=0.05)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, o_look = oracle.Trie(wl.patterns).scan(wl.text)
    for cfg in (light(t), persistent(t), light(t, checked=1), no_deep(light(t))
                if pm.pm_stats(t)["deep_k"] else light(t, row_search=1), light(t, layout=1)):
        ids, cnt, _ = gpu_scan(t, wl.text, cfg=cfg)
        assert_same(ids, cnt, o_ids, o_cnt)
    ids, cnt, look = gpu_scan(t, wl.text, cfg=light(t), lookups=True)
    assert_same(ids, cnt, o_ids, o_cnt)
    assert look == o_look
    ids, cnt, _ = gpu_scan(t, wl.text, cfg=light(t), offset=3)
    assert_same(ids, cnt, o_ids, o_cnt)


@pytest.mark.parametrize("letters", [b"ACGT", bytes([0, 8, 16, 24]), bytes([0, 1, 0x40, 0x41]),
                                     bytes([7, 15, 23, 255]), b"TGCA"])
def test_four_letter_alphabets(letters):
    """Four letters and patterns of 13 or more: 2-bit classes, filter depth
    10 and deep level 13 fixed at compile time. Letter sets that a 3-bit
    field of the byte tells apart (ACGT: the low three bits; 0, 8, 16, 24
    and 7, 15, 23, 255: bits 2..4) are classified four bytes at a time;
    others (0, 1, 0x40, 0x41) through the shared-memory table. Bytes of no
    pattern, among them bytes with a letter's field, are found either way:
    every id equals the oracle's, single text and batch."""
    wl = W.random_case(31, 3000, 200_003, 4, 13, 24, plant_rate=0.05)
    m = np.arange(256, dtype=np.uint8)
    m[ord("a"):ord("a") + 4] = np.frombuffer(letters, np.uint8)
    pats = W.PatternSet(m[wl.patterns.data], wl.patterns.off.copy())
    text = m[wl.text]
    rng = np.random.Generator(np.random.MT19937(31))
    others = np.setdiff1d(np.arange(256), np.frombuffer(letters, np.uint8)).astype(np.uint8)
    pos = np.flatnonzero(rng.random(len(text)) < 0.003)
    text[pos] = others[rng.integers(0, len(others), size=pos.size)]
    t = pm.pm_build(pats)
    st = pm.pm_stats(t)
    assert st["alphabet"] == 5 and st["deep_k"] == 13
    cfg = pm.pm_get_config(t)
    assert cfg["dense_k"] == 10 and cfg["deep"] == 1
    ot = oracle.Trie(pats)
    o_ids, o_cnt, _ = ot.scan(text)
    assert o_cnt > 0
    for c in (None, persistent(t), persistent(t, positions=4), dict(cfg, checked=1),
              small_cfg(t, dense_k=10), light(t), persistent(t, schedule=pm.PM_SCHED_DYNAMIC)):
        ids, cnt, _ = gpu_scan(t, text, cfg=c)
        assert_same(ids, cnt, o_ids, o_cnt)
    pieces, a = [], 0
    for n in [0, 1, 12, 13, 14, 3, 100, 5000, 16, 2, 70_000]:
        pieces.append(text[a:a + n])
        a += n + 5
    data, off = W.concat(pieces)
    bw = W.Workload("four_batch", 31, pats, data, off)
    b_ids, b_counts, _ = ot.scan_batch(data, off)
    for c in (None, small_cfg(t, dense_k=10)):
        ids, counts = batch_gpu(t, bw, c)
        assert np.array_equal(ids, b_ids) and np.array_equal(counts, b_counts)


@pytest.mark.parametrize("sched", [1, 2])
def test_schedules(sched):
    """Static schedule (warp w: tiles w, w + W, ...) and dynamic schedule
    (CTAs take runs of PM_CHUNK_TILES tiles from a global counter, warps take
    the run's tiles as they finish one) give the oracle's bits: texts ending
    inside the first tile, on a run's end, one byte past it and in a partial
    last run; 31-warp CTAs (runs not a multiple of the warps), 256-byte
    tiles, three stages; and a batch."""
    assert pm.PM_CHUNK_TILES == 32 and sched in (pm.PM_SCHED_STATIC, pm.PM_SCHED_DYNAMIC)
    wl = W.paper_scale(7, text_bytes=3 * W.MiB + 13, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    ot = oracle.Trie(wl.patterns)
    cfgs = (persistent(t, schedule=sched), persistent(t, schedule=sched, tile=256, threads=992, positions=8),
            small_cfg(t, schedule=sched),
            persistent(t, schedule=sched, stages=3, positions=4, threads=512))
    for n in (1, 255, 32 * 1024, 32 * 1024 + 1, 5 * 32 * 1024 + 7, len(wl.text)):
        text = wl.text[:n]
        o_ids, o_cnt, _ = ot.scan(text, threads=HOST_THREADS)
        for c in cfgs:
            ids, cnt, _ = gpu_scan(t, text, cfg=c)
            assert_same(ids, cnt, o_ids, o_cnt)
    pieces, a = [], 0
    for n in [0, 5, 40_000, 70_000, 1, 300_000, 33 * 1024, 17]:
        pieces.append(wl.text[a:a + n])
        a += n + 3
    data, off = W.concat(pieces)
    bw = W.Workload("sched_batch", 7, wl.patterns, data, off)
    b_ids, b_counts, _ = ot.scan_batch(data, off)
    for c in cfgs[:2]:
        ids, counts = batch_gpu(t, bw, c)
        assert np.array_equal(ids, b_ids) and np.array_equal(counts, b_counts)


def test_sixteen_positions():
    """Sixteen positions a lane (512-position groups) at the byte alphabet's
    Bloom level, the default there: one and two groups a tile, checked mode,
    three stages, small CTAs, unaligned text, a text ending inside a group,
    and a batch; every id equals the oracle's."""
    wl = W.paper_scale(8, text_bytes=2 * W.MiB + 333, n_patterns=4000)
    t = pm.pm_build(wl.patterns)
    assert pm.pm_get_config(t)["positions"] == 16
    ot = oracle.Trie(wl.patterns)
    o_ids, o_cnt, _ = ot.scan(wl.text, threads=HOST_THREADS)
    for c in (persistent(t), persistent(t, tile=512), persistent(t, checked=1),
              persistent(t, stages=3, threads=512), small_cfg(t, positions=16, tile=512),
              persistent(t, schedule=2)):
        ids, cnt, _ = gpu_scan(t, wl.text, cfg=c)
        assert_same(ids, cnt, o_ids, o_cnt)
        ids, cnt, _ = gpu_scan(t, wl.text, cfg=c, offset=5)
        assert_same(ids, cnt, o_ids, o_cnt)
    for n in (511, 513, 100_001):
        e_ids, e_cnt, _ = ot.scan(wl.text[:n])
        ids, cnt, _ = gpu_scan(t, wl.text[:n], cfg=persistent(t))
        assert_same(ids, cnt, e_ids, e_cnt)
    pieces, a = [], 0
    for n in [0, 7, 511, 512, 513, 40_000, 3, 200_000]:
        pieces.append(wl.text[a:a + n])
        a += n + 11
    data, off = W.concat(pieces)
    bw = W.Workload("p16_batch", 8, wl.patterns, data, off)
    b_ids, b_counts, _ = ot.scan_batch(data, off)
    for c in (None, persistent(t), persistent(t, checked=1)):
        ids, counts = batch_gpu(t, bw, c)
        assert np.array_equal(ids, b_ids) and np.array_equal(counts, b_counts)


def test_unary_chains():
    """Runs of single-child nodes are walked by comparing the text with the
    run's labels 16 bytes at a time. Texts that leave a run at every offset,
    runs from the root, patterns that end inside a run (prefixes of longer
    patterns), runs longer than several 16-byte blocks, a text that ends
    inside a run, unaligned texts and batches: all against the oracle."""
    rng = np.random.Generator(np.random.MT19937(77))
    base = [rng.integers(0, 256, size=L, dtype=np.uint8).tobytes() for L in (3, 17, 40, 100, 301)]
    cases = [
        base + [b[:k] for b in base[2:] for k in (5, 16, 33)],   # finals inside runs
        [base[4]],                                               # one run from the root
        [b"ACGT" * 8 + b"A", b"ACGT" * 8 + b"C", b"ACGTACGA"],   # small alphabet
    ]
    for pats in cases:
        pieces = []
        for b in pats:
            for k in range(len(b)):                    # leave the run at offset k
                x = bytearray(b)
                x[k] ^= 0x5A
                pieces.append(bytes(x))
            pieces.append(b)
        filler = rng.integers(0, 256, size=5000, dtype=np.uint8).tobytes()
        text = np.frombuffer(b"".join(pieces) + filler + pats[-1][:-1], np.uint8)
        t = pm.pm_build(pats)
        ot = oracle.Trie(pats)
        o_ids, o_cnt, _ = ot.scan(text)
        assert o_cnt > 0
        cfg = pm.pm_get_config(t)
        for c in (None, dict(cfg, positions=4), dict(cfg, checked=1), dict(cfg, layout=1),
                  small_cfg(t), dict(cfg, row_search=1)):
            ids, cnt, _ = gpu_scan(t, text, cfg=c)
            assert_same(ids, cnt, o_ids, o_cnt)
        for off in (1, 2, 3):
            ids, cnt, _ = gpu_scan(t, text, offset=off)
            assert_same(ids, cnt, o_ids, o_cnt)
        # a batch whose texts end inside runs
        cut = [0, 7, len(pats[0]) - 1, 500, 2001, len(text)]
        data, off = W.concat([text[a:b] for a, b in zip(cut, cut[1:])])
        bw = W.Workload("chains", 0, W.PatternSet.from_list(pats), data, off)
        b_ids, b_counts, _ = ot.scan_batch(data, off)
        ids, counts = batch_gpu(t, bw)
        assert np.array_equal(ids, b_ids) and np.array_equal(counts, b_counts)


def test_bitmapped_node_layout():
    """Walks over the bitmapped nodes of Section III (256-bit child bitmap +
    first child, child = first + rank) give the same bits as the CRS row
    records: byte alphabets with long rows, small alphabets, a deep level,
    checked, counting and batched."""
    cases = [W.random_case(31, 500, 99_999, 256, 1, 8, plant_rate=0.05),
             W.random_case(32, 300, 70_003, 3, 1, 9, plant_rate=0.05),
             W.random_case(33, 2000, 120_001, 4, 12, 24, plant_rate=0.05),
             W.paper_scale(3, text_bytes=2 * W.MiB + 3, n_patterns=3000)]
    for wl in cases:
        t = pm.pm_build(wl.patterns)
        ot = oracle.Trie(wl.patterns)
        o_ids, o_cnt, o_look = ot.scan(wl.text, threads=8)
        base = pm.pm_get_config(t)
        for c in (dict(base, layout=1), dict(base, layout=1, checked=1),
                  small_cfg(t, layout=1, dense_k=0, deep=0)):
            ids, cnt, _ = gpu_scan(t, wl.text, cfg=c)
            assert_same(ids, cnt, o_ids, o_cnt)
        _, _, look = gpu_scan(t, wl.text, cfg=dict(base, layout=1), lookups=True)
        assert look == o_look
    wl = W.batched(5, ntexts=300, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    o_ids, o_counts, _ = oracle.Trie(wl.patterns).scan_batch(wl.text, wl.offsets)
    ids, counts = batch_gpu(t, wl, cfg=dict(pm.pm_get_config(t), layout=1))
    assert np.array_equal(ids, o_ids) and np.array_equal(counts, o_counts)


def walks_of(t, text, cfg=None):
    tv = dev(text)
    ids = torch.empty(len(text), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    wk = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    pm.pm_scan_walks(t, tv, ids, cnt, wk, cfg=cfg)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), int(cnt.item()), int(wk.item())


def test_truncated_levels_settle_positions():
    """The filter, dense tables and deep level are the trie truncated at a
    depth below the shortest pattern, used as an exact prefilter: every
    matched position is walked (verified in the full trie), most others are
    settled without a walk, and the bits are the oracle's either way."""
    for wl, frac in ((W.paper_scale(1, text_bytes=6 * W.MiB + 1), 0.005),
                     (W.acgt(1, text_bytes=4 * W.MiB + 7, n_patterns=100_000), 0.05)):
        t = pm.pm_build(wl.patterns)
        o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=HOST_THREADS)
        ids, cnt, walks = walks_of(t, wl.text)
        assert_same(ids, cnt, o_ids, o_cnt)
        matched = int((o_ids >= 0).sum())
        assert matched <= walks <= frac * len(wl.text)
        if pm.pm_stats(t)["deep_k"]:
            ids0, cnt0, walks0 = walks_of(t, wl.text, cfg=no_deep(pm.pm_get_config(t)))
            assert_same(ids0, cnt0, o_ids, o_cnt)
            assert walks0 > 5 * walks       # the filter alone passes several times as many


def test_tiny_config_full():
    wl = W.tiny(0)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=HOST_THREADS)
    ids, cnt, _ = gpu_scan(t, wl.text)
    assert_same(ids, cnt, o_ids, o_cnt)
    assert cnt >= 256  # one plant per 4 KiB block


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_paper_scale_reduced_full(seed):
    wl = W.paper_scale(seed, text_bytes=6 * W.MiB + 13)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=HOST_THREADS)
    ids, cnt, _ = gpu_scan(t, wl.text)
    assert_same(ids, cnt, o_ids, o_cnt)


def test_acgt_reduced_full():
    wl = W.acgt(0, text_bytes=4 * W.MiB + 5, n_patterns=100_000)
    t = pm.pm_build(wl.patterns)
    o_ids, o_cnt, o_look = oracle.Trie(wl.patterns).scan(wl.text, threads=HOST_THREADS)
    ids, cnt, _ = gpu_scan(t, wl.text)
    assert_same(ids, cnt, o_ids, o_cnt)
    _, _, look = gpu_scan(t, wl.text, lookups=True)
    assert look == o_look


def batch_gpu(trie, wl, cfg=None):
    tx = dev(wl.text)
    off = dev(wl.offsets.astype(np.int64))
    ids = torch.full((len(wl.text),), -7, dtype=torch.int32, device="cuda")
    counts = torch.full((wl.ntexts,), -7, dtype=torch.int64, device="cuda")
    if cfg is None:
        pm.pm_scan_batch(trie, tx, off, ids, counts)
    else:
        pm.pm_scan_ex(trie, tx, off, ids, counts, cfg=cfg)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), counts.cpu().numpy()


def test_batched_config_full():
    wl = W.batched(0)
    t = pm.pm_build(wl.patterns)
    o_ids, o_counts, _ = oracle.Trie(wl.patterns).scan_batch(wl.text, wl.offsets,
                                                             threads=1)
    ids, counts = batch_gpu(t, wl)
    assert np.array_equal(ids, o_ids)
    assert np.array_equal(counts, o_counts)
    ids, counts = batch_gpu(t, wl, cfg=small_cfg(t))
    assert np.array_equal(ids, o_ids) and np.array_equal(counts, o_counts)


def test_batch_edge_cases():
    pats = [b"abc", b"bc", b"c", b"cab"]
    texts = [b"", b"ab", b"cabc", b"", b"c", b"abcabc" * 300, b"", b"b"]
    data, off = W.concat([np.frombuffer(x, np.uint8) for x in texts])
    wl = W.Workload("edge", 0, W.PatternSet.from_list(pats), data, off)
    t = pm.pm_build(pats)
    o_ids, o_counts, _ = oracle.Trie(pats).scan_batch(data, off)
    for cfg in (None, small_cfg(t)):
        ids, counts = batch_gpu(t, wl, cfg)
        assert np.array_equal(ids, o_ids) and np.array_equal(counts, o_counts)


def test_batch_graph_capture_and_streams():
    wl = W.batched(3, ntexts=512, n_patterns=2000)
    t = pm.pm_build(wl.patterns)
    o_ids, o_counts, _ = oracle.Trie(wl.patterns).scan_batch(wl.text, wl.offsets)
    tx = dev(wl.text)
    off = dev(wl.offsets.astype(np.int64))
    ids = torch.empty(len(wl.text), dtype=torch.int32, device="cuda")
    counts = torch.empty(wl.ntexts, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pm.pm_scan_batch(t, tx, off, ids, counts)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pm.pm_scan_batch(t, tx, off, ids, counts)
    for _ in range(3):
        ids.fill_(-9)
        counts.fill_(-9)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ids.cpu().numpy(), o_ids)
        assert np.array_equal(counts.cpu().numpy(), o_counts)
    # two streams scanning different texts with the same handle at once
    wl2 = W.random_case(9, 100, 300_000, 256, 1, 6)
    t2 = pm.pm_build(wl.patterns)
    tx2 = dev(wl2.text)
    ids2 = torch.empty(len(wl2.text), dtype=torch.int32, device="cuda")
    c2 = torch.empty(1, dtype=torch.int64, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(4):
        with torch.cuda.stream(s1):
            pm.pm_scan_batch(t, tx, off, ids, counts)
        with torch.cuda.stream(s2):
            pm.pm_scan(t2, tx2, ids2, c2)
    torch.cuda.synchronize()
    o2, oc2, _ = oracle.Trie(wl.patterns).scan(wl2.text)
    assert np.array_equal(ids.cpu().numpy(), o_ids)
    assert np.array_equal(ids2.cpu().numpy(), o2) and int(c2.item()) == oc2


def test_dynamic_schedule_capture_and_streams():
    """PM_SCHED_DYNAMIC asks for a run counter per launch from a stream-ordered
    pool. Captured into a CUDA graph the launch takes the static schedule
    instead (no allocation in the graph) and replays bit-exactly; launched on
    two streams at once with one handle, each launch has its own counter."""
    wl = W.paper_scale(5, text_bytes=12 * W.MiB + 1, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    dyn = dict(pm.pm_get_config(t), schedule=pm.PM_SCHED_DYNAMIC)
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=HOST_THREADS)
    tx = dev(wl.text)
    ids = torch.empty(len(wl.text), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pm.pm_scan_ex(t, tx, None, ids, cnt, cfg=dyn)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pm.pm_scan_ex(t, tx, None, ids, cnt, cfg=dyn)
    for _ in range(2):
        ids.fill_(-9)
        g.replay()
        torch.cuda.synchronize()
        assert_same(ids.cpu().numpy(), int(cnt.item()), o_ids, o_cnt)
    ids2 = torch.empty_like(ids)
    cnt2 = torch.empty_like(cnt)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(4):
        with torch.cuda.stream(s1):
            pm.pm_scan_ex(t, tx, None, ids, cnt, cfg=dyn)
        with torch.cuda.stream(s2):
            pm.pm_scan_ex(t, tx, None, ids2, cnt2, cfg=dyn)
    torch.cuda.synchronize()
    assert_same(ids.cpu().numpy(), int(cnt.item()), o_ids, o_cnt)
    assert_same(ids2.cpu().numpy(), int(cnt2.item()), o_ids, o_cnt)
    assert pm.pm_device_error() == pm.PM_OK


def test_scan_host_chunks():
    """pm_scan_host cuts the text into chunks that overlap by max_len-1; a
    match straddling the chunk boundary must be found."""
    pats = W.paper_scale(0, text_bytes=16, n_patterns=2000).patterns
    rng = np.random.Generator(np.random.MT19937(3))
    n = 70 * W.MiB + 123
    text = rng.integers(0, 256, size=n, dtype=np.uint8)
    p = np.frombuffer(pats.get(0), np.uint8)
    for cut in (32 * W.MiB, 64 * W.MiB):
        text[cut - len(p) // 2: cut - len(p) // 2 + len(p)] = p
    t = pm.pm_build(pats)
    h_text = torch.from_numpy(text).pin_memory()
    h_ids = torch.empty(n, dtype=torch.int32).pin_memory()
    cnt = pm.pm_scan_host(t, h_text.numpy(), h_ids.numpy())
    ids_d, cnt_d, _ = gpu_scan(t, text)
    assert cnt == cnt_d
    assert np.array_equal(h_ids.numpy(), ids_d)
    ot = oracle.Trie(pats)
    for cut in (32 * W.MiB, 64 * W.MiB):
        a, b = cut - 5000, cut + 5000
        o_ids, _, _ = ot.scan(text, a, b)
        assert np.array_equal(h_ids.numpy()[a:b], o_ids)
        assert h_ids.numpy()[cut - len(p) // 2] >= 0


# --------------------------------------------------------------------------
# full-size workloads, launch configuration of the benchmark


def sampled_windows(n, k, w, seed):
    rng = np.random.Generator(np.random.MT19937(seed))
    starts = np.sort(rng.integers(0, max(n - w, 1), size=k))
    return [(int(s), int(min(n, s + w))) for s in starts] + [(max(0, n - w), n)]


def check_windows(ot, text, ids, windows):
    for a, b in windows:
        o_ids, _, _ = ot.scan(text, a, b)
        bad = np.flatnonzero(ids[a:b] != o_ids)
        assert bad.size == 0, f"window {a}: {bad.size} mismatches"


def test_paper_scale_full_size():
    """Every one of the 268 M positions and the count, in the benchmark's
    launch configuration; sampled windows first for a quick failure report."""
    wl = W.paper_scale(0)
    t = pm.pm_build(wl.patterns)
    ids, cnt, _ = gpu_scan(t, wl.text)
    ot = oracle.Trie(wl.patterns)
    check_windows(ot, wl.text, ids, sampled_windows(len(wl.text), 48, 4096, 1))
    assert int((ids >= 0).sum()) >= 4096
    o_ids, o_cnt, _ = ot.scan(wl.text, threads=HOST_THREADS)
    assert_same(ids, cnt, o_ids, o_cnt)


def test_acgt_full_size():
    """Every one of the 1,074 M positions and the count (1 GiB ACGT text)."""
    wl = W.acgt(0)
    t = pm.pm_build(wl.patterns)
    ids, cnt, _ = gpu_scan(t, wl.text)
    ot = oracle.Trie(wl.patterns)
    check_windows(ot, wl.text, ids, sampled_windows(len(wl.text), 32, 4096, 2))
    o_ids, o_cnt, _ = ot.scan(wl.text, threads=HOST_THREADS)
    assert_same(ids, cnt, o_ids, o_cnt)
    del o_ids


def test_autotune_keeps_bits():
    """The autotuner only changes speed: its pick gives the oracle's bits."""
    from paper_1702_03657_gb300.tune import autotune
    wl = W.batched(4, ntexts=300, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    tx = dev(wl.text)
    off = dev(wl.offsets.astype(np.int64))
    res = autotune(t, tx, off, reps=2)
    assert res["tried"] >= 4
    assert pm.pm_get_config(t) == res["config"]
    o_ids, o_counts, _ = oracle.Trie(wl.patterns).scan_batch(wl.text, wl.offsets)
    ids, counts = batch_gpu(t, wl)
    assert np.array_equal(ids, o_ids) and np.array_equal(counts, o_counts)
