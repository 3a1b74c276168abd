"""The seeded generators: determinism and the stated shapes (no GPU)."""
import numpy as np

from paper_1702_03657_gb300 import workloads as W


def test_deterministic():
    a = W.tiny(0, text_bytes=64 * 1024)
    b = W.tiny(0, text_bytes=64 * 1024)
    c = W.tiny(1, text_bytes=64 * 1024)
    assert a.sha256() == b.sha256()
    assert a.sha256() != c.sha256()


def test_tiny_shape():
    wl = W.tiny(0, text_bytes=128 * 1024)
    L = wl.patterns.lengths()
    assert wl.patterns.n == 100 and L.min() >= 4 and L.max() <= 16
    assert len(set(wl.patterns.as_list())) == 100
    assert wl.text.min() >= ord("a") and wl.text.max() <= ord("z")
    # one plant per 4 KiB block: each block holds some pattern
    text = wl.text.tobytes()
    for b in range(len(text) // 4096):
        blk = text[b * 4096:(b + 1) * 4096]
        assert any(p in blk for p in wl.patterns.as_list())


def test_paper_scale_shape():
    wl = W.paper_scale(0, text_bytes=1 << 20, n_patterns=2000)
    pats = wl.patterns.as_list()
    L = wl.patterns.lengths()
    assert L.min() >= 8 and L.max() <= 64 and len(set(pats)) == len(pats)
    # about half the patterns share a prefix with an earlier one
    firsts = {}
    shared = 0
    for p in pats:
        shared += p[:2] in firsts
        firsts[p[:2]] = 1
    assert shared > 0.3 * len(pats)


def test_acgt_shape():
    wl = W.acgt(0, text_bytes=1 << 20, n_patterns=2000)
    assert set(np.unique(wl.text).tolist()) <= set(b"ACGT")
    L = wl.patterns.lengths()
    assert L.min() >= 20 and L.max() <= 32


def test_acgt_plant_overwrite_order():
    """Plants are applied left to right; the later plant wins an overlap."""
    pats = W.PatternSet.from_list([b"XXXX", b"YYYY"])
    text = np.zeros(64, np.uint8)

    class FixedRng:
        def random(self, n):
            r = np.ones(n)
            r[[3, 5]] = 0.0
            return r

        def integers(self, lo, hi, size):
            return np.array([0, 1])

    W._plant_bernoulli(FixedRng(), text, pats, 0.5)
    assert text[3:9].tobytes() == b"XXYYYY"


def test_batched_shape():
    wl = W.batched(0, ntexts=256, n_patterns=500)
    lens = np.diff(wl.offsets.astype(np.int64))
    assert lens.min() >= 64 and lens.max() <= 65536
    assert wl.offsets[-1] == len(wl.text)
    assert 700 < np.median(lens) < 3000
