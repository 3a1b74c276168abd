"""Sharded scans through pm_scan_range: one text cut into contiguous ranges
of start positions, each range scanned from its own device buffer holding
the range plus the longest pattern - 1 bytes after it (the overlap rule of
Section II-B), as one rank of a multi-GPU scan would. The ranges' ids
concatenate, and their counts add up, to the oracle's scan of the whole
text; bit-exact (integer output)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1702_03657_gb300 import dist as D
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


def plant_across(text, pats, cuts):
    """A pattern planted across every cut, so that walks cross each shard's
    end into its halo."""
    lens = pats.lengths()
    j = int(np.argmax(lens))
    p = np.frombuffer(pats.get(j), np.uint8)
    for c in cuts:
        a = max(0, c - len(p) // 2)
        text[a:a + len(p)] = p[:len(text) - a]


@pytest.mark.parametrize("world", [2, 3])
def test_halo_shards_recombine(world):
    for wl in (W.paper_scale(4, text_bytes=3 * W.MiB + 101, n_patterns=3000),
               W.acgt(4, text_bytes=2 * W.MiB + 33, n_patterns=20000)):
        text = wl.text.copy()
        n = len(text)
        max_len = int(wl.patterns.lengths().max())
        shards = [D.shard_text(n, max_len, r, world) for r in range(world)]
        plant_across(text, wl.patterns, [a for a, _, _ in shards[1:]])
        o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(text, threads=8)
        t = pm.pm_build(wl.patterns)
        ids_all, total = [], 0
        for a, b, limit in shards:
            buf = torch.from_numpy(text[a:limit].copy()).cuda()   # the rank's bytes only
            ids = torch.full((b - a,), -7, dtype=torch.int32, device="cuda")
            cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
            pm.pm_scan_range(t, buf, 0, b - a, limit - a, ids, cnt)
            torch.cuda.synchronize()
            ids_all.append(ids.cpu().numpy())
            total += int(cnt.item())
        got = np.concatenate(ids_all)
        bad = np.flatnonzero(got != o_ids)
        assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}"
        assert total == o_cnt


def test_ranges_of_one_device_text():
    """Ranges inside one device buffer: unaligned starts, a limit at the end
    of the range (walks cut there), an empty range."""
    wl = W.paper_scale(5, text_bytes=W.MiB + 17, n_patterns=2000)
    t = pm.pm_build(wl.patterns)
    tv = torch.from_numpy(wl.text).cuda()
    ot = oracle.Trie(wl.patterns)
    n = len(wl.text)
    for start, end, limit in ((0, n, n), (1, 4097, n), (333, 70001, 70001 + 63),
                              (70001, 70001, 70001), (5000, 9000, 9000), (n - 100, n, n)):
        ids = torch.full((max(end - start, 1),), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        pm.pm_scan_range(t, tv, start, end, limit, ids[:end - start], cnt)
        torch.cuda.synchronize()
        o_ids, o_cnt, _ = ot.scan(wl.text[:limit], start, end)
        assert np.array_equal(ids[:end - start].cpu().numpy(), o_ids)
        assert int(cnt.item()) == o_cnt
    with pytest.raises(pm.PMError):
        pm.pm_scan_range(t, tv, 10, 5, n, ids, cnt)
    with pytest.raises(pm.PMError):
        pm.pm_scan_range(t, tv, 0, 10, 5, ids, cnt)
