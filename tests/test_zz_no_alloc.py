"""pm_scan_host_static, the host-buffer scan that allocates no device memory.

For callers that cannot let a library call cudaMalloc (device memory owned
by one allocator, or latency-sensitive request paths): the entry point
stages its text, ids and count in a static device array of libpm. Its
results must equal those of the device-buffer entry point pm_scan on the
same trie and text, call after call (the array keeps the previous call's
contents, which must not leak into the next result). Integer output, so the
comparison is exact. The entry point exists so that nothing is allocated on
the device: after one call has loaded the module that holds the static
array, further calls, the first on a freshly built trie included, leave the
device's free memory and torch's reserved memory unchanged.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

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


def scan_device(trie, text):
    """The existing entry point: pm_scan on device buffers."""
    tv = torch.from_numpy(text.copy()).cuda()
    ids = torch.empty(len(text), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    pm.pm_scan(trie, tv, ids, cnt)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), int(cnt.item())


def test_static_equals_device_scan_two_calls():
    wl = W.paper_scale(7, text_bytes=pm.PM_STATIC_MAX_LEN, n_patterns=4000)
    trie = pm.pm_build(wl.patterns)
    # a full-size text, then a shorter one with more matches: the second call
    # must not see the first call's ids or count
    rng = np.random.Generator(np.random.MT19937(11))
    second = rng.integers(0, 256, size=300_001, dtype=np.uint8)
    for j in range(0, len(second) - 64, 997):
        p = wl.patterns.get(int(rng.integers(0, wl.patterns.n)))
        second[j:j + len(p)] = np.frombuffer(p, np.uint8)
    for text in (wl.text, second):
        ids = np.full(len(text), -9, dtype=np.int32)
        cnt = pm.pm_scan_host_static(trie, text, ids)
        exp_ids, exp_cnt = scan_device(trie, text)
        assert cnt == exp_cnt
        assert np.array_equal(ids, exp_ids)
        assert cnt > 0
    # the second text against the CPU oracle as well
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(second, threads=8)
    assert cnt == o_cnt and np.array_equal(ids, o_ids)


def test_static_allocates_nothing():
    # one call loads the module that holds the static array (lazy loading)
    warm = pm.pm_build([b"abc", b"bcd"])
    w_text = np.frombuffer(b"abcdabcd" * 64, np.uint8).copy()
    pm.pm_scan_host_static(warm, w_text, np.empty(len(w_text), np.int32))
    wl = W.paper_scale(8, text_bytes=200_003, n_patterns=3000)
    trie = pm.pm_build(wl.patterns)
    exp_ids, exp_cnt = scan_device(trie, wl.text)   # loads the scan kernel
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(2):              # the first call on this trie, then another
        ids = np.full(len(wl.text), -9, dtype=np.int32)
        cnt = pm.pm_scan_host_static(trie, wl.text, ids)
        assert cnt == exp_cnt and np.array_equal(ids, exp_ids)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_reserved() == reserved0


def test_static_rejects_oversize():
    trie = pm.pm_build([b"abc"])
    text = np.zeros(pm.PM_STATIC_MAX_LEN + 1, dtype=np.uint8)
    ids = np.empty(len(text), dtype=np.int32)
    with pytest.raises(pm.PMError) as e:
        pm.pm_scan_host_static(trie, text, ids)
    assert e.value.code == pm.PM_ERR_INVAL
    assert "PM_STATIC_MAX_LEN" in str(e.value)
