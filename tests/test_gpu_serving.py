"""Serving with continuous batching (pm_server_*), on the GPU.

Each request's result in the mix must be bit-identical to scanning it alone
with pm_scan (integer output: exact), whatever batch it lands in, while the
scheduler admits requests by device memory and overlaps batches.
"""
import threading
import time

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


@pytest.fixture(scope="module")
def setup():
    pats = W.serving_patterns(0, n_patterns=8000)
    reqs = W.serving_requests(1, 240, pats, large=(64 << 10, 3 << 20), p_large=0.15)
    reqs.append(np.zeros(0, np.uint8))                          # empty request
    reqs.append(np.frombuffer(pats.get(3), np.uint8).copy())    # exactly a pattern
    trie = pm.pm_build(pats)
    return pats, reqs, trie


def alone(trie, text):
    n = len(text)
    tv = torch.from_numpy(text.copy()).cuda() if n else torch.zeros(1, dtype=torch.uint8, device="cuda")
    ids = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    pm.pm_scan(trie, tv, ids, cnt, length=n)
    torch.cuda.synchronize()
    return ids[:n].cpu().numpy(), int(cnt.item())


def outputs(reqs):
    ids = [torch.full((max(len(t), 1),), -9, dtype=torch.int32, device="cuda") for t in reqs]
    cnt = [torch.full((1,), -9, dtype=torch.int64, device="cuda") for _ in reqs]
    return ids, cnt


def test_same_alone_and_in_the_mix(setup):
    pats, reqs, trie = setup
    srv = pm.pm_server_create(trie, max_inflight=4)
    ids, cnt = outputs(reqs)
    rng = np.random.Generator(np.random.MT19937(4))
    rids = [None] * len(reqs)

    def client(lo, hi):
        for i in range(lo, hi):
            rids[i] = pm.pm_submit(srv, reqs[i], ids[i], cnt[i])
            if rng.random() < 0.2:
                time.sleep(0.0005)     # arrivals while earlier batches run

    half = len(reqs) // 2
    th = [threading.Thread(target=client, args=(0, half)),
          threading.Thread(target=client, args=(half, len(reqs)))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for r in rids:
        pm.pm_wait(srv, r, 20000)
    st = pm.pm_server_get_stats(srv)
    pm.pm_server_destroy(srv)
    assert st["completed"] == len(reqs)
    assert st["batches"] < len(reqs)          # requests were batched together
    for i, text in enumerate(reqs):
        exp_ids, exp_cnt = alone(trie, text)
        n = len(text)
        assert int(cnt[i].item()) == exp_cnt, i
        assert np.array_equal(ids[i][:n].cpu().numpy(), exp_ids), i
    # and a few against the oracle itself
    ot = oracle.Trie(pats)
    for i in range(0, len(reqs), 37):
        o_ids, o_cnt, _ = ot.scan(reqs[i])
        assert np.array_equal(ids[i][:len(reqs[i])].cpu().numpy(), o_ids)
        assert int(cnt[i].item()) == o_cnt


def test_admission_waits_for_device_memory(setup):
    pats, reqs, trie = setup
    big = [t for t in reqs if len(t) > (256 << 10)][:6]
    assert len(big) >= 3
    srv = pm.pm_server_create(trie, arena_bytes=max(len(t) for t in big) + 4096,
                              max_inflight=2)
    ids, cnt = outputs(big)
    rids = [pm.pm_submit(srv, t, ids[i], cnt[i]) for i, t in enumerate(big)]
    for r in rids:
        pm.pm_wait(srv, r, 20000)
    st = pm.pm_server_get_stats(srv)
    pm.pm_server_destroy(srv)
    assert st["admission_waits"] > 0          # arena too small for two at once
    for i, text in enumerate(big):
        exp_ids, exp_cnt = alone(trie, text)
        assert int(cnt[i].item()) == exp_cnt
        assert np.array_equal(ids[i][:len(text)].cpu().numpy(), exp_ids)


def test_replay_server_and_plain(setup):
    pats, reqs, trie = setup
    reqs = [t for t in reqs if len(t)]
    n = len(reqs)
    pinned = [torch.from_numpy(t.copy()).pin_memory() for t in reqs]
    hp = [p.data_ptr() for p in pinned]
    lens = [len(t) for t in reqs]
    arr = (W.poisson_arrivals(3, n, 20000.0) * 1e9).astype(np.uint64)
    ids_s, cnt_s = outputs(reqs)
    srv = pm.pm_server_create(trie)
    lat_s, wall_s = pm.pm_server_replay(srv, hp, lens, arr, [x.data_ptr() for x in ids_s],
                                        [x.data_ptr() for x in cnt_s])
    pm.pm_server_destroy(srv)
    ids_p, cnt_p = outputs(reqs)
    dtx = [torch.empty(len(t), dtype=torch.uint8, device="cuda") for t in reqs]
    lat_p, wall_p = pm.pm_replay_plain(trie, hp, lens, arr, [x.data_ptr() for x in dtx],
                                       [x.data_ptr() for x in ids_p],
                                       [x.data_ptr() for x in cnt_p])
    torch.cuda.synchronize()
    assert wall_s > 0 and wall_p > 0 and lat_s.min() > 0 and lat_p.min() > 0
    for i, text in enumerate(reqs):
        exp_ids, exp_cnt = alone(trie, text)
        for ids, cnt in ((ids_s, cnt_s), (ids_p, cnt_p)):
            assert int(cnt[i].item()) == exp_cnt
            assert np.array_equal(ids[i][:len(text)].cpu().numpy(), exp_ids)


def test_mixed_small_and_large_in_one_batch(setup):
    """Many small requests and several large ones submitted at once land in
    shared batches (small ones gathered through the staging buffer, large
    ones copied directly); every id and count must match the scan alone."""
    pats, reqs, trie = setup
    rng = np.random.Generator(np.random.MT19937(21))
    pool = rng.integers(0, 256, size=24 << 20, dtype=np.uint8)
    W._plant_bernoulli(rng, pool, pats, 1.0 / 1024)
    sizes = [int(x) for x in rng.integers(40, 1500, 400)] + [(2 << 20) + 7, (5 << 20) + 1,
                                                              70 << 10, 3 << 20]
    rng.shuffle(sizes)
    starts = [int(rng.integers(0, len(pool) - z)) for z in sizes]
    texts = [pool[a:a + z] for a, z in zip(starts, sizes)]
    ids, cnt = outputs(texts)
    srv = pm.pm_server_create(trie, max_inflight=1, max_batch=4096,
                              max_batch_bytes=64 << 20)
    rids = [pm.pm_submit(srv, t, ids[i], cnt[i]) for i, t in enumerate(texts)]
    for r in rids:
        pm.pm_wait(srv, r, 20000)
    st = pm.pm_server_get_stats(srv)
    pm.pm_server_destroy(srv)
    assert st["completed"] == len(texts) and st["max_batch_seen"] > 8
    for i, text in enumerate(texts):
        exp_ids, exp_cnt = alone(trie, text)
        assert int(cnt[i].item()) == exp_cnt, i
        assert np.array_equal(ids[i][:len(text)].cpu().numpy(), exp_ids), i


def test_server_errors(setup):
    pats, reqs, trie = setup
    host = pm.pm_build_host([b"abc"])
    with pytest.raises(pm.PMError) as e:
        pm.pm_server_create(host)
    assert e.value.code == pm.PM_ERR_HOST_ONLY
    srv = pm.pm_server_create(trie, arena_bytes=1 << 20)
    big = np.zeros((1 << 20) + 1, np.uint8)
    ids = torch.empty(len(big), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_submit(srv, big, ids, cnt)
    assert e.value.code == pm.PM_ERR_INVAL
    with pytest.raises(pm.PMError) as e:
        pm.pm_poll(srv, 123456789)
    assert e.value.code == pm.PM_ERR_NOT_FOUND
    pm.pm_server_destroy(srv)
