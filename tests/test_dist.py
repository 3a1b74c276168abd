"""Multi-rank host logic on CPU (gloo, world size 2): sharded scans of one
text and of a batch recombine to the whole scan; the count exchange and the
max-over-ranks timing. The per-rank scan here is the oracle's (no GPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1702_03657_gb300 import dist as D
from paper_1702_03657_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = D.dist_env()
        # one long text split by start positions, each rank reading a halo
        wl = W.random_case(3, 80, 50_003, 4, 2, 12, plant_rate=0.05)
        max_len = int(wl.patterns.lengths().max())
        a, b, limit = D.shard_text(len(wl.text), max_len, r, w)
        t = oracle.Trie(wl.patterns)
        ids, cnt, _ = t.scan(wl.text[:limit], a, b)
        total = D.sum_over_ranks(cnt)
        parts = D.gather_slices((a, b, ids), w)
        # a batch split by texts
        bw = W.batched(5, ntexts=64, n_patterns=500)
        t0, t1 = D.shard_texts(bw.offsets, r, w)
        bt = oracle.Trie(bw.patterns)
        lo, hi = int(bw.offsets[t0]), int(bw.offsets[t1])
        sub_off = bw.offsets[t0:t1 + 1].astype(np.int64) - lo
        _, counts, _ = bt.scan_batch(bw.text[lo:hi], sub_off)
        bparts = D.gather_slices((t0, t1, counts), w)
        slowest = D.max_over_ranks(1.0 + r)
        if r == 0:
            q.put(("ok", parts, total, bparts, slowest))
    except Exception as e:  # report, never hang the parent
        q.put(("error", repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_recombine():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
    assert res[0] == "ok", res
    _, parts, total, bparts, slowest = res
    import oracle
    wl = W.random_case(3, 80, 50_003, 4, 2, 12, plant_rate=0.05)
    full_ids, full_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text)
    assert total == full_cnt
    assert parts[0][0] == 0 and parts[0][1] == parts[1][0] and parts[1][1] == len(wl.text)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), full_ids)
    bw = W.batched(5, ntexts=64, n_patterns=500)
    _, full_counts, _ = oracle.Trie(bw.patterns).scan_batch(bw.text, bw.offsets)
    assert bparts[0][1] == bparts[1][0] and bparts[1][1] == 64
    assert np.array_equal(np.concatenate([p[2] for p in bparts]), full_counts)
    assert slowest == 2.0


def test_shard_bounds():
    for n in (0, 1, 7, 1000, 10**9 + 3):
        for world in (1, 2, 3, 8):
            spans = [D.shard_text(n, 64, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b, lim), nxt in zip(spans, spans[1:] + [(n, n, n)]):
                assert a <= b == nxt[0] and b <= lim <= min(n, b + 63)
    off = np.array([0, 10, 10, 500, 501, 2000])
    for world in (1, 2, 3, 5, 7):
        spans = [D.shard_texts(off, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == 5
        assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
