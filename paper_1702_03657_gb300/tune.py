"""Autotuner for the scan's launch configuration.

Times candidate `pm_config`s (threads per CTA, walker warps, text bytes per
warp tile, stages in flight, shared-memory filter level and width) on a
representative device input with CUDA events, keeps the fastest and installs
it on the handle with pm_set_config. Results can be cached in a JSON file
keyed by GPU name and trie shape (nodes, longest pattern, alphabet size, and
the input's size class). Every candidate computes the same bits; only speed
differs.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, Iterable, List, Optional

from . import pm


def candidates(trie: pm.Trie, total_bytes: int) -> List[dict]:
    st = pm.pm_stats(trie)
    base = pm.pm_get_config(trie)
    kmax = st["dense_k_max"]
    ks = sorted({kmax, max(kmax - 1, 0)})
    out = []
    for threads, tile, stages, k, bits, share in itertools.product(
            (1024, 512), (1024, 2048, 4096), (2, 3), ks, (8, 16, 32),
            ("2", "4", "8", "1/4", "1/2", "7/8")):
        # walker warps: a few (selective filters) up to most of the CTA
        # (tries whose filter passes most positions, e.g. DNA alphabets)
        warps = threads // 32
        walkers = int(share) if "/" not in share else \
            warps * int(share[0]) // int(share[2])
        if walkers >= warps or (share == "8" and walkers in (warps // 2, warps // 4)) or \
                (share == "4" and walkers == warps // 4):
            continue
        c = dict(base, threads=threads, tile=tile, stages=stages, dense_k=k,
                 filter_bits=bits, row_search=0, checked=0, ctas_per_sm=0,
                 walkers=walkers, deep=1 if st["deep_k"] else 0)
        try:
            pm.pm_set_config(trie, c)  # validates (shared memory, filter exists)
        except pm.PMError:
            continue
        out.append(c)
    pm.pm_set_config(trie, base)
    return out


def _time(run, reps: int) -> float:
    import torch
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _key(trie: pm.Trie, total_bytes: int, batch: bool) -> str:
    import torch
    st = pm.pm_stats(trie)
    size_class = max(total_bytes, 1).bit_length()
    return "|".join(str(x) for x in (torch.cuda.get_device_name(), st["n_nodes"],
                                      st["max_len"], st["alphabet"], size_class,
                                      int(batch)))


def autotune(trie: pm.Trie, texts, offsets=None, ids=None, counts=None,
             reps: int = 10, cache_path: Optional[str] = None,
             cands: Optional[Iterable[dict]] = None) -> Dict:
    """Pick the fastest configuration for this trie on this input (device
    tensors), install it, and return {"config", "ms", "tried"}."""
    import torch
    total = texts.numel()
    batch = offsets is not None
    key = _key(trie, total, batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            try:
                pm.pm_set_config(trie, cache[key]["config"])
                return dict(cache[key], cached=True)
            except pm.PMError:
                pass
    if ids is None:
        ids = torch.empty(total, dtype=torch.int32, device=texts.device)
    if counts is None:
        counts = torch.empty(offsets.numel() - 1 if batch else 1, dtype=torch.int64,
                             device=texts.device)
    best = None
    tried = 0
    for c in (list(cands) if cands is not None else candidates(trie, total)):
        def run(c=c):
            pm.pm_scan_ex(trie, texts, offsets, ids, counts, cfg=c)
        try:
            ms = _time(run, reps)
        except pm.PMError:
            continue
        tried += 1
        if best is None or ms < best[1]:
            best = (c, ms)
    if best is None:
        raise pm.PMError(pm.PM_ERR_INVAL, "autotune", "no valid configuration")
    pm.pm_set_config(trie, best[0])
    res = {"config": best[0], "ms": best[1], "tried": tried}
    if cache_path:
        cache[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
