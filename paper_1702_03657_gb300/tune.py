"""Autotuner for the scan's launch configuration.

Times candidate `pm_config`s on a representative device input with CUDA
events, keeps the fastest and installs it on the handle with pm_set_config.
The knobs: threads per CTA (the largest that fits, and smaller CTAs for
small inputs), text bytes per warp tile, tiles in flight per warp, start
positions per lane (4 or 8), the shared-memory filter level (and, for the
byte alphabet, its width), and the search of a CRS row's byte column
(linear or binary). Results can be cached in a JSON file keyed by GPU name
and trie shape (nodes, longest pattern, alphabet size, and the input's size
class). Every candidate computes the same bits; only speed differs.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, Iterable, List, Optional

from . import pm


def candidates(trie: pm.Trie, total_bytes: int, single: bool = False) -> List[dict]:
    """Valid configurations to time for an input of `total_bytes` bytes (a
    single text when `single`: short ones may also take the light form)."""
    st = pm.pm_stats(trie)
    base = pm.pm_get_config(trie)
    kmax = st["dense_k_max"]
    ks = sorted({kmax, max(kmax - 1, 0)})
    ident = st["alphabet"] == 256
    widths = (8, 16, 32) if ident else (8,)
    # small inputs cannot fill large CTAs: smaller ones launch and start faster
    threads = list(dict.fromkeys([base["threads"], 1024, 992, 896, 512] +
                                 ([256, 128] if total_bytes <= (4 << 20) else [])))
    tiles = (256, 1024, 2048) if total_bytes <= (4 << 20) else (512, 1024, 2048)
    lights = (0, 1 << 30) if single and total_bytes <= (1 << 20) else (0,)
    out, seen = [], set()
    for th, tile, stages, k, bits, pos, rs, lm in itertools.product(
            threads, tiles, (2, 3), ks, widths, (4, 8, 16), (0, 1), lights):
        c = dict(base, threads=th, tile=tile, stages=stages, dense_k=k, filter_bits=bits,
                 positions=pos, row_search=rs, checked=0, ctas_per_sm=0, layout=0,
                 wait_clocks=0, light_max=lm, schedule=0,
                 deep=0 if ident else (1 if st["deep_k"] else 0))
        key = tuple(sorted(c.items()))
        if key in seen:
            continue
        try:
            pm.pm_set_config(trie, c)  # validates (shared memory, filter, window)
        except pm.PMError:
            continue
        seen.add(key)
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
    for c in (list(cands) if cands is not None else candidates(trie, total, single=not batch)):
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
