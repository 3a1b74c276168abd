"""Benchmark of the PFAC scan (one JSON line on rank 0).

A step is one pm_scan of the paper-scale workload: 20,000 byte patterns
(lengths 8-64, half of them sharing a prefix with an earlier one) over a
256 MiB uniform random text with one planted pattern per 64 KiB, text and
outputs resident in HBM. The metric is Gbps of text scanned (8 * bytes /
time), with the kernel's roofline fraction beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload paper|acgt|tiny]

The default workload is the paper-scale one; ``--workload acgt`` (100,000
patterns of 20-32 bytes over ACGT, 1 GiB text, 1 % planted) and ``tiny``
(100 patterns over 'a'-'z', 1 MiB) time the other plain configurations in
the same way, without the batched and serving legs.

Under torchrun each rank scans its own text (weak scaling, no data-path
collective); the step time is the max over ranks. ``--impl reference`` times
the CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbps scanned & % roofline, batched/served vs plain PFAC (bit-exact); p99 ms"
WORKLOAD = ("paper-scale plain PFAC: 20,000 patterns over bytes 0-255, lengths 8-64, "
            "p=0.5 shared prefix with an earlier pattern; 256 MiB uniform text, "
            "1 planted pattern per 64 KiB; seed 0")
N_PATTERNS = 20000
WORKLOADS = {
    "paper": (WORKLOAD, 256),
    "acgt": ("dense small alphabet plain PFAC: 100,000 patterns over ACGT, lengths 20-32; "
             "{mib} MiB i.i.d. uniform ACGT text, 1 % of positions start a planted "
             "pattern; seed 0", 1024),
    "tiny": ("tiny plain PFAC: 100 patterns over 'a'-'z', lengths 4-16; {mib} MiB text "
             "over 'a'-'z', one planted pattern per 4 KiB; seed 0", 1),
}


def make_workload(W, name: str, seed: int, mib: int):
    if name == "acgt":
        return W.acgt(seed, text_bytes=mib << 20)
    if name == "tiny":
        return W.tiny(seed, text_bytes=mib << 20)
    return W.paper_scale(seed, text_bytes=mib << 20, n_patterns=N_PATTERNS)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-all-matches", action="store_true")
    ap.add_argument("--no-streaming", action="store_true")
    ap.add_argument("--no-layouts", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--workload", default="paper", choices=sorted(WORKLOADS))
    ap.add_argument("--shard-text", action="store_true",
                    help="under torchrun: shard ONE text over the ranks (each scans its "
                         "range with a max_len-1 halo through pm_scan_range; strong scaling)")
    ap.add_argument("--text-mib", type=int, default=None,
                    help="text size (the metric is quoted at 256; smaller sizes "
                         "are for profiler captures)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------


def kernel_source_sha():
    """sha256 of the scan kernel's source (pm_scan.cu, pm_internal.h) with
    comments and blank lines removed: a profile stays valid across
    comment-only edits and is dropped by any change to the code."""
    h = hashlib.sha256()
    for f in ("pm_scan.cu", "pm_internal.h"):
        with open(os.path.join(ROOT, "paper_1702_03657_gb300", "csrc", f)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update("\n".join(l.rstrip() for l in txt.splitlines() if l.strip()).encode())
    return h.hexdigest()


def profiled_traffic(workload: str = "paper"):
    """DRAM bytes per launch from the committed ncu summary of the workload,
    if it was taken on the current kernel source (else None)."""
    name = {"paper": "pfac_scan_paper_scale.md", "acgt": "pfac_scan_acgt.md"}.get(workload)
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m1 = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    m2 = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not (m1 and m2) or m1.group(1) != kernel_source_sha():
        return None
    return float(m2.group(1))


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


L2_METHOD = ("torch copy between two L2-resident 40 MiB buffers, 50 copies per CUDA "
             "graph, read + write bytes over CUDA-event time, best of 5 replays")


def measured_l2_gbs(torch):
    """L2 bandwidth for the trie term (see L2_METHOD); no driver-measured
    figure exists for it."""
    a = torch.empty(40 << 20, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(5):
            b.copy_(a)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(50):
            b.copy_(a)
    g.replay()
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * a.numel() * 50 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del g
    return round(best, 1)


def cpu_baseline(wl, seconds: float, name: str = "256 MiB paper-scale"):
    """The oracle's PFAC walk, as it stands, on the host cores, over a
    bounded contiguous sample of the same text."""
    import oracle
    cores = os.cpu_count() or 1
    t = oracle.Trie(wl.patterns)
    probe = 1 << 18
    t0 = time.perf_counter()
    t.scan(wl.text, 0, probe, threads=cores)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    n = int(min(len(wl.text), max(probe, rate * seconds)))
    t0 = time.perf_counter()
    t.scan(wl.text, 0, n, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": round(8 * n / dt / 1e9, 4), "unit": "Gbps", "cores": cores,
            "kind": "oracle",
            "sample": f"start positions 0..{n} of the {name} text "
                      f"({n / len(wl.text) * 100:.2f}%), PFAC pointer-trie walk, "
                      f"{cores} threads, {dt:.1f} s"}


def bench_batched(pm, W, torch, reps: int):
    """Batched config: 4,096 texts scanned by one persistent launch over a
    device offset table, captured in a CUDA graph, against one pm_scan launch
    per text (host loop, and the same loop captured in a graph). Both must
    give identical ids and per-text counts."""
    from paper_1702_03657_gb300.tune import autotune
    wl = W.batched(0)
    trie = pm.pm_build(wl.patterns)
    total = len(wl.text)
    tx = torch.from_numpy(wl.text).cuda()
    off_h = wl.offsets.astype(np.int64)
    off = torch.from_numpy(off_h).cuda()
    nt = wl.ntexts
    ids_b = torch.empty(total, dtype=torch.int32, device="cuda")
    cnt_b = torch.empty(nt, dtype=torch.int64, device="cuda")
    tuned = autotune(trie, tx, off, ids_b, cnt_b, reps=20)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pm.pm_scan_batch(trie, tx, off, ids_b, cnt_b)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pm.pm_scan_batch(trie, tx, off, ids_b, cnt_b)

    # one launch per text, on its own handle tuned for one text of the
    # median length (the light launch form competes with the persistent one)
    trie_p = pm.pm_build(wl.patterns)
    lens = np.diff(off_h)
    med = int(np.argsort(lens)[len(lens) // 2])
    tv_med = tx[off_h[med]:off_h[med + 1]]
    tuned_p = autotune(trie_p, tv_med, None, reps=50)
    ids_l = torch.empty(total, dtype=torch.int32, device="cuda")
    cnt_l = torch.empty(nt, dtype=torch.int64, device="cuda")
    views = [(tx[off_h[t]:off_h[t + 1]], ids_l[off_h[t]:off_h[t + 1]], cnt_l[t:t + 1])
             for t in range(nt)]

    def loop():
        for tv, iv, cv in views:
            pm.pm_scan(trie_p, tv, iv, cv)

    with torch.cuda.stream(s):
        loop()
    torch.cuda.synchronize()
    gl = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gl, stream=s):
        loop()

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms_graph = timed(g.replay, reps)
    ms_loop = timed(loop, max(3, reps // 20))
    ms_loop_graph = timed(gl.replay, max(3, reps // 10))
    g.replay()
    gl.replay()
    torch.cuda.synchronize()
    mism = int((ids_b != ids_l).sum().item()) + int((cnt_b != cnt_l).sum().item())
    gb = lambda ms: round(8.0 * total / (ms / 1e3) / 1e9, 2)
    return {"workload": f"{nt} texts, {total} bytes, lengths log-normal median 1536 clipped "
                        f"64..65536, 10,000 patterns of 8-48 bytes, 1 plant per 2 KiB",
            "persistent_graph_gbps": gb(ms_graph), "persistent_graph_ms": round(ms_graph, 4),
            "per_text_loop_gbps": gb(ms_loop), "per_text_loop_ms": round(ms_loop, 3),
            "per_text_loop_in_graph_gbps": gb(ms_loop_graph),
            "per_text_loop_in_graph_ms": round(ms_loop_graph, 3),
            "per_text_device_us": round(ms_loop_graph / nt * 1e3, 2),
            "speedup_vs_loop": round(ms_loop / ms_graph, 1),
            "speedup_vs_loop_in_graph": round(ms_loop_graph / ms_graph, 1),
            "mismatches": mism, "matches": int(cnt_b.sum().item()),
            "tuned_config": tuned["config"], "configs_tried": tuned["tried"],
            "per_text_tuned_config": tuned_p["config"],
            "per_text_configs_tried": tuned_p["tried"],
            "per_text_form": "light" if tuned_p["config"]["light_max"] >= int(lens.max())
                             else "persistent"}


def bench_serving(pm, W, torch, n_req: int, loads=(0.1, 0.25, 0.5, 0.75, 0.9)):
    """Serving config: 50,000 byte patterns (6-64 B); requests 90 % U[40,1500]
    B and 10 % log-uniform [1,16] MiB of uniform bytes with plants at 1 per
    2 KiB, arriving as a Poisson process. Each request's text is a slice of
    one pinned pool (so the trace needs no per-request host buffers). The
    continuous-batching server and plain per-request launches replay the same
    traces natively; latency = completion seen on the host - scheduled
    arrival."""
    pats = W.serving_patterns(0)
    trie = pm.pm_build(pats)
    rng = np.random.Generator(np.random.MT19937(7))
    large = rng.random(n_req) < 0.1
    sizes = np.where(large,
                     np.exp(rng.uniform(np.log(1 << 20), np.log(16 << 20), n_req)).astype(np.int64),
                     rng.integers(40, 1501, n_req))
    pool_n = (96 << 20)
    pool = rng.integers(0, 256, size=pool_n, dtype=np.uint8)
    W._plant_bernoulli(rng, pool, pats, 1.0 / 2048)
    pool_t = torch.from_numpy(pool).pin_memory()
    starts = rng.integers(0, pool_n - sizes + 1)
    h_ptrs = [pool_t.data_ptr() + int(o) for o in starts]
    lens = [int(x) for x in sizes]
    total = int(sizes.sum())
    out_off = np.concatenate([[0], np.cumsum(sizes)])
    ids_s = torch.empty(total, dtype=torch.int32, device="cuda")
    ids_p = torch.empty(total, dtype=torch.int32, device="cuda")
    cnt_s = torch.empty(n_req, dtype=torch.int64, device="cuda")
    cnt_p = torch.empty(n_req, dtype=torch.int64, device="cuda")
    dtx = torch.empty(total, dtype=torch.uint8, device="cuda")
    ip_s = [ids_s.data_ptr() + 4 * int(o) for o in out_off[:-1]]
    ip_p = [ids_p.data_ptr() + 4 * int(o) for o in out_off[:-1]]
    cp_s = [cnt_s.data_ptr() + 8 * i for i in range(n_req)]
    cp_p = [cnt_p.data_ptr() + 8 * i for i in range(n_req)]
    tp = [dtx.data_ptr() + int(o) for o in out_off[:-1]]
    srv = pm.pm_server_create(trie)

    def gbps(nbytes, ns):
        return 8.0 * nbytes / max(ns, 1)

    def run(arr):
        lat_s, wall_s = pm.pm_server_replay(srv, h_ptrs, lens, arr, ip_s, cp_s)
        lat_p, wall_p = pm.pm_replay_plain(trie, h_ptrs, lens, arr, tp, ip_p, cp_p)
        torch.cuda.synchronize()
        q = lambda lat, p_: round(float(np.percentile(lat, p_)) / 1e6, 4)
        return {"server": {"gbps": round(gbps(total, wall_s), 2), "p50_ms": q(lat_s, 50),
                           "p99_ms": q(lat_s, 99)},
                "plain": {"gbps": round(gbps(total, wall_p), 2), "p50_ms": q(lat_p, 50),
                          "p99_ms": q(lat_p, 99)}}

    zero = np.zeros(n_req, dtype=np.uint64)
    run(zero)                                   # warm-up
    sat = run(zero)                             # everything arrives at once
    max_gbps = sat["server"]["gbps"]
    mean_bytes = total / n_req
    points = []
    for f in loads:
        rate = f * max_gbps * 1e9 / 8 / mean_bytes          # requests per second
        arr = (W.poisson_arrivals(11, n_req, rate) * 1e9).astype(np.uint64)
        r = run(arr)
        r["offered_gbps"] = round(f * max_gbps, 2)
        r["load"] = f
        points.append(r)
    mism = int((ids_s != ids_p).sum().item()) + int((cnt_s != cnt_p).sum().item())
    st = pm.pm_server_get_stats(srv)
    pm.pm_server_destroy(srv)
    return {"workload": f"{n_req} requests, {total} bytes, 90 % U[40,1500] B / 10 % "
                        f"log-uniform [1,16] MiB, 50,000 patterns of 6-64 B, Poisson arrivals",
            "saturation": sat, "max_served_gbps": max_gbps, "points": points,
            "mismatches_server_vs_plain": mism,
            "server_stats": {k: st[k] for k in ("batches", "max_batch_seen",
                                                "max_inflight_seen", "admission_waits")}}


def run_reference(args, rank, world):
    """CPU oracle arm: rank 0 only; each step a bounded sample."""
    if rank != 0:
        return
    from paper_1702_03657_gb300 import workloads as W
    import oracle
    desc, def_mib = WORKLOADS[args.workload]
    mib = args.text_mib or def_mib
    wl = make_workload(W, args.workload, 0, mib)
    cores = os.cpu_count() or 1
    t = oracle.Trie(wl.patterns)
    probe = 1 << 18
    t0 = time.perf_counter()
    t.scan(wl.text, 0, probe, threads=cores)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    budget = 90.0
    per_step = int(max(4096, min(len(wl.text) // 2, rate * budget / max(1, args.steps + args.warmup))))
    rng = np.random.Generator(np.random.MT19937(1))
    starts = rng.integers(0, len(wl.text) - per_step, size=args.steps + args.warmup)
    for i in range(args.warmup):
        t.scan(wl.text, int(starts[i]), int(starts[i]) + per_step, threads=cores)
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        t.scan(wl.text, int(starts[i]), int(starts[i]) + per_step, threads=cores)
    dt = time.perf_counter() - t0
    value = 8 * per_step * args.steps / dt / 1e9
    sample = (f"{per_step} consecutive start positions per step at seeded random offsets "
              f"of the {mib} MiB {args.workload} text; PFAC pointer-trie walk on "
              f"{cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gbps",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc.format(mib=mib), "sample_positions_per_step": per_step},
            "cpu_baseline": {"value": round(value, 4), "unit": "Gbps", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Gbps", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    from paper_1702_03657_gb300.dist import dist_env, max_over_ranks
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_1702_03657_gb300 import pm
    from paper_1702_03657_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pm.load()

    desc, def_mib = WORKLOADS[args.workload]
    mib = args.text_mib or def_mib
    shard = args.shard_text and world > 1
    # shard mode: every rank draws the same text and scans its own range of
    # start positions (plus the halo its walks may read); otherwise each rank
    # scans its own text
    wl = make_workload(W, args.workload, 0 if shard else rank, mib)
    trie = pm.pm_build(wl.patterns)
    stats = pm.pm_stats(trie)
    cfg = pm.pm_get_config(trie)
    if shard:
        from paper_1702_03657_gb300.dist import shard_text, sum_over_ranks
        n_full = len(wl.text)
        a, b, limit = shard_text(n_full, int(stats["max_len"]), rank, world)
        wl.text = np.ascontiguousarray(wl.text[a:limit])
        n = b - a
        for flag in ("no_batched", "no_serving", "no_all_matches", "no_streaming", "no_layouts",
                     "no_cpu_baseline"):
            setattr(args, flag, True)
        args.e2e_steps = 0
    else:
        n = len(wl.text)
    text = torch.from_numpy(wl.text).cuda()
    ids = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def scan():
        if shard:
            pm.pm_scan_range(trie, text, 0, n, text.numel(), ids[:n], cnt)
        else:
            pm.pm_scan(trie, text, ids, cnt)

    # trie-lookup count (instrumented kernel, outside the timed region) on
    # the first 1 MiB of the text, scaled to the whole text
    look_n = min(n, 1 << 20)
    look = torch.zeros(1, dtype=torch.int64, device="cuda")
    pm.pm_scan_ex(trie, text, None, ids, cnt, lookups=look, length=look_n)
    torch.cuda.synchronize()
    lookups = int(look.item()) * n // look_n

    for _ in range(max(args.warmup, 3)):
        scan()
    torch.cuda.synchronize()

    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(K):
        scan()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    total_ms = max_over_ranks(total_ms, "cuda")
    count = int(cnt.item())
    if shard:
        count = sum_over_ranks(count, "cuda")   # the one exchange: 8 bytes
        gbps = 8.0 * n_full * K / (total_ms / 1e3) / 1e9
    else:
        gbps = 8.0 * n * world * K / (total_ms / 1e3) / 1e9
    avg_launch_s = statistics.mean(step_ms) / 1e3
    alg_bytes = n + 4 * n + 8                   # text read + int32 ids + count
    achieved = alg_bytes / avg_launch_s / 1e9   # GB/s
    peak, peak_kind = measured_peak_hbm()
    traffic = profiled_traffic(args.workload) if mib == def_mib else None
    # trie term: 4 bytes per transition the oracle attempts, at L2 bandwidth
    # the oracle's root walks need lookups; the kernel's dense levels, filter
    # and deep level skip most of them, so the HBM term is the one its
    # traffic follows (the roofline object); both terms are reported
    l2 = measured_l2_gbs(torch)
    trie_bytes = 4 * lookups
    t_hbm, t_trie = alg_bytes / (peak * 1e9), trie_bytes / (l2 * 1e9)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind}

    # end to end through the C ABI with host buffers (pm_scan_host)
    e2e = None
    if args.e2e_steps > 0:
        h_text = torch.from_numpy(wl.text).pin_memory()
        h_ids = torch.empty(n, dtype=torch.int32).pin_memory()
        hn, hi = h_text.numpy(), h_ids.numpy()
        hc = pm.pm_scan_host(trie, hn, hi)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            hc = pm.pm_scan_host(trie, hn, hi)
        e2e_s = max(time.perf_counter() - t0, 1e-9)
        e2e_s = max_over_ranks(e2e_s, "cuda")
        chunk = 32 << 20
        nchunks = (n + chunk - 1) // chunk
        h2d = n + (nchunks - 1) * (stats["max_len"] - 1)
        d2h = 4 * n + 8 * nchunks
        e2e = {"value": round(8.0 * n * world * args.e2e_steps / e2e_s / 1e9, 2), "unit": "Gbps",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "pm_scan_host (pinned host text in, host ids + count out)"}
        assert hc == count, "pm_scan_host count differs from pm_scan"

    # the same scan with walks over the paper's bitmapped nodes (Section III:
    # 256-bit child bitmap + first child, 36 bytes a node) instead of the
    # 16-byte CRS row records
    bitmap_nodes = None
    if not args.no_layouts:
        cfg_bm = dict(cfg, layout=1)
        for _ in range(3):
            pm.pm_scan_ex(trie, text, None, ids, cnt, cfg=cfg_bm)
        torch.cuda.synchronize()
        Kb = max(1, min(K, 200))
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record(stream)
        for _ in range(Kb):
            pm.pm_scan_ex(trie, text, None, ids, cnt, cfg=cfg_bm)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = max_over_ranks(e0.elapsed_time(e1) / Kb, "cuda")
        assert int(cnt.item()) == count, "bitmapped-node count differs"
        nn = int(stats["n_nodes"])
        bitmap_nodes = {"gbps": round(8.0 * n * world / (ms_b / 1e3) / 1e9, 2),
                        "ms_per_step": round(ms_b, 5), "steps": Kb,
                        "node_bytes": 36 * nn, "row_record_bytes": 16 * nn,
                        "csr_bytes": int(stats["csr_bytes"])}

    # the truncated levels as an exact prefilter: walks queued vs positions
    prefilter = None
    if not shard:
        wk = torch.zeros(1, dtype=torch.int64, device="cuda")
        pm.pm_scan_walks(trie, text, ids, cnt, wk)
        torch.cuda.synchronize()
        walks = int(wk.item())
        prefilter = {"walks": walks, "walks_per_position": round(walks / max(n, 1), 6),
                     "settled_without_walk": round(1.0 - walks / max(n, 1), 6),
                     "matched_positions_walked": True}

    # every occurrence (pm_scan_all): the same scan plus the ordered list
    all_matches = None
    if not args.no_all_matches:
        cap = count + 1024
        mt = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
        work = torch.empty(pm.pm_scan_all_work_bytes(n), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            pm.pm_scan_all(trie, text, ids, cnt, mt, work)
        torch.cuda.synchronize()
        Ka = max(1, min(K, 200))
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record(stream)
        for _ in range(Ka):
            pm.pm_scan_all(trie, text, ids, cnt, mt, work)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_all = max_over_ranks(e0.elapsed_time(e1) / Ka, "cuda")
        assert int(cnt.item()) == count, "pm_scan_all count differs from pm_scan"
        all_matches = {"gbps": round(8.0 * n * world / (ms_all / 1e3) / 1e9, 2),
                       "ms_per_step": round(ms_all, 5), "matches": count,
                       "list_bytes": 16 * count, "steps": Ka,
                       "overhead_vs_scan": round(ms_all / (total_ms / K) - 1.0, 4),
                       "api": "pm_scan_all (ids + count + every occurrence, position "
                              "order, longest first)"}

    # every occurrence with host buffers (pm_scan_all_host): only the list
    # comes back, 16 bytes per occurrence instead of 4 bytes per position
    all_matches_host = None
    if not args.no_all_matches and args.e2e_steps > 0:
        hm = np.zeros((count + 16, 2), dtype=np.int64)
        hm_t = torch.from_numpy(hm).pin_memory()
        hm = hm_t.numpy()
        assert pm.pm_scan_all_host(trie, hn, hm) == count
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            got = pm.pm_scan_all_host(trie, hn, hm)
        ah_s = max_over_ranks(max(time.perf_counter() - t0, 1e-9), "cuda")
        assert got == count, "pm_scan_all_host count differs from pm_scan"
        all_matches_host = {
            "value": round(8.0 * n * world * args.e2e_steps / ah_s / 1e9, 2), "unit": "Gbps",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * count + 8 * nchunks,
            "api": "pm_scan_all_host (pinned host text in, host list of every occurrence out)"}

    # the same text as a stream of chunks (pm_scanner_*), device-resident
    streaming = None
    if not args.no_streaming:
        streaming = []
        H = max(int(stats["max_len"]) - 1, 0)
        for chunk in (1 << 20, 64 << 10):
            sc = pm.pm_scanner_open(trie)
            sids = torch.empty(chunk + H + 1, dtype=torch.int32, device="cuda")
            scnt = torch.empty(1, dtype=torch.int64, device="cuda")
            acc = torch.zeros(1, dtype=torch.int64, device="cuda")

            def one_stream():
                for a in range(0, n, chunk):
                    sc.push(text[a:a + chunk], sids, scnt)
                    acc.add_(scnt)
                sc.finish(sids, scnt)
                acc.add_(scnt)
            one_stream()
            torch.cuda.synchronize()
            acc.zero_()
            reps = 3
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(stream)
            for _ in range(reps):
                one_stream()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s = max_over_ranks(e0.elapsed_time(e1) / reps, "cuda")
            ok_count = int(acc.item()) == reps * count
            # the same stream captured once in a CUDA graph (device time
            # without the Python loop; each replay starts from an empty carry)
            g = torch.cuda.CUDAGraph()
            gs = torch.cuda.Stream()
            gs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(gs):
                with torch.cuda.graph(g, stream=gs):
                    one_stream()
            torch.cuda.current_stream().wait_stream(gs)
            acc.zero_()
            g.replay()
            torch.cuda.synchronize()
            ok_graph = int(acc.item()) == count
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_g = max_over_ranks(e0.elapsed_time(e1) / reps, "cuda")
            del g
            streaming.append({"chunk_bytes": chunk, "pushes": (n + chunk - 1) // chunk,
                              "gbps": round(8.0 * n * world / (ms_s / 1e3) / 1e9, 2),
                              "ms_per_stream": round(ms_s, 4),
                              "gbps_graph": round(8.0 * n * world / (ms_g / 1e3) / 1e9, 2),
                              "ms_per_stream_graph": round(ms_g, 4),
                              "count_equal": ok_count and ok_graph,
                              "loop": "Python loop over pm_scanner_push; graph: the same "
                                      "pushes captured once and replayed"})
            sc.close()
            assert ok_count and ok_graph, "streamed count differs from pm_scan"

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(wl, args.cpu_seconds, f"{mib} MiB {args.workload}")
    other = args.workload != "paper"
    batched = None if args.no_batched or other else bench_batched(pm, W, torch, reps=200)
    serving = None if args.no_serving or other else \
        bench_serving(pm, W, torch, args.serving_requests)
    line = {
        "metric": METRIC, "value": round(gbps, 2), "unit": "Gbps", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(total_ms / K, 5),
        "higher_is_better": True, "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": desc.format(mib=mib), "text_bytes": n,
                   "patterns": int(stats["n_patterns"]),
                   "launch": cfg,
                   "l2": (f"inputs larger than L2 ({mib} MiB text + {4 * mib} MiB ids per "
                          "step), no flush") if 5 * mib > 126 else
                         f"inputs ({5 * mib} MiB) fit in L2: not a roofline claim",
                   "parallelism": (f"one text sharded over {world} ranks (pm_scan_range, "
                                   f"max_len-1 halo, count summed)") if shard else
                                  f"independent text per rank x{world}"},
        "roofline": dict(roof, **{
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "hbm_term": {"bytes": alg_bytes, "peak_gbs": peak,
                                  "bound_ms": round(t_hbm * 1e3, 4)},
                     "trie_term": {"lookups": lookups,
                                   "lookups_per_byte": round(lookups / n, 4),
                                   "bytes": trie_bytes, "l2_gbs": l2, "l2_method": L2_METHOD,
                                   "bound_ms": round(t_trie * 1e3, 4),
                                   "sample": f"counted on the first {look_n} bytes, scaled"},
                     "two_term": {"binding": "hbm" if t_hbm >= t_trie else "trie",
                                  "frac_of_time": round(max(t_hbm, t_trie) / avg_launch_s, 4),
                                  "rule": "max(hbm bytes / HBM peak, 4 B x oracle lookups / "
                                          "L2 bandwidth) / kernel time"}}),
        "e2e": e2e,
        "e2e_all_matches_host": all_matches_host,
        "gpu_launches": K,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
        "trie": {k: stats[k] for k in ("n_nodes", "nnz", "csr_bytes", "dense256_bytes",
                                       "bitmap36_bytes", "crs_elements", "alphabet",
                                       "dense_k_max", "deep_k", "deep_bytes",
                                       "device_bytes")},
        "matches": count,
        "all_matches": all_matches,
        "bitmap_nodes": bitmap_nodes,
        "prefilter": prefilter,
        "streaming": streaming,
        "batched": batched,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
