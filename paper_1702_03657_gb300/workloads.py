"""Seeded synthetic workloads for the PFAC scan (patterns + texts).

This module only draws random bytes. It holds no trie, no matching and no
other part of the scan's arithmetic, so both the CUDA path and the CPU oracle
can be fed from it without sharing any of the method.

The paper evaluates on the King James Bible with patterns picked from the text
by a Mersenne Twister (Section V); that text is not available here, so seeded
synthetic inputs of the shapes below stand in for it. Every generator draws
from ``numpy.random.Generator(MT19937(seed))``.

Workloads (sizes are defaults; tests pass smaller ones):

* ``tiny``        100 patterns, lengths U[4,16] over 'a'..'z', deduplicated;
                  1 MiB text over 'a'..'z', one pattern planted per 4 KiB block.
* ``paper_scale`` 20,000 patterns over bytes 0..255, lengths U[8,64]; with
                  probability 1/2 a pattern starts with a prefix (length
                  U[1, min(len, len_j) - 1]) of a uniformly chosen earlier
                  pattern j; deduplicated. 256 MiB uniform text, one pattern
                  planted per 64 KiB block.
* ``acgt``        100,000 patterns over {A,C,G,T}, lengths U[20,32],
                  deduplicated; 1 GiB i.i.d. ACGT text in which every position
                  starts a planted pattern with probability 0.01 (plants are
                  applied left to right; a later plant overwrites an earlier
                  one where they overlap).
* ``batched``     10,000 byte patterns, lengths U[8,48]; 4,096 texts with
                  length clip(round(LogNormal(ln 1536, 1.0)), 64, 65536) of
                  uniform bytes, concatenated, with a plant starting at each
                  byte with probability 1/2048 (kept only if it fits in its
                  text).
* ``serving``     50,000 byte patterns, lengths U[6,64]; requests of which 90%
                  are U[40,1500] bytes and 10% log-uniform in [1,16] MiB,
                  uniform bytes with plants at rate 1/2048 per byte; Poisson
                  arrival times for a given offered rate.
"""
from __future__ import annotations

import dataclasses
import hashlib
from typing import List, Optional

import numpy as np

KiB = 1024
MiB = 1024 * 1024
GiB = 1024 * MiB

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.MT19937(seed))


@dataclasses.dataclass
class PatternSet:
    """Patterns packed back to back: pattern j is data[off[j]:off[j+1]]."""

    data: np.ndarray  # uint8
    off: np.ndarray   # int64, n+1

    @property
    def n(self) -> int:
        return len(self.off) - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.off).astype(np.uint32)

    def get(self, j: int) -> bytes:
        return self.data[self.off[j]:self.off[j + 1]].tobytes()

    def as_list(self) -> List[bytes]:
        return [self.get(j) for j in range(self.n)]

    @staticmethod
    def from_list(pats: List[bytes]) -> "PatternSet":
        lens = np.array([len(p) for p in pats], dtype=np.int64)
        off = np.zeros(len(pats) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        data = np.frombuffer(b"".join(pats), dtype=np.uint8).copy()
        return PatternSet(data, off)

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(self.off.astype("<i8").tobytes())
        h.update(self.data.tobytes())
        return h.hexdigest()


@dataclasses.dataclass
class Workload:
    name: str
    seed: int
    patterns: PatternSet
    text: np.ndarray                      # uint8, all texts concatenated
    offsets: Optional[np.ndarray] = None  # uint64, ntexts+1 (batched only)

    @property
    def ntexts(self) -> int:
        return 1 if self.offsets is None else len(self.offsets) - 1

    def sha256(self) -> str:
        h = hashlib.sha256(self.patterns.sha256().encode())
        h.update(self.text.tobytes())
        if self.offsets is not None:
            h.update(self.offsets.astype("<u8").tobytes())
        return h.hexdigest()


# --------------------------------------------------------------------------
# pattern generators
# --------------------------------------------------------------------------

def _unique_patterns(rng, n, lo, hi, alphabet=None, prefix_share=0.0):
    """n distinct random patterns, lengths U[lo,hi]; a duplicate is redrawn."""
    seen = set()
    out: List[bytes] = []
    while len(out) < n:
        L = int(rng.integers(lo, hi + 1))
        if alphabet is None:
            body = rng.integers(0, 256, size=L, dtype=np.uint8)
        else:
            body = alphabet[rng.integers(0, len(alphabet), size=L)]
        if prefix_share > 0.0 and out and rng.random() < prefix_share:
            j = int(rng.integers(0, len(out)))
            m = min(L, len(out[j])) - 1
            if m >= 1:
                k = int(rng.integers(1, m + 1))
                body = body.copy()
                body[:k] = np.frombuffer(out[j][:k], dtype=np.uint8)
        p = body.tobytes()
        if p in seen:
            continue
        seen.add(p)
        out.append(p)
    return PatternSet.from_list(out)


def _plant_per_block(rng, text, pats: PatternSet, block):
    """One uniformly chosen pattern per block at a uniform offset inside it."""
    lens = pats.lengths()
    nblk = len(text) // block
    for b in range(nblk):
        j = int(rng.integers(0, pats.n))
        L = int(lens[j])
        if L > block:
            continue
        o = b * block + int(rng.integers(0, block - L + 1))
        text[o:o + L] = pats.data[pats.off[j]:pats.off[j + 1]]


def _plant_bernoulli(rng, text, pats: PatternSet, rate, bounds=None):
    """A plant starts at each byte with probability ``rate``; plants are applied
    in increasing start order, a later plant overwriting an earlier one.

    ``bounds`` (optional, sorted text offsets) confines each plant to its own
    text; a plant that would cross its text's end is dropped.
    """
    n = len(text)
    if n == 0 or pats.n == 0:
        return
    starts = np.flatnonzero(rng.random(n) < rate)
    if len(starts) == 0:
        return
    which = rng.integers(0, pats.n, size=len(starts))
    lens = pats.lengths()[which].astype(np.int64)
    ends = starts + lens
    if bounds is None:
        keep = ends <= n
    else:
        t = np.searchsorted(bounds, starts, side="right") - 1
        keep = ends <= bounds[t + 1]
    starts, which, lens = starts[keep], which[keep], lens[keep]
    if len(starts) == 0:
        return
    maxl = int(lens.max())
    # Byte o of a plant lands at start+o. Writing offsets from the largest to
    # the smallest leaves, at each byte, the plant with the largest start that
    # covers it, i.e. the left-to-right overwrite order; within one offset the
    # target indices are distinct, so each assignment is well defined.
    src0 = pats.off[which]
    for o in range(maxl - 1, -1, -1):
        sel = lens > o
        text[starts[sel] + o] = pats.data[src0[sel] + o]


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def tiny(seed: int = 0, text_bytes: int = 1 * MiB, n_patterns: int = 100) -> Workload:
    rng = rng_for(seed)
    alpha = np.arange(ord("a"), ord("z") + 1, dtype=np.uint8)
    pats = _unique_patterns(rng, n_patterns, 4, 16, alphabet=alpha)
    text = alpha[rng.integers(0, 26, size=text_bytes)]
    _plant_per_block(rng, text, pats, 4 * KiB)
    return Workload("tiny", seed, pats, text)


def paper_scale(seed: int = 0, text_bytes: int = 256 * MiB,
                n_patterns: int = 20000) -> Workload:
    rng = rng_for(seed)
    pats = _unique_patterns(rng, n_patterns, 8, 64, prefix_share=0.5)
    text = rng.integers(0, 256, size=text_bytes, dtype=np.uint8)
    _plant_per_block(rng, text, pats, 64 * KiB)
    return Workload("paper_scale", seed, pats, text)


def acgt(seed: int = 0, text_bytes: int = 1 * GiB, n_patterns: int = 100000,
         plant_rate: float = 0.01) -> Workload:
    rng = rng_for(seed)
    pats = _unique_patterns(rng, n_patterns, 20, 32, alphabet=ACGT)
    text = ACGT[rng.integers(0, 4, size=text_bytes, dtype=np.uint8)]
    _plant_bernoulli(rng, text, pats, plant_rate)
    return Workload("acgt", seed, pats, text)


def batched(seed: int = 0, ntexts: int = 4096, n_patterns: int = 10000,
            median: float = 1536.0, sigma: float = 1.0,
            min_len: int = 64, max_len: int = 65536) -> Workload:
    rng = rng_for(seed)
    pats = _unique_patterns(rng, n_patterns, 8, 48)
    lens = np.clip(np.round(rng.lognormal(np.log(median), sigma, size=ntexts)),
                   min_len, max_len).astype(np.int64)
    offsets = np.zeros(ntexts + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    total = int(offsets[-1])
    text = rng.integers(0, 256, size=total, dtype=np.uint8)
    _plant_bernoulli(rng, text, pats, 1.0 / 2048, bounds=offsets.astype(np.int64))
    return Workload("batched", seed, pats, text, offsets)


def serving_patterns(seed: int = 0, n_patterns: int = 50000) -> PatternSet:
    return _unique_patterns(rng_for(seed), n_patterns, 6, 64)


def serving_requests(seed: int, n_requests: int, pats: PatternSet,
                     small=(40, 1500), large=(1 * MiB, 16 * MiB),
                     p_large: float = 0.1) -> List[np.ndarray]:
    """Request texts: 90% packet-sized U[40,1500] B, 10% log-uniform in
    [1,16] MiB; uniform bytes with plants at rate 1/2048 per byte."""
    rng = rng_for(seed + 1000003)
    out = []
    for _ in range(n_requests):
        if rng.random() < p_large:
            size = int(np.exp(rng.uniform(np.log(large[0]), np.log(large[1]))))
        else:
            size = int(rng.integers(small[0], small[1] + 1))
        t = rng.integers(0, 256, size=size, dtype=np.uint8)
        _plant_bernoulli(rng, t, pats, 1.0 / 2048)
        out.append(t)
    return out


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = rng_for(seed + 2000003)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def concat(texts: List[np.ndarray]):
    """Concatenate texts; returns (bytes, offsets u64[n+1])."""
    offsets = np.zeros(len(texts) + 1, dtype=np.uint64)
    np.cumsum([len(t) for t in texts], out=offsets[1:])
    data = np.concatenate(texts) if texts else np.zeros(0, np.uint8)
    return data, offsets


def random_case(seed: int, n_patterns: int, text_bytes: int, alphabet: int,
                lo: int = 1, hi: int = 8, plant_rate: float = 0.05) -> Workload:
    """Small random case over the first ``alphabet`` byte values, for parity
    and brute-force checks (short patterns give many overlapping matches)."""
    rng = rng_for(seed)
    alpha = np.arange(alphabet, dtype=np.uint8) + (ord("a") if alphabet <= 26 else 0)
    n_patterns = min(n_patterns, sum(alphabet ** L for L in range(lo, hi + 1)))
    pats = _unique_patterns(rng, n_patterns, lo, hi, alphabet=alpha)
    text = alpha[rng.integers(0, alphabet, size=text_bytes)]
    _plant_bernoulli(rng, text, pats, plant_rate)
    return Workload(f"random_a{alphabet}", seed, pats, text)


CONFIGS = {
    "tiny": tiny,
    "paper_scale": paper_scale,
    "acgt": acgt,
    "batched": batched,
}
