// PFAC scan kernels for sm_103a (Section II-C: one failure-less walk per
// start position over the CRS trie of Section III).
//
// One persistent, warp-specialized kernel serves the single-text and the
// batched scan; one 1024-thread CTA per SM. After the CTA loads the shared
// tables (its only CTA-wide barrier), its warps split in two.
//
// Producer warps, each an independent pipeline over its own text tiles:
//  a1 staging   lane 0 streams tile + halo (>= longest pattern) into one of
//               `stages` shared-memory buffers with a 1-D TMA bulk copy
//               completing on an mbarrier, `stages` tiles ahead (text whose
//               base is not 16-byte aligned is staged with plain loads);
//  a2 filter    four consecutive positions per lane: a blocked Bloom probe
//               of each 4-gram (byte alphabet) or an exact test of each
//               (k+1)-gram of byte classes, in shared memory; a position
//               that fails cannot match (every pattern is longer);
//     start     a passing position's depth-k node from the dense bitmap +
//               rank table (shared memory); byte-class tries also look up
//               the deep level's bitmap + rank table in L2, settling most
//               positions there;
//  a4 -1        every position gets -1 (one 16-byte streaming store per
//               lane); walks that match patch their id later;
//     hand-off  each remaining walk {position, start depth, start node,
//               text} goes to a shared-memory ring (ballot/popc compaction,
//               per-cell sequence numbers).
// Walker warps take up to 32 ring entries at a time, one walk per lane:
//  a3 CRS walk  each step reads the node's 16-byte row record (row start,
//               length, has-match bit, first eight column bytes) with the
//               next text byte; the child of non-zero e is node e + 1 (BFS
//               order); longer rows are searched in the column array. With
//               layout 1 the walk reads the bitmapped nodes of Section III
//               instead (256-bit child bitmap + first child, rank gives the
//               child);
//  a4 emit      ids[i] = best[v], count += nfinal[v] of the deepest node v;
//  a5 reduce    per-lane counts, warp shuffle reduction, one atomic per warp
//               (per match and text in batch mode).
//
// Every wait (mbarriers, ring cells, idle walkers) is bounded by a clock
// budget counted from the last progress; on expiry the warp records
// PM_ERR_TIMEOUT in a device word, waits (bounded) for its copies in flight
// and returns. The checked variant bounds-checks every shared and global
// index and records PM_ERR_BOUNDS instead of touching memory out of range.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>

#include "pm_internal.h"

namespace pm {

__device__ int g_pm_dev_error;

namespace {

constexpr long long kWaitBudget = 4000000000LL;  // SM clocks (~2 s)
constexpr uint32_t kSuspendHintNs = 1000000u;      // 1 ms per try_wait
constexpr int kMaxStages = 4;

enum Mode { MODE_FAST = 0, MODE_CHECKED = 1, MODE_LOOKUPS = 2 };

struct KParams {
    TrieDev t;
    const uint8_t *text;
    const uint64_t *offsets;
    uint32_t ntexts;
    unsigned long long total;   // single text: start positions to scan
    unsigned long long limit;   // single text: readable bytes (>= total)
    int32_t *ids;
    int32_t *const *out_ids;    // batch: per-text id buffers (nullptr: ids + offset)
    int64_t *counts;
    unsigned long long *lookups;
    uint32_t *tile_counts;      // single text, optional: matches per position tile
    unsigned long long *walks;  // optional: walks queued
    const uint32_t *filter;     // filter table of level k, width W (global)
    const uint2 *dense;         // dense table of level k (k >= 1, global)
    uint32_t first_k;           // BFS id of the first depth-k node
    uint32_t ck1;               // C^(k-1) (k >= 1): weight of a k-gram's first class
    uint32_t kload;             // byte classes: classes a group reads (k or deep_k, + 4)
    uint32_t uk1;               // U^(deep_k - 1): weight of a deep gram's first class
    uint32_t deep_on;           // look up the deep level before walking
    uint32_t gram;              // bytes the filter tests per position (k+1 or k+2)
    uint32_t tile;
    uint32_t halo;
    uint32_t k;
    uint32_t lw;                // log2 W
    uint32_t binary;
    uint32_t bitmap;            // walks read bitmapped nodes instead of row records
    uint32_t stages;
    uint32_t walkers;           // walker warps per CTA (the rest produce)
    uint32_t aligned;
    uint32_t ids_aligned;
    // shared-memory layout (byte offsets)
    uint32_t off_dense, off_lut, off_ring, off_warp;  // shared tables and ring, then per-warp blocks
    uint32_t warp_bytes;          // bytes of one producer warp's block
    uint32_t off_stages;          // inside a warp's block (after its mbarriers)
    uint32_t stage_bytes;         // tile + halo
    uint32_t filt_u4;             // filter size in 16-byte units
    uint32_t dense_u4;            // dense table size in 16-byte units (0: none)
    uint32_t filt_words;          // filter size in u32 words
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One try_wait: the thread is suspended until the phase completes or the
// hinted time (ns) passes, so a waiting warp takes no issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase), "r"(kSuspendHintNs)
        : "memory");
    return done != 0;
}

// Bounded wait: false if the phase did not complete within the budget.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (clock64() - t0 > kWaitBudget) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void record_error(int code)
{
    atomicCAS(&g_pm_dev_error, 0, code);
}

// L2 policy "evict last" for the trie: it stays resident while the text
// and the ids stream through L2.
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint32_t ld_trie_u32(const void *ptr, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint4 ld_trie_u4(const uint4 *ptr, uint64_t pol)
{
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint2 ld_trie_u2(const uint2 *ptr, uint64_t pol)
{
    uint2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
        : "=r"(v.x), "=r"(v.y)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_trie_u8(const void *ptr, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Bytes staged for the tile at t0: tile + halo, clipped to the readable end
// (the total in batch mode, the single text's limit otherwise).
__device__ __forceinline__ unsigned long long tile_bytes(const KParams &p, unsigned long long t0,
                                                         unsigned long long end)
{
    unsigned long long want = (unsigned long long)p.tile + p.halo;
    unsigned long long left = end - t0;
    return left < want ? left : want;
}

// Issue the TMA copy of the tile at text offset t0 into stage `s` of a warp
// (lane 0).
__device__ __forceinline__ void issue_tile(const KParams &p, uint8_t *stages, uint64_t *bars,
                                           uint32_t s, unsigned long long t0,
                                           unsigned long long end)
{
    uint32_t nb = (uint32_t)tile_bytes(p, t0, end);
    uint32_t nb16 = nb & ~15u;
    if (p.aligned && nb16) {
        mbar_arrive_tx(&bars[s], nb16);
        tma_load_1d(stages + (size_t)s * p.stage_bytes, p.text + t0, nb16, &bars[s]);
    } else {
        mbar_arrive(&bars[s]);
    }
}

// Index of the text containing byte position `pos` (largest t with
// offsets[t] <= pos); texts of length 0 are skipped.
__device__ __forceinline__ uint32_t find_text(const uint64_t *off, uint32_t ntexts,
                                              unsigned long long pos)
{
    uint32_t lo = 0, hi = ntexts;  // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Walk ring, in shared memory, between the producer warps (tiles, filter)
// and the walker warps (CRS walks). An entry is one walk (walk_entry_of):
// x = start position (low 32 bits), y = its bits 32..39 | start depth << 8,
// z = start node, w = text index (batch) or 0xFFFFFFFF.
// Each cell carries a sequence number (a bounded multi-producer,
// multi-consumer ring): cell i starts at i; the producer of slot s waits for
// s, fills the cell and sets s+1; the walker of slot s waits for s+1, takes
// the entry and sets s+kRing, freeing the cell for slot s+kRing only.
constexpr uint32_t kRing = 512;  // entries (power of two)

struct Ring {
    unsigned int wr;        // slots reserved by producers
    unsigned int rd;        // slots taken by walkers
    unsigned int pdone;     // producer warps finished
    unsigned int progress;  // tiles finished by producers (walkers' heartbeat)
};

// Bounded spin: true while the budget lasts (a few seconds of SM clocks).
__device__ __forceinline__ bool spin_ok(long long t0)
{
    return clock64() - t0 < kWaitBudget;
}

// Position of byte b in the CRS row [r0, r0 + deg) whose first eight bytes
// (ascending, zero padded) are packed in lab0/lab1, or 0xFFFFFFFF. Bytes
// past the eighth are searched in col by halving (rows longer than 16, or
// `binary`) or in order.
__device__ __forceinline__ uint32_t row_find(const uint8_t *col, uint32_t r0, uint32_t deg,
                                             uint32_t lab0, uint32_t lab1, uint32_t b,
                                             uint32_t binary, uint64_t pol)
{
    if (deg <= 8u || b <= (lab1 >> 24)) {
        // labels are unique and ascending, padding sits above the row's end:
        // the lowest zero byte of (labels xor b) is the match. The zero-byte
        // test (x - 0x01..) & ~x & 0x80.. flags every zero byte and, through
        // borrows, only bytes above one, so its lowest flag is exact.
        const uint32_t bb = b * 0x01010101u;
        const uint32_t x0 = lab0 ^ bb;
        const uint32_t z0 = (x0 - 0x01010101u) & ~x0 & 0x80808080u;
        uint32_t i;
        if (z0 || deg <= 4u) {
            i = z0 ? (uint32_t)(__ffs(z0) - 1) >> 3 : 8u;
        } else {
            const uint32_t x1 = lab1 ^ bb;
            const uint32_t z1 = (x1 - 0x01010101u) & ~x1 & 0x80808080u;
            i = z1 ? 4u + ((uint32_t)(__ffs(z1) - 1) >> 3) : 8u;
        }
        return i < min(deg, 8u) ? r0 + i : 0xFFFFFFFFu;
    }
    const uint32_t r1 = r0 + deg;
    if (binary || deg > 16u) {
        uint32_t lo = r0 + 8u, hi = r1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (ld_trie_u8(col + mid, pol) < b) lo = mid + 1;
            else hi = mid;
        }
        return lo < r1 && ld_trie_u8(col + lo, pol) == b ? lo : 0xFFFFFFFFu;
    }
    for (uint32_t e = r0 + 8u; e < r1; ++e) {
        const uint32_t cb = ld_trie_u8(col + e, pol);
        if (cb >= b) return cb == b ? e : 0xFFFFFFFFu;
    }
    return 0xFFFFFFFFu;
}

// End of the current text relative to the tile start, clipped to 32 bits.
__device__ __forceinline__ uint32_t rel_end_of(unsigned long long e, unsigned long long t0)
{
    const unsigned long long r = e - t0;
    return r > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)r;
}

// Class of byte b from the lane-replicated LUT (identity for the byte alphabet).
template <bool IDENT>
__device__ __forceinline__ uint32_t class_of(const uint32_t *s_lut, uint32_t lane, uint32_t b)
{
    if (IDENT) return b;
    return (s_lut[(b >> 2) * 32 + lane] >> ((b & 3) * 8)) & 0xFFu;
}

// A walk from position pos ended at node v after matching `depth` bytes;
// has: v's has-match bit (2: not read). Writes the position's id and adds
// its count when a pattern ends on the path.
template <bool BATCH>
__device__ __forceinline__ void emit_walk(const KParams &p, unsigned long long pos, uint32_t txt,
                                          uint32_t v, uint32_t depth, uint32_t has,
                                          unsigned long long &acc)
{
    if (depth < p.t.min_len || has == 0u) return;
    const int2 em = __ldg(p.t.emit + v);
    if (!em.y) return;
    if (BATCH && p.out_ids)
        p.out_ids[txt][pos - __ldg(p.offsets + txt)] = em.x;
    else
        p.ids[pos] = em.x;
    if (BATCH) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p.counts + txt), (unsigned long long)em.y);
    } else {
        acc += (unsigned)em.y;
        if (p.tile_counts) atomicAdd(p.tile_counts + (pos >> kMatchTileShift), (unsigned)em.y);
    }
}

// A ring entry is one walk: the start position (40 bits), the bytes already
// matched from it (its start depth: 0, k or the deep level's), the node at
// that depth, and (batch) the index of its text, or 0xFFFFFFFF if unknown.
__device__ __forceinline__ uint4 walk_entry_of(unsigned long long pos, uint32_t depth,
                                               uint32_t node, uint32_t txt)
{
    return make_uint4((uint32_t)pos, ((uint32_t)(pos >> 32) & 0xFFu) | (depth << 8), node, txt);
}

// Run one walk (Section II-C): from its start node, read each node's row
// record and the next text byte together, move to the child on that byte,
// and stop at a mismatch, a leaf or the text end; then patch the
// position's id when a pattern ends on the path.
template <bool BATCH, int MODE>
__device__ __forceinline__ void run_walk(const KParams &p, uint4 e, unsigned long long end,
                                         uint64_t pol, unsigned long long &acc,
                                         unsigned long long &look)
{
    const TrieDev &t = p.t;
    const unsigned long long pos = ((unsigned long long)(e.y & 0xFFu) << 32) | e.x;
    uint32_t jo = e.y >> 8;
    uint32_t v = e.z;
    uint32_t txt = 0;
    unsigned long long tend = end;
    if (BATCH) {
        txt = e.w != 0xFFFFFFFFu ? e.w : find_text(p.offsets, p.ntexts, pos);
        tend = __ldg(p.offsets + txt + 1);
    }
    const uint32_t te = rel_end_of(tend, pos);
    const uint8_t *tp = p.text + pos;
    uint32_t has = 2u;  // has-match bit of the final node (2: not read)
    while (jo < te) {
        if (MODE == MODE_CHECKED && v >= t.n_nodes) {
            record_error(PM_ERR_BOUNDS);
            return;
        }
        const uint32_t b = __ldg(tp + jo);
        if (p.bitmap) {
            // bitmapped node (Section III, Fig. 3): the child on byte b is
            // first + (set bits below b) when bit b is set
            const uint4 lo = ld_trie_u4(t.bm + 2 * (size_t)v, pol);
            const uint4 hi = ld_trie_u4(t.bm + 2 * (size_t)v + 1, pol);
            const uint32_t first = ld_trie_u32(t.bm_first + v, pol);
            if (MODE == MODE_LOOKUPS) ++look;
            const uint32_t w = b >> 5, bit = b & 31u;
            uint32_t below = 0, hitw = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t wi = i == 0 ? lo.x : i == 1 ? lo.y : i == 2 ? lo.z : i == 3 ? lo.w
                                  : i == 4 ? hi.x : i == 5 ? hi.y : i == 6 ? hi.z : hi.w;
                const uint32_t m = (uint32_t)i < w ? 0xFFFFFFFFu
                                   : (uint32_t)i == w ? (1u << bit) - 1u : 0u;
                below += __popc(wi & m);
                if ((uint32_t)i == w) hitw = wi;
            }
            if (!((hitw >> bit) & 1u)) break;
            if (MODE == MODE_CHECKED && first + below >= t.n_nodes) {
                record_error(PM_ERR_BOUNDS);
                return;
            }
            v = first + below;
            ++jo;
            continue;
        }
        const uint4 r = ld_trie_u4(t.row + v, pol);
        const uint32_t deg = r.y & 0x1FFu;
        has = r.y >> 31;
        if (MODE == MODE_CHECKED && (r.x > t.nnz || deg > t.nnz - r.x)) {
            record_error(PM_ERR_BOUNDS);
            return;
        }
        if (MODE == MODE_LOOKUPS) ++look;
        if (deg == 0) break;  // leaf
        const uint32_t ei = row_find(t.col, r.x, deg, r.z, r.w, b, p.binary, pol);
        if (ei == 0xFFFFFFFFu) break;
        v = ei + 1u;  // BFS order: the child of non-zero e is node e + 1
        ++jo;
        has = 2u;
    }
    emit_walk<BATCH>(p, pos, txt, v, jo, has, acc);
}

// Walker warp: takes up to 32 ring entries at a time, one walk per lane,
// until every producer warp has finished and the ring is empty; the wait
// for entries is bounded, counted from the producers' last progress.
template <bool BATCH, int MODE>
__device__ __forceinline__ void walker_loop(const KParams &p, Ring *ring, const uint4 *entries,
                                            unsigned int *flags, uint32_t NP,
                                            unsigned long long end, uint32_t lane,
                                            unsigned long long &acc, unsigned long long &look)
{
    volatile Ring *vr = ring;
    volatile unsigned int *vf = flags;
    const uint64_t pol = policy_evict_last();
    long long t0 = clock64();
    uint32_t seen = vr->progress;
    while (true) {
        uint32_t base = 0, take = 0;  // take 0xFFFFFFFF: stop
        if (lane == 0) {
            while (true) {
                const uint32_t rd = vr->rd, wr = vr->wr;
                if ((int32_t)(wr - rd) > 0) {
                    const uint32_t n = min(32u, wr - rd);
                    if (atomicCAS(&ring->rd, rd, rd + n) == rd) {
                        base = rd;
                        take = n;
                        break;
                    }
                    continue;
                }
                if (vr->pdone >= NP) {
                    __threadfence_block();
                    if ((int32_t)(vr->wr - vr->rd) <= 0) {
                        take = 0xFFFFFFFFu;
                        break;
                    }
                    continue;
                }
                const uint32_t now = vr->progress;
                if (now != seen) {
                    seen = now;
                    t0 = clock64();
                } else if (!spin_ok(t0)) {
                    record_error(PM_ERR_TIMEOUT);
                    take = 0xFFFFFFFFu;
                    break;
                }
                __nanosleep(64);
            }
        }
        take = __shfl_sync(0xffffffffu, take, 0);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take == 0xFFFFFFFFu) break;
        if (lane < take) {
            const uint32_t slot = base + lane, idx = slot & (kRing - 1);
            const long long w0 = clock64();
            bool ok = true;
            while (vf[idx] != slot + 1u) {  // until the producer has filled it
                if (clock64() - w0 > kWaitBudget) {
                    record_error(PM_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
            }
            if (ok) {
                __threadfence_block();
                const uint4 e = entries[idx];
                __threadfence_block();
                vf[idx] = slot + kRing;  // free for the slot one lap later
                run_walk<BATCH, MODE>(p, e, end, pol, acc, look);
            }
        }
        __syncwarp();
    }
}

// KF: the filter level k when fixed at compile time (byte alphabet), or -1
// for a runtime k over byte classes. G: bytes the byte-alphabet Bloom filter
// tests (3 or 4), 0 when not fixed.
template <int KF, int G, bool IDENT, bool BATCH, int MODE>
__global__ void __launch_bounds__(1024, 1) pfac_scan_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const TrieDev &t = p.t;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t NW = blockDim.x >> 5;
    const uint32_t NP = NW - p.walkers;  // producer warps; the rest walk

    const unsigned long long total = BATCH ? __ldg(p.offsets + p.ntexts) : p.total;
    const unsigned long long end = BATCH ? total : p.limit;
    const unsigned long long ntiles = (total + p.tile - 1) / p.tile;
    if ((unsigned long long)blockIdx.x * NP >= ntiles) return;

    uint32_t *s_filt = reinterpret_cast<uint32_t *>(smem);
    uint2 *s_dense = reinterpret_cast<uint2 *>(smem + p.off_dense);
    uint32_t *s_lut = reinterpret_cast<uint32_t *>(smem + p.off_lut);
    uint4 *entries = reinterpret_cast<uint4 *>(smem + p.off_ring);
    unsigned int *flags = reinterpret_cast<unsigned int *>(smem + p.off_ring + kRing * 16);
    Ring *ring = reinterpret_cast<Ring *>(smem + p.off_ring + kRing * 20);

    // Tables into shared memory, shared by all warps of the CTA.
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.filter);
        uint4 *dst = reinterpret_cast<uint4 *>(s_filt);
        for (uint32_t i = tid; i < p.filt_u4; i += blockDim.x) dst[i] = __ldg(src + i);
        const uint4 *dsrc = reinterpret_cast<const uint4 *>(p.dense);
        uint4 *ddst = reinterpret_cast<uint4 *>(s_dense);
        for (uint32_t i = tid; i < p.dense_u4; i += blockDim.x) ddst[i] = __ldg(dsrc + i);
        if (!IDENT) {
            // class LUT replicated per lane: word (b/4)*32 + lane holds the
            // classes of bytes 4*(b/4) .. +3, so lane l always hits bank l.
            for (uint32_t i = tid; i < 64 * 32; i += blockDim.x) {
                const uint32_t w = i >> 5;
                s_lut[i] = (uint32_t)__ldg(t.cls + 4 * w) | ((uint32_t)__ldg(t.cls + 4 * w + 1) << 8) |
                           ((uint32_t)__ldg(t.cls + 4 * w + 2) << 16) |
                           ((uint32_t)__ldg(t.cls + 4 * w + 3) << 24);
            }
        }
        for (uint32_t i = tid; i < kRing; i += blockDim.x) flags[i] = i;  // cell i free for slot i
        if (tid == 0) *ring = Ring{0u, 0u, 0u, 0u};
    }
    __syncthreads();  // the only CTA-wide barrier: warps run independently below

    constexpr uint32_t KFU = KF > 0 ? (uint32_t)KF : 0u;  // KF as unsigned (0 if runtime)
    const uint32_t k = KF >= 0 ? KFU : p.k;
    const uint32_t gram = p.gram;
    unsigned long long acc = 0;   // matches (single text)
    unsigned long long look = 0;  // lookups (MODE_LOOKUPS)

    if (warp >= NP) {
        walker_loop<BATCH, MODE>(p, ring, entries, flags, NP, end, lane, acc, look);
    } else {
        const unsigned long long gw = (unsigned long long)blockIdx.x * NP + warp;
        const unsigned long long TW = (unsigned long long)gridDim.x * NP;
        const unsigned long long my_tiles = gw < ntiles ? (ntiles - 1 - gw) / TW + 1 : 0;

        uint8_t *wsm = smem + p.off_warp + (size_t)warp * p.warp_bytes;
        uint64_t *bars = reinterpret_cast<uint64_t *>(wsm);
        uint8_t *stages = wsm + p.off_stages;
        volatile unsigned int *vf = flags;

        const unsigned long long tstride = TW * p.tile;  // text between a warp's tiles
        if (lane == 0 && my_tiles) {
            for (uint32_t s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            const unsigned long long pre = my_tiles < p.stages ? my_tiles : p.stages;
            for (unsigned long long i = 0; i < pre; ++i)
                issue_tile(p, stages, bars, (uint32_t)i, (gw + i * TW) * p.tile, end);
        }
        __syncwarp();

        const uint32_t C = t.C;
        const uint64_t tpol = policy_evict_last();  // deep-level lookups
        const uint32_t lw = p.lw;
        const uint32_t wmask = (1u << lw) - 1u;
        // IDENT: filter bit index = low 8k+lw bits of the little-endian window
        const uint32_t imask = KF >= 0 ? (uint32_t)((1ull << (8 * KFU + lw)) - 1ull) : 0u;
        bool failed = false;

        uint32_t s = 0, phase = 0;            // stage and its mbarrier phase
        unsigned long long t0 = gw * p.tile;  // start of the current tile
        const unsigned long long ahead = (unsigned long long)p.stages * tstride;
        for (unsigned long long it = 0; it < my_tiles && !failed; ++it, t0 += tstride) {
            const uint32_t nbytes = (uint32_t)tile_bytes(p, t0, end);
            uint8_t *st = stages + (size_t)s * p.stage_bytes;

            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[s], phase));
            if (!ok) {
                if (lane == 0) {
                    record_error(PM_ERR_TIMEOUT);
                    // copies still in flight: tiles it .. it+stages-1
                    for (unsigned long long j = 0; j < p.stages && it + j < my_tiles; ++j) {
                        const uint32_t sj = (uint32_t)((s + j) % p.stages);
                        mbar_wait_bounded(&bars[sj], phase ^ (uint32_t)((s + j) >= p.stages));
                    }
                }
                break;
            }
            const uint32_t nb16 = p.aligned ? (nbytes & ~15u) : 0u;
            if (nb16 < nbytes) {
                for (uint32_t i = nb16 + lane; i < nbytes; i += 32) st[i] = __ldg(p.text + t0 + i);
                __syncwarp();
            }

            const uint32_t tile_n = (uint32_t)(total - t0 < p.tile ? total - t0 : p.tile);
            uint32_t cur = 0;
            unsigned long long text_end = end;
            if (BATCH) {
                cur = find_text(p.offsets, p.ntexts, t0 + 4 * lane < total ? t0 + 4 * lane : t0);
                text_end = __ldg(p.offsets + cur + 1);
            }
            uint32_t rel_end = rel_end_of(text_end, t0);
            // groups [lp0, lp0+4) with lp0 + 4 <= fast_n take the fast path
            auto fast_bound = [&]() -> uint32_t {
                const uint32_t r = rel_end >= gram - 1 ? rel_end - (gram - 1) : 0u;
                return r < tile_n ? r : tile_n;
            };
            uint32_t fast_n = fast_bound();
            int32_t *idt = p.ids + t0;  // this tile's ids

            const uint32_t iters = (tile_n + 127) >> 7;
            for (uint32_t i = 0; i < iters; ++i) {
                const uint32_t lp0 = (i << 7) + 4 * lane;
                const uint32_t *wp = reinterpret_cast<const uint32_t *>(st + lp0);
                if (BATCH && lp0 < tile_n && t0 + lp0 >= text_end) {
                    while (t0 + lp0 >= text_end) {
                        ++cur;
                        text_end = __ldg(p.offsets + cur + 1);
                    }
                    rel_end = rel_end_of(text_end, t0);
                    fast_n = fast_bound();
                }
                const uint32_t cur0 = cur;  // text of position lp0
                const uint32_t w0 = wp[0], w1 = wp[1];  // bytes lp0 .. lp0+7 (staged)
                uint32_t need = 0;   // bit q: position lp0+q passed the filter
                uint32_t rk[4] = {0u, 0u, 0u, 0u};  // node ranks in the start level
                uint32_t deepm = 0;  // bit q: position lp0+q starts at the deep level
                uint32_t rootm = 0;  // bit q: position lp0+q is walked from the root
                if (MODE != MODE_LOOKUPS && lp0 + 4 <= fast_n) {
                    // Fast path: four positions, all bytes up to lp0+3+gram-1
                    // inside the text. The filter decides, in shared memory,
                    // which positions can reach depth k+1.
                    if (IDENT && KF >= (int)kBloomK) {
                        // blocked Bloom test of the g-gram at each position
                        const uint32_t sh = 32u - (8u * KFU + lw - 5u);
                        const uint32_t gsh = G > 0 ? 32u - 8u * G : 32u - 8u * gram;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t win = q == 0 ? w0 : __funnelshift_r(w0, w1, 8 * q);
                            // bytes q .. q+g-1, shifted to the top
                            const uint32_t h = __umulhi(G == 4 ? win : win << gsh, kBloomMul);
                            const uint32_t word = h >> sh;
                            if (MODE == MODE_CHECKED && word >= p.filt_words) {
                                record_error(PM_ERR_BOUNDS);
                                continue;
                            }
                            // both Bloom bits, each rotated down to bit 0 (the
                            // funnel shift takes its amount mod 32)
                            const uint32_t val = s_filt[word];
                            const uint32_t r = __funnelshift_r(val, val, h) & __funnelshift_r(val, val, h >> 5);
                            need |= (r & 1u) << q;
                        }
                    } else if (IDENT && KF >= 0) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t x = q == 0 ? w0 : __funnelshift_r(w0, w1, 8 * q);
                            const uint32_t idx = x & imask;
                            const uint32_t word = idx >> 5;
                            if (MODE == MODE_CHECKED && word >= p.filt_words) {
                                record_error(PM_ERR_BOUNDS);
                                continue;
                            }
                            need |= ((s_filt[word] >> (idx & 31u)) & 1u) << q;
                        }
                    } else {
                        // byte classes: the k-gram code of position lp0 by
                        // Horner's rule, then rolled one position at a time
                        // (drop the first class, append the next); a position
                        // that passes the filter gets the rank of its depth-k
                        // node from the dense table
                        uint32_t cw[4];  // classes of bytes lp0 .. lp0+15, four to a word
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const uint32_t word = w == 0 ? w0 : w == 1 ? w1 : (uint32_t)(4 * w) < p.kload ? wp[w] : 0u;
                            cw[w] = 0;
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                cw[w] |= class_of<IDENT>(s_lut, lane, (word >> (8 * b)) & 0xFFu) << (8 * b);
                        }
                        // class of byte lp0 + j (j known at compile time)
#define PM_CLS(j) ((cw[(j) >> 2] >> (8 * ((j) & 3))) & 0xFFu)
                        uint32_t cd = 0;
#pragma unroll
                        for (int j = 0; j < 12; ++j)
                            if (j < (int)k) cd = cd * C + PM_CLS(j);
                        // classes k .. k+3: the byte after each position's k-gram
                        const uint32_t kw = k >> 2;
                        const uint32_t wa = kw == 0 ? cw[0] : kw == 1 ? cw[1] : kw == 2 ? cw[2] : cw[3];
                        const uint32_t wb = kw == 0 ? cw[1] : kw == 1 ? cw[2] : cw[3];
                        const uint32_t nc4 = __funnelshift_r(wa, wb, 8u * (k & 3u));
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t nc = (nc4 >> (8 * q)) & 0xFFu;
                            const uint32_t idx = (cd << lw) | (nc & wmask);
                            const uint32_t word = idx >> 5;
                            if (MODE == MODE_CHECKED && word >= p.filt_words) {
                                record_error(PM_ERR_BOUNDS);
                            } else if ((s_filt[word] >> (idx & 31u)) & 1u) {
                                if (k == 0) {
                                    need |= 1u << q;
                                } else if (MODE == MODE_CHECKED && (cd >> 5) >= p.dense_u4 * 2) {
                                    record_error(PM_ERR_BOUNDS);
                                } else {
                                    const uint2 d = s_dense[cd >> 5];
                                    const uint32_t bit = cd & 31u;
                                    if ((d.x >> bit) & 1u) {
                                        need |= 1u << q;
                                        rk[q] = d.y + __popc(d.x & ((1u << bit) - 1u));
                                    }
                                }
                            }
                            if (q < 3 && k > 0) cd = (cd - PM_CLS(q) * p.ck1) * C + nc;
                        }
                        if (p.deep_on && need) {
                            // deep level: a flagged position whose first
                            // deep_k bytes lie in its text looks up its
                            // deep_k-gram (base U, first class most
                            // significant) in L2. A byte of the "other" class
                            // or a gram that is not a root path means no match
                            // (deep_k < shortest pattern); else the walk
                            // starts at depth deep_k.
                            const uint32_t K2 = t.deep_k, U = t.deep_U;
                            // bit j: the byte at lp0 + j is of the "other" class
                            // (an exact zero-byte test of class xor U per word,
                            // its four byte flags gathered by one multiply)
                            uint32_t om = 0;
#pragma unroll
                            for (int w = 0; w < 4; ++w) {
                                const uint32_t x = cw[w] ^ (U * 0x01010101u);
                                const uint32_t nz = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
                                const uint32_t zf = (~nz & 0x80808080u) >> 7;  // 1 per zero byte
                                om |= (((zf * 0x00204081u) >> 21) & 0xFu) << (4 * w);
                            }
                            const uint32_t kmask = (1u << K2) - 1u;
                            // the first position's deep code by Horner's rule,
                            // the next ones by rolling (classes K2 .. K2+2 enter)
                            uint32_t cc = 0;
#pragma unroll
                            for (int j = 0; j < (int)kDeepMaxK; ++j)
                                if (j < (int)K2) cc = cc * U + PM_CLS(j);
                            const uint32_t kw2 = K2 >> 2;
                            const uint32_t ea = kw2 == 0 ? cw[0] : kw2 == 1 ? cw[1] : kw2 == 2 ? cw[2] : cw[3];
                            const uint32_t eb = kw2 == 0 ? cw[1] : kw2 == 1 ? cw[2] : cw[3];
                            const uint32_t enter = __funnelshift_r(ea, eb, 8u * (K2 & 3u));
                            uint2 d2[4];
                            uint32_t bits2 = 0;  // 5 bits per position: its code's bit in the word
                            uint32_t dm = 0;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint32_t cq = cc;
                                if (q < 3) cc = (cc - PM_CLS(q) * p.uk1) * U + ((enter >> (8 * q)) & 0xFFu);
                                if (!((need >> q) & 1u) || lp0 + q + K2 > rel_end) continue;
                                if ((om >> q) & kmask) {
                                    need &= ~(1u << q);
                                    continue;
                                }
                                if (MODE == MODE_CHECKED && (cq >> 5) >= t.deep_words) {
                                    record_error(PM_ERR_BOUNDS);
                                    need &= ~(1u << q);
                                    continue;
                                }
                                bits2 |= (cq & 31u) << (5 * q);
                                d2[q] = ld_trie_u2(t.deep + (cq >> 5), tpol);
                                dm |= 1u << q;
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (!((dm >> q) & 1u)) continue;
                                const uint32_t bit = (bits2 >> (5 * q)) & 31u;
                                if ((d2[q].x >> bit) & 1u)
                                    rk[q] = d2[q].y + __popc(d2[q].x & ((1u << bit) - 1u));
                                else
                                    need &= ~(1u << q);
                            }
                            deepm = dm & need;
                        }
#undef PM_CLS
                    }
                    if (IDENT && KF >= 1 && need) {
                        // byte alphabet: the depth-k node of each flagged
                        // position (its k-gram's code, first byte most
                        // significant); a k-gram that is not a root path
                        // (a Bloom false positive) needs no walk
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (!((need >> q) & 1u)) continue;
                            const uint32_t x = q == 0 ? w0 : __funnelshift_r(w0, w1, 8 * q);
                            const uint32_t code = KF == 1 ? (x & 0xFFu) : __byte_perm(x, 0u, 0x4401u);
                            if (MODE == MODE_CHECKED && (code >> 5) >= p.dense_u4 * 2) {
                                record_error(PM_ERR_BOUNDS);
                                need &= ~(1u << q);
                                continue;
                            }
                            const uint2 d = s_dense[code >> 5];
                            const uint32_t bit = code & 31u;
                            if ((d.x >> bit) & 1u)
                                rk[q] = d.y + __popc(d.x & ((1u << bit) - 1u));
                            else
                                need &= ~(1u << q);
                        }
                    }
                } else {
                    // ragged group (tile end, text boundary, last bytes of a
                    // text): every position that passes the filter, or that
                    // is too close to its text end to test, is walked from the
                    // root
                    for (uint32_t q = 0; q < 4; ++q) {
                        const uint32_t lp = lp0 + q;
                        if (lp >= tile_n) break;
                        const unsigned long long pos = t0 + lp;
                        if (BATCH) {
                            while (pos >= text_end) {
                                ++cur;
                                text_end = __ldg(p.offsets + cur + 1);
                            }
                            rel_end = rel_end_of(text_end, t0);
                            fast_n = fast_bound();
                        }
                        if (MODE == MODE_LOOKUPS || lp + gram > rel_end) {
                            rootm |= 1u << q;
                            continue;
                        }
                        uint32_t word, bits;
                        if (IDENT && KF >= (int)kBloomK) {
                            uint32_t x = 0;
                            for (uint32_t j = 0; j < gram; ++j) x |= (uint32_t)st[lp + j] << (8 * j);
                            const BloomProbe b = bloom_probe(x, gram, 8u * KFU + lw - 5u);
                            word = b.word;
                            bits = b.mask;
                        } else if (IDENT && KF >= 0) {
                            uint32_t x = 0;
                            for (uint32_t j = 0; j <= k; ++j) x |= (uint32_t)st[lp + j] << (8 * j);
                            const uint32_t idx = x & imask;
                            word = idx >> 5;
                            bits = 1u << (idx & 31u);
                        } else {
                            uint32_t cd = 0;
                            for (uint32_t j = 0; j + 1 <= k; ++j) cd = cd * C + class_of<IDENT>(s_lut, lane, st[lp + j]);
                            const uint32_t idx = (cd << lw) | (class_of<IDENT>(s_lut, lane, st[lp + k]) & wmask);
                            word = idx >> 5;
                            bits = 1u << (idx & 31u);
                        }
                        if (MODE == MODE_CHECKED && word >= p.filt_words) {
                            record_error(PM_ERR_BOUNDS);
                            continue;
                        }
                        if ((s_filt[word] & bits) == bits) rootm |= 1u << q;
                    }
                }
                // every position gets -1 now; the walkers patch the matches
                if (BATCH && p.out_ids) {
                    // per-text output buffers: each position to its own text's
                    uint32_t c2 = cur0;
                    unsigned long long e2 = __ldg(p.offsets + c2 + 1);
                    for (uint32_t q = 0; q < 4 && lp0 + q < tile_n; ++q) {
                        const unsigned long long pos = t0 + lp0 + q;
                        while (pos >= e2) {
                            ++c2;
                            e2 = __ldg(p.offsets + c2 + 1);
                        }
                        __stcs(p.out_ids[c2] + (pos - __ldg(p.offsets + c2)), -1);
                    }
                } else if (p.ids_aligned && lp0 + 4 <= tile_n) {
                    __stcs(reinterpret_cast<int4 *>(idt + lp0), make_int4(-1, -1, -1, -1));
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (lp0 + q < tile_n) __stcs(idt + lp0 + q, -1);
                }
                // warp ballot/popc compaction of the walks into the shared
                // ring, one entry per walk (position, start depth, node)
                const uint32_t work = need | rootm;
                const uint32_t mg = __ballot_sync(0xffffffffu, work != 0);
                if (mg) {
                    // slots: walks ordered by position within the group, then
                    // by lane; with at most one walk per lane (the common case
                    // under a selective filter) one ballot gives them all
                    uint32_t mq[4], off[4], tot = 0;
                    if (!__any_sync(0xffffffffu, (work & (work - 1u)) != 0)) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            mq[q] = mg;
                            off[q] = 0;
                        }
                        tot = __popc(mg);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            mq[q] = __ballot_sync(0xffffffffu, (work >> q) & 1u);
                            off[q] = tot;
                            tot += __popc(mq[q]);
                        }
                    }
                    uint32_t base = 0;
                    if (lane == 0) {
                        base = atomicAdd(&ring->wr, tot);
                        if (p.walks) atomicAdd(p.walks, (unsigned long long)tot);
                    }
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!((work >> q) & 1u) || failed) continue;
                        const uint32_t slot = base + off[q] + __popc(mq[q] & below);
                        const uint32_t idx = slot & (kRing - 1);
                        const long long w0c = clock64();
                        while (vf[idx] != slot) {  // until the cell is free for this slot
                            if (clock64() - w0c > kWaitBudget) {
                                record_error(PM_ERR_TIMEOUT);
                                failed = true;
                                break;
                            }
                        }
                        if (failed) break;
                        const bool root = (rootm >> q) & 1u;
                        const bool dp = (deepm >> q) & 1u;
                        const uint32_t depth = root ? 0u : dp ? t.deep_k : k;
                        const uint32_t node = root || depth == 0 ? 0u
                                              : (dp ? t.deep_first : p.first_k) + rk[q];
                        entries[idx] = walk_entry_of(t0 + lp0 + q, depth, node,
                                                     BATCH && !root ? cur0 : 0xFFFFFFFFu);
                        __threadfence_block();  // the -1 store and the entry before the flag
                        vf[idx] = slot + 1u;
                    }
                    failed = __any_sync(0xffffffffu, failed);
                    if (failed) break;
                }
            }

            __syncwarp();  // stage s fully consumed by this warp
            if (failed) {
                // drain this warp's copies still in flight (tiles it+1 ..
                // it+stages-1) before leaving
                if (lane == 0)
                    for (unsigned long long j = 1; j < p.stages && it + j < my_tiles; ++j) {
                        const uint32_t sj = (uint32_t)((s + j) % p.stages);
                        mbar_wait_bounded(&bars[sj], phase ^ (uint32_t)((s + j) >= p.stages));
                    }
                break;
            }
            if (lane == 0) {
                if (it + p.stages < my_tiles) {
                    fence_proxy_async();
                    issue_tile(p, stages, bars, s, t0 + ahead, end);
                }
                atomicAdd(&ring->progress, 1u);
            }
            if (++s == p.stages) {
                s = 0;
                phase ^= 1u;
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();  // the last reservations before the done count
            atomicAdd(&ring->pdone, 1u);
        }
    }

    // warp reductions: single-text count and lookups
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        look += __shfl_xor_sync(0xffffffffu, look, o);
    }
    if (lane == 0) {
        if (!BATCH && acc) atomicAdd(reinterpret_cast<unsigned long long *>(p.counts), acc);
        if (MODE == MODE_LOOKUPS && look && p.lookups) atomicAdd(p.lookups, look);
    }
}

typedef void (*KernelFn)(KParams);

template <int KF, int G, bool IDENT>
KernelFn pick_mode(bool batch, int mode)
{
    if (batch) {
        switch (mode) {
        case MODE_CHECKED: return pfac_scan_kernel<KF, G, IDENT, true, MODE_CHECKED>;
        case MODE_LOOKUPS: return pfac_scan_kernel<KF, G, IDENT, true, MODE_LOOKUPS>;
        default: return pfac_scan_kernel<KF, G, IDENT, true, MODE_FAST>;
        }
    }
    switch (mode) {
    case MODE_CHECKED: return pfac_scan_kernel<KF, G, IDENT, false, MODE_CHECKED>;
    case MODE_LOOKUPS: return pfac_scan_kernel<KF, G, IDENT, false, MODE_LOOKUPS>;
    default: return pfac_scan_kernel<KF, G, IDENT, false, MODE_FAST>;
    }
}

// Byte alphabet (C = 256): k is 0, 1 or 2 and fixed at compile time, and so
// is the Bloom gram length at k = 2.
KernelFn pick_kernel(uint32_t C, uint32_t k, uint32_t gram, bool batch, int mode)
{
    if (C == 256) {
        if (k == 0) return pick_mode<0, 0, true>(batch, mode);
        if (k == 1) return pick_mode<1, 0, true>(batch, mode);
        if (gram == 4) return pick_mode<2, 4, true>(batch, mode);
        return pick_mode<2, 3, true>(batch, mode);
    }
    return pick_mode<-1, 0, false>(batch, mode);
}

// Per-text count finalisation: counts[t] to the caller's *out[t].
__global__ void pm_counts_scatter_kernel(const int64_t *counts, int64_t *const *out, uint32_t n)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) *out[t] = counts[t];
}

uint32_t round16(uint64_t x) { return (uint32_t)((x + 15) & ~15ull); }

struct Layout {
    uint32_t off_dense, off_lut, off_ring, off_warp, warp_bytes, off_stages, stage_bytes, total;
    uint32_t filt_u4, dense_u4, filt_words, halo;
};

int width_index(int32_t bits) { return bits == 8 ? 0 : bits == 16 ? 1 : 2; }

// Shared memory: [filter][dense table][class LUT][walk ring] shared by the CTA, then one
// block per producer warp: [mbarriers][stages x (tile + halo)].
Layout layout(const TrieDev &t, const pm_config &cfg)
{
    Layout L{};
    const uint32_t k = (uint32_t)cfg.dense_k;
    L.filt_words = t.filter_words[k][width_index(cfg.filter_bits)];
    L.filt_u4 = L.filt_words / 4;
    uint32_t off = round16((uint64_t)L.filt_words * 4);
    L.off_dense = off;
    L.dense_u4 = k > 0 ? t.dense_words[k] / 2 : 0;  // the walkers' depth-k lookups
    off += L.dense_u4 * 16;
    L.off_lut = off;
    if (t.C != 256) off += 64 * 32 * 4;
    L.off_ring = off;
    off += kRing * 16 + kRing * 4 + (uint32_t)sizeof(Ring);
    off = round16(off);
    L.off_warp = off;
    L.halo = round16(t.max_len > 16 ? t.max_len : 16);
    L.stage_bytes = (uint32_t)cfg.tile + L.halo;
    L.off_stages = round16((uint64_t)kMaxStages * 8);
    L.warp_bytes = L.off_stages + (uint32_t)cfg.stages * L.stage_bytes;
    const uint32_t producers = (uint32_t)(cfg.threads / 32 - cfg.walkers);
    L.total = off + producers * L.warp_bytes;
    return L;
}

std::mutex g_attr_mu;

struct LaunchKey {
    const void *fn;
    uint32_t smem, threads;
    int device;
    bool operator<(const LaunchKey &o) const
    {
        if (fn != o.fn) return fn < o.fn;
        if (smem != o.smem) return smem < o.smem;
        if (threads != o.threads) return threads < o.threads;
        return device < o.device;
    }
};
std::map<LaunchKey, int> g_occ;  // guarded by g_attr_mu
// largest dynamic shared memory set per (kernel, device); only ever raised
std::map<std::pair<const void *, int>, uint32_t> g_smem_set;  // guarded by g_attr_mu

}  // namespace

uint64_t scan_smem_bytes(const TrieDev &t, const pm_config &cfg)
{
    return layout(t, cfg).total;
}

int launch_scan(const TrieDev &t, const pm_config &cfg, const ScanArgs &a, void *stream,
                int device_sms, std::string &msg)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool batch = a.offsets != nullptr;
    const uint32_t ncount = batch ? a.ntexts : 1;
    if (ncount && !a.keep_counts) {
        cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(int64_t) * ncount, st);
        if (e != cudaSuccess) {
            msg = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
    }
    if (a.lookups) {
        cudaError_t e = cudaMemsetAsync(a.lookups, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) {
            msg = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
    }
    if (batch ? a.ntexts == 0 : a.len == 0) return PM_OK;

    const int mode = a.lookups ? MODE_LOOKUPS : (cfg.checked ? MODE_CHECKED : MODE_FAST);
    KernelFn fn = pick_kernel(t.C, (uint32_t)cfg.dense_k, t.gram[cfg.dense_k], batch, mode);
    Layout L = layout(t, cfg);

    KParams p{};
    p.t = t;
    p.text = a.text;
    p.offsets = a.offsets;
    p.ntexts = a.ntexts;
    p.total = a.len;
    p.limit = a.limit > a.len ? a.limit : a.len;
    p.ids = a.ids;
    p.out_ids = a.out_ids;
    p.counts = a.counts;
    p.lookups = a.lookups;
    p.tile_counts = batch ? nullptr : a.tile_counts;
    p.walks = a.walks;
    p.tile = (uint32_t)cfg.tile;
    p.halo = L.halo;
    p.k = (uint32_t)cfg.dense_k;
    p.lw = cfg.filter_bits == 8 ? 3u : cfg.filter_bits == 16 ? 4u : 5u;
    p.filter = t.filter[cfg.dense_k][width_index(cfg.filter_bits)];
    p.dense = cfg.dense_k > 0 ? t.dense[cfg.dense_k] : nullptr;
    p.first_k = t.first[cfg.dense_k];
    p.ck1 = 1u;
    for (int32_t i = 1; i < cfg.dense_k; ++i) p.ck1 *= t.C;
    p.deep_on = cfg.deep && t.deep_k > 0 && t.C != 256 ? 1u : 0u;
    p.kload = (uint32_t)cfg.dense_k + 4u;
    p.uk1 = 1u;
    for (uint32_t i = 1; i < t.deep_k; ++i) p.uk1 *= t.deep_U;
    if (p.deep_on && t.deep_k + 4u > p.kload) p.kload = t.deep_k + 4u;
    p.gram = t.gram[cfg.dense_k];
    p.binary = cfg.row_search ? 1u : 0u;
    p.bitmap = cfg.layout == 1 ? 1u : 0u;
    p.stages = (uint32_t)cfg.stages;
    p.walkers = (uint32_t)cfg.walkers;
    p.aligned = ((uintptr_t)a.text & 15u) == 0;
    p.ids_aligned = ((uintptr_t)a.ids & 15u) == 0;
    p.off_dense = L.off_dense;
    p.off_lut = L.off_lut;
    p.off_ring = L.off_ring;
    p.off_warp = L.off_warp;
    p.warp_bytes = L.warp_bytes;
    p.off_stages = L.off_stages;
    p.stage_bytes = L.stage_bytes;
    p.filt_u4 = L.filt_u4;
    p.dense_u4 = L.dense_u4;
    p.filt_words = L.filt_words;

    cudaError_t e;
    int occ = 0;
    {
        // the shared-memory attribute and the occupancy of each (kernel,
        // shared bytes, threads, device) are set and queried once
        int dev = -1;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) {
            msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
        const LaunchKey key{reinterpret_cast<const void *>(fn), L.total, (uint32_t)cfg.threads, dev};
        std::lock_guard<std::mutex> g(g_attr_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) {
            occ = it->second;
        } else {
            uint32_t &set = g_smem_set[{key.fn, dev}];
            if (set < L.total) {
                e = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
                if (e != cudaSuccess) {
                    msg = std::string("shared memory ") + std::to_string(L.total) +
                          " bytes: " + cudaGetErrorString(e);
                    return PM_ERR_INVAL;
                }
                set = L.total;
            }
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, reinterpret_cast<const void *>(fn), cfg.threads, L.total);
            if (e != cudaSuccess || occ < 1) {
                msg = "configuration does not fit on an SM (threads " +
                      std::to_string(cfg.threads) + ", shared " + std::to_string(L.total) + ")";
                return PM_ERR_INVAL;
            }
            g_occ.emplace(key, occ);
        }
    }
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < occ) occ = cfg.ctas_per_sm;
    unsigned long long grid = (unsigned long long)device_sms * occ;
    const unsigned long long known = batch ? a.total_hint : a.len;
    if (known) {
        const unsigned long long warps = cfg.threads / 32 - cfg.walkers;
        unsigned long long ntiles = (known + cfg.tile - 1) / cfg.tile;
        unsigned long long need = (ntiles + warps - 1) / warps;
        if (need < grid) grid = need;
    }
    fn<<<(unsigned)grid, cfg.threads, L.total, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        msg = std::string("scan launch: ") + cudaGetErrorString(e);
        return PM_ERR_CUDA;
    }
    if (batch && a.out_counts) {
        pm_counts_scatter_kernel<<<(a.ntexts + 255) / 256, 256, 0, st>>>(a.counts, a.out_counts,
                                                                         a.ntexts);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            msg = std::string("count scatter launch: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
    }
    return PM_OK;
}

int read_device_error(int *code, std::string &msg)
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_pm_dev_error, sizeof(int));
    if (e == cudaSuccess) {
        int z = 0;
        e = cudaMemcpyToSymbol(g_pm_dev_error, &z, sizeof(int));
    }
    if (e != cudaSuccess) {
        msg = std::string("device error word: ") + cudaGetErrorString(e);
        return PM_ERR_CUDA;
    }
    *code = v;
    return PM_OK;
}

}  // namespace pm
