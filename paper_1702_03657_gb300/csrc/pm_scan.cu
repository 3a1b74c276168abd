// PFAC scan kernels for sm_103a (Section II-C: one failure-less walk per
// start position over the CRS trie of Section III).
//
// One persistent kernel serves the single-text and the batched scan, one CTA
// per SM. After the CTA loads its shared-memory filter (its only CTA-wide
// barrier), every warp is an independent pipeline over its own text tiles:
//  a1 staging   lane 0 streams tile + halo (>= longest pattern) into one of
//               `stages` shared-memory buffers with a 1-D TMA bulk copy
//               completing on an mbarrier, `stages` tiles ahead (text whose
//               base is not 16-byte aligned is staged with plain loads);
//  a2 filter    P consecutive start positions per lane (P = 4 or 8):
//               byte alphabet: a blocked Bloom probe of each position's
//                 4-gram (or an exact test of short grams) in shared memory;
//               byte classes: each lane packs the classes of its P bytes
//                 (cb bits each, from a lane-replicated table), takes its
//                 neighbours' packed classes by warp shuffles, and tests each
//                 position's F-gram in an exact shared-memory bitmap, then
//                 the D-gram of each passing position in the deep level's
//                 bitmap (L2);
//               a position that fails cannot match (F, D and the Bloom gram
//               are at most the shortest pattern);
//  a4 -1        every position gets -1 (16-byte streaming stores);
//     queue     each remaining walk (start position, how it starts) goes to
//               the warp's own queue in shared memory (ballot/popc
//               compaction, no atomics); whenever 32 are queued the warp runs
//               them as one round, one walk per lane;
//  a3 CRS walk  a walk first resolves its start node (the dense table of
//               level k, the deep level's rank, or the root), then reads each
//               node's 16-byte row record (row start, length, has-match bit,
//               first eight column bytes) with the next text byte; the child
//               of non-zero e is node e + 1 (BFS order); longer rows are
//               searched in the column array. With layout 1 the walk reads
//               the bitmapped nodes of Section III instead (256-bit child
//               bitmap + first child, rank gives the child);
//  a4 emit      ids[i] = best[v], count += nfinal[v] of the deepest node v;
//               the queue's rounds run in the warp that wrote the -1, after a
//               __syncwarp, so the patch lands after it;
//  a5 reduce    per-lane counts, warp shuffle reduction, one atomic per warp
//               (per match and text in batch mode).
//
// Every mbarrier wait is bounded by a clock budget (pm_config.wait_clocks,
// default about 2 s); on expiry the warp records PM_ERR_TIMEOUT in a device
// word, waits with the full budget for its copies in flight and stops. The
// checked variant bounds-checks every shared and global index and records
// PM_ERR_BOUNDS instead of touching memory out of range.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "pm_internal.h"

namespace pm {

__device__ int g_pm_dev_error;

namespace {

constexpr long long kWaitBudget = 4000000000LL;  // SM clocks (~2 s)
constexpr uint32_t kSuspendHintNs = 1000000u;      // 1 ms per try_wait
constexpr int kMaxStages = 4;
constexpr uint32_t kQueue = 64;                    // walk queue entries per warp
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kMaxNeighbours = 8;                  // byte classes: chunks a window takes
constexpr uint32_t kStagePad = 16;                 // bytes past tile + halo a lane may read
constexpr uint32_t kWarpHeader = 32;               // mbarriers of a warp's block
constexpr uint32_t kChunkRing = 16;                // run starts a CTA keeps published

enum Mode { MODE_FAST = 0, MODE_CHECKED = 1, MODE_LOOKUPS = 2 };

// How a queued walk starts (bits 61..62 of its position word): from the
// root; from the depth-k node of the byte alphabet's dense table; from the
// depth-D node of the byte classes' deep level. The code word holds the
// k-gram or D-gram for the last two.
enum WalkKind : uint32_t { WALK_ROOT = 0, WALK_DENSE = 1, WALK_DEEP = 2 };
constexpr unsigned long long kPosMask = (1ull << 40) - 1;

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
    uint32_t *match_bits;       // with tile_counts: a bit per position with a match
    unsigned long long *walks;  // optional: walks run
    unsigned int *chunk_ctr;    // dynamic schedule: runs of tiles handed out (zeroed), or null
    const uint32_t *filter;     // source of the shared-memory filter (or null)
    const uint2 *dense;         // byte alphabet: dense table of level k (global)
    uint32_t first_k;           // byte alphabet: BFS id of the first depth-k node
    uint32_t gram;              // bytes the filter tests per position
    uint32_t cb;                // byte classes: bits per class
    uint32_t F;                 // byte classes: filter depth (0: none)
    uint32_t D;                 // byte classes: deep level depth (0: not used)
    uint32_t nnb;               // byte classes: neighbour chunks a lane's window takes
    uint32_t tile;
    uint32_t halo;
    uint32_t k;
    uint32_t lw;                // log2 W (byte alphabet)
    uint32_t binary;
    uint32_t bitmap;            // walks read bitmapped nodes instead of row records
    uint32_t stages;
    uint32_t aligned;
    uint32_t ids_aligned;
    long long wait_budget;      // SM clocks per TMA wait
    uint32_t light_add;         // light form, one CTA: add to the count, not overwrite
    // shared-memory layout (byte offsets)
    uint32_t off_lut, off_warp;   // class table, then the per-warp blocks
    uint32_t off_sched;           // after the warp blocks: ticket counter, run ring
    uint32_t warp_bytes;          // bytes of one warp's block
    uint32_t off_queue;           // inside a warp's block (after its mbarriers)
    uint32_t off_stages;          // inside a warp's block (after its queue)
    uint32_t stage_bytes;         // tile + halo + pad
    uint32_t filt_u4;             // filter size in 16-byte units
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase), "r"(hint_ns)
        : "memory");
    return done != 0;
}

// Non-blocking test of the phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return done != 0;
}

// Bounded wait: false if the phase did not complete within `budget` clocks.
// Budgets of a few milliseconds or more wait in suspending try_waits (1 ms
// hint each); shorter ones poll with test_wait, since a suspended thread may
// only wake when the phase completes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, long long budget)
{
    const long long t0 = clock64();
    if (budget < 8ll * kSuspendHintNs) {
        while (!mbar_test_wait(bar, phase)) {
            if (clock64() - t0 > budget) return false;
        }
        return true;
    }
    while (!mbar_try_wait(bar, phase, kSuspendHintNs)) {
        if (clock64() - t0 > budget) return false;
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
    const unsigned long long want = (unsigned long long)p.tile + p.halo;
    const unsigned long long left = end - t0;
    return left < want ? left : want;
}

// Issue the TMA copy of the tile at text offset t0 into stage `s` of a warp
// (lane 0).
__device__ __forceinline__ void issue_tile(const KParams &p, uint8_t *stages, uint64_t *bars,
                                           uint32_t s, unsigned long long t0,
                                           unsigned long long end)
{
    const uint32_t nb = (uint32_t)tile_bytes(p, t0, end);
    const uint32_t nb16 = nb & ~15u;
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
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
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

// A walk from position pos ended at a node whose emit is {best, nfinal}
// after matching `depth` bytes: writes the position's id and adds its count
// when a pattern ends on the path.
template <bool BATCH>
__device__ __forceinline__ void emit_values(const KParams &p, unsigned long long pos, uint32_t txt,
                                            uint32_t depth, int2 em, unsigned long long &acc)
{
    if (depth < p.t.min_len || em.y <= 0) return;
    if (BATCH && p.out_ids)
        p.out_ids[txt][pos - __ldg(p.offsets + txt)] = em.x;
    else
        p.ids[pos] = em.x;
    if (BATCH) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p.counts + txt), (unsigned long long)em.y);
    } else {
        acc += (unsigned)em.y;
        if (p.tile_counts) {
            atomicAdd(p.tile_counts + (pos >> kMatchTileShift), (unsigned)em.y);
            atomicOr(p.match_bits + (pos >> 5), 1u << (pos & 31u));
        }
    }
}

// A walk from position pos ended at node v after matching `depth` bytes;
// has: v's has-match bit (2: not read).
template <bool BATCH>
__device__ __forceinline__ void emit_walk(const KParams &p, unsigned long long pos, uint32_t txt,
                                          uint32_t v, uint32_t depth, uint32_t has,
                                          unsigned long long &acc)
{
    if (depth < p.t.min_len || has == 0u) return;
    emit_values<BATCH>(p, pos, txt, depth, __ldg(p.t.emit + v), acc);
}

// Number of leading bytes on which a[0 .. n) and lab[0 .. n) agree, 16
// bytes at a time: both are read as aligned 32-bit words, a text word only
// when it holds a byte below a + n (lab is padded past its end).
__device__ __forceinline__ uint32_t chain_match(const uint8_t *a, uint32_t n, const uint8_t *lab,
                                                uint64_t pol)
{
    const uintptr_t aend = (uintptr_t)(a + n);
    uint32_t m = 0;
    while (m < n) {
        const uintptr_t ta = (uintptr_t)(a + m), la = (uintptr_t)(lab + m);
        const uint32_t *tw = reinterpret_cast<const uint32_t *>(ta & ~(uintptr_t)3);
        const uint32_t *lw = reinterpret_cast<const uint32_t *>(la & ~(uintptr_t)3);
        const uint32_t ts = (uint32_t)(ta & 3u) * 8u, ls = (uint32_t)(la & 3u) * 8u;
        uint32_t x[5], y[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            x[k] = (uintptr_t)(tw + k) < aend ? __ldg(tw + k) : 0u;
            y[k] = ld_trie_u32(lw + k, pol);
        }
        uint32_t d = 16;
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            const uint32_t z = __funnelshift_r(x[k], x[k + 1], ts) ^ __funnelshift_r(y[k], y[k + 1], ls);
            if (z) d = 4u * k + ((uint32_t)(__ffs(z) - 1) >> 3);
        }
        m += d;
        if (d < 16) break;
    }
    return m < n ? m : n;
}

// The node at which a rank table (uint2 {bits, base} per 32 codes) places
// `code`: first + base + set bits below it, or 0xFFFFFFFF if its bit is
// clear (the gram is not a root path).
template <int MODE>
__device__ __forceinline__ uint32_t rank_node(const uint2 *tab, uint32_t words, uint32_t first,
                                              uint32_t code, uint64_t pol)
{
    if (MODE == MODE_CHECKED && (code >> 5) >= words) {
        record_error(PM_ERR_BOUNDS);
        return 0xFFFFFFFFu;
    }
    const uint2 d = ld_trie_u2(tab + (code >> 5), pol);
    const uint32_t bit = code & 31u;
    if (!((d.x >> bit) & 1u)) return 0xFFFFFFFFu;
    return first + d.y + __popc(d.x & ((1u << bit) - 1u));
}

// Run one queued walk (Section II-C): resolve its start node, then read
// each node's row record and the next text byte together, move to the child
// on that byte, and stop at a mismatch, a leaf or the text end; then patch
// the position's id when a pattern ends on the path.
template <bool BATCH, int MODE>
__device__ __forceinline__ void run_walk(const KParams &p, unsigned long long qp, uint32_t code,
                                         unsigned long long end, uint64_t pol,
                                         unsigned long long &acc, unsigned long long &look,
                                         unsigned long long &nwalk)
{
    const TrieDev &t = p.t;
    const unsigned long long pos = qp & kPosMask;
    const uint32_t kind = (uint32_t)(qp >> 61) & 3u;
    uint32_t jo = 0, v = 0;
    if (kind == WALK_DENSE) {
        v = rank_node<MODE>(p.dense, t.dense_words[p.k], p.first_k, code, pol);
        if (v == 0xFFFFFFFFu) return;  // the k-gram is not a root path
        jo = p.k;
    } else if (kind == WALK_DEEP) {
        v = rank_node<MODE>(t.deep, t.deep_words, t.deep_first, code, pol);
        if (v == 0xFFFFFFFFu) return;
        jo = t.deep_k;
    }
    ++nwalk;
    uint32_t txt = 0;
    unsigned long long tend = end;
    if (BATCH) {
        txt = find_text(p.offsets, p.ntexts, pos);
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
        if (MODE != MODE_LOOKUPS && deg == 1u && (r.z >> 8) >= 2u) {
            // a unary chain: the next R edges are forced; compare the text
            // with their labels in one go and land on the node reached
            const uint32_t R = r.z >> 8, ci = r.w;
            if (MODE == MODE_CHECKED && (ci >= t.ch_len || R > t.ch_len - 1u - ci)) {
                record_error(PM_ERR_BOUNDS);
                return;
            }
            const uint32_t m = chain_match(tp + jo, min(R, te - jo), t.ch_lab + ci, pol);
            const int2 inf = __ldg(t.ch_info + ci + m);
            jo += m;
            if (m < R) {  // stopped inside the chain: mismatch or text end
                emit_values<BATCH>(p, pos, txt, jo, inf, acc);
                return;
            }
            v = (uint32_t)inf.x;  // the chain's end node
            has = 2u;
            continue;
        }
        const uint32_t ei = row_find(t.col, r.x, deg, r.z, r.w, b, p.binary, pol);
        if (ei == 0xFFFFFFFFu) break;
        v = ei + 1u;  // BFS order: the child of non-zero e is node e + 1
        ++jo;
        has = 2u;
    }
    emit_walk<BATCH>(p, pos, txt, v, jo, has, acc);
}

// Classes of the P bytes at st[o .. o + P), packed msb-first (byte o's class
// in the top cb bits of a P*cb-bit chunk), from the lane-replicated table
// (word (b/4)*32 + lane holds the entries of bytes 4*(b/4) .. +3, so lane l
// always reads bank l); *oth (meaningful with other_check, where classes
// take at most 7 bits): some byte is of the "other" class.
template <int P>
__device__ __forceinline__ uint32_t classify(const uint8_t *st, const uint32_t *s_lut,
                                             uint32_t lane, uint32_t cb, uint32_t &oth)
{
    const uint32_t cmask = (1u << cb) - 1u;
    uint32_t c = 0, o = 0;
#pragma unroll
    for (int w = 0; w < P / 4; ++w) {
        const uint32_t word = *reinterpret_cast<const uint32_t *>(st + 4 * w);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t b = (word >> (8 * j)) & 0xFFu;
            const uint32_t v = (s_lut[(b >> 2) * 32 + lane] >> ((b & 3u) * 8u)) & 0xFFu;
            c = (c << cb) | (v & cmask);
            o |= v;
        }
    }
    oth = o >> 7;
    return c;
}

// The P bytes at s (P-byte aligned in shared memory) as P/4 little-endian
// words in w[0 .. P/4), read as wide as their alignment allows, and the 4
// bytes after them in w[P/4].
template <int P>
__device__ __forceinline__ void load_words(const uint8_t *s, uint32_t *w)
{
    if constexpr (P % 16 == 0) {
#pragma unroll
        for (int j = 0; j < P / 16; ++j) {
            const uint4 v = *reinterpret_cast<const uint4 *>(s + 16 * j);
            w[4 * j] = v.x;
            w[4 * j + 1] = v.y;
            w[4 * j + 2] = v.z;
            w[4 * j + 3] = v.w;
        }
    } else if constexpr (P == 8) {
        const uint2 v = *reinterpret_cast<const uint2 *>(s);
        w[0] = v.x;
        w[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < P / 4; ++j) w[j] = *reinterpret_cast<const uint32_t *>(s + 4 * j);
    }
    w[P / 4] = *reinterpret_cast<const uint32_t *>(s + P);
}

// Shifts bit 0 of r in at the top of acc: after P steps the first step's bit
// is at bit 32 - P and the last's at bit 31, so acc >> (32 - P) has step q's
// bit at bit q.
__device__ __forceinline__ uint32_t funnel_in(uint32_t acc, uint32_t r)
{
    return __funnelshift_r(acc, r, 1);
}

// classify for four letters told apart by the field f = (b >> sh) & 7, four
// bytes at a time: the fields of a word become a byte-permute selector, which
// reads each byte's class and letter out of the 8-byte tables (cl, sy). A
// byte that differs from its field's letter is of no pattern (oth = 1). The
// four 2-bit classes are packed first byte highest by one multiply: class j
// sits at bit 8j and is moved to bit 30 - 2j, and no two partial products
// overlap in bits 24..31.
template <int P>
__device__ __forceinline__ uint32_t classify4(const uint8_t *st, uint32_t sh, uint32_t cl0,
                                              uint32_t cl1, uint32_t sy0, uint32_t sy1,
                                              uint32_t &oth)
{
    uint32_t c = 0;
    bool bad = false;
#pragma unroll
    for (int w = 0; w < P / 4; ++w) {
        const uint32_t word = *reinterpret_cast<const uint32_t *>(st + 4 * w);
        const uint32_t f = (word >> sh) & 0x07070707u;
        // byte j of f | f >> 4 holds f_j | f_{j+1} << 4: bytes 0 and 2
        // give the four selector nibbles
        const uint32_t sel = __byte_perm(f | (f >> 4), 0u, 0x20u);
        bad |= __byte_perm(sy0, sy1, sel) != word;
        c = (c << 8) | ((__byte_perm(cl0, cl1, sel) * 0x40100401u) >> 24);
    }
    oth = bad ? 1u : 0u;
    return c;
}

// KF: the byte alphabet's filter level k (0, 1, 2), or -1 for byte classes.
// G: bytes the byte alphabet's Bloom filter tests (3 or 4), 0 otherwise.
// P: start positions per lane and group.
// CB, FC, DC (byte classes): bits per class, filter depth and deep-level
// depth fixed at compile time (all shifts of the packed codes become
// constants), or 0 when taken from the parameters at run time.
template <int KF, int G, bool IDENT, bool BATCH, int MODE, int P, int CB = 0, int FC = 0, int DC = 0>
__global__ void __launch_bounds__(1024, 1) pfac_scan_kernel(const KParams p)
{
    constexpr bool FIXED = CB > 0 && FC > 0 && DC > 0;
    constexpr uint32_t NNBC = FIXED ? ((FC > DC ? FC : DC) - 1 + P - 1) / P : 0;
    extern __shared__ __align__(16) uint8_t smem[];
    const TrieDev &t = p.t;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t NW = blockDim.x >> 5;
    constexpr uint32_t GP = 32 * P;  // positions per group

    const unsigned long long total = BATCH ? __ldg(p.offsets + p.ntexts) : p.total;
    const unsigned long long end = BATCH ? total : p.limit;
    const unsigned long long ntiles = (total + p.tile - 1) / p.tile;
    if ((unsigned long long)blockIdx.x * NW >= ntiles) return;

    uint32_t *s_filt = reinterpret_cast<uint32_t *>(smem);
    uint32_t *s_lut = reinterpret_cast<uint32_t *>(smem + p.off_lut);
    // dynamic schedule: the CTA's tickets (one per tile a warp takes) and the
    // global runs of its local runs m, published as {m, run} in slot m % ring
    unsigned long long *s_run = reinterpret_cast<unsigned long long *>(smem + p.off_sched);
    unsigned int &s_tick = *reinterpret_cast<unsigned int *>(smem + p.off_sched + 8 * kChunkRing);
    if (p.chunk_ctr != nullptr && tid == 0) {
        s_tick = 0;
        // local runs 0 and 1 now, in order; the other slots read as not yet
        // published (their m is behind any run asked for)
        s_run[0] = atomicAdd(p.chunk_ctr, 1u);
        s_run[1] = (1ull << 32) | atomicAdd(p.chunk_ctr, 1u);
        for (uint32_t i = 2; i < kChunkRing; ++i)
            s_run[i] = (unsigned long long)(i - kChunkRing) << 32;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.filter);
        uint4 *dst = reinterpret_cast<uint4 *>(s_filt);
        for (uint32_t i = tid; i < p.filt_u4; i += blockDim.x) dst[i] = __ldg(src + i);
        if (!IDENT) {
            // class table replicated per lane (see classify)
            for (uint32_t i = tid; i < 64 * 32; i += blockDim.x) {
                const uint32_t w = i >> 5;
                s_lut[i] = (uint32_t)__ldg(t.cls + 4 * w) | ((uint32_t)__ldg(t.cls + 4 * w + 1) << 8) |
                           ((uint32_t)__ldg(t.cls + 4 * w + 2) << 16) |
                           ((uint32_t)__ldg(t.cls + 4 * w + 3) << 24);
            }
        }
    }
    __syncthreads();  // the only CTA-wide barrier: warps run independently below

    const uint64_t pol = policy_evict_last();
    unsigned long long acc = 0;    // matches (single text)
    unsigned long long look = 0;   // lookups (MODE_LOOKUPS)
    unsigned long long nwalk = 0;  // walks run
    const unsigned long long gw = (unsigned long long)blockIdx.x * NW + warp;
    // The warp's next tile (lane 0; start byte, kNoTile past the last, or
    // kFailTile when a bounded wait ran out). Static: tiles gw, gw + W, ... (W
    // warps in the grid).
    // Dynamic: ticket j of the CTA is tile j % PM_CHUNK_TILES of the CTA's
    // local run j / PM_CHUNK_TILES. The taker of a run's first ticket asks
    // the global counter for the run two ahead, once the run one ahead is
    // published: global runs then grow with m, so past the first missing
    // tile every later ticket misses too, and a warp stops at its first.
    // (what grab needs is re-read from the parameters at each call, so that
    // no more than the static cursor stays live across the tile loop)
    constexpr unsigned long long kNoTile = ~0ull, kFailTile = ~1ull;
    unsigned long long st_next = gw * p.tile;  // static: start of the warp's next tile
    auto run_of = [&](uint32_t m, unsigned long long &run) -> bool {
        const volatile unsigned long long *slot = s_run + m % kChunkRing;
        unsigned long long e = *slot;
        if ((uint32_t)(e >> 32) == m) {  // published (the usual case)
            run = (uint32_t)e;
            return true;
        }
        const long long t_end = clock64() + p.wait_budget;
        for (;;) {
            const int d = (int)((uint32_t)(e >> 32) - m);
            if (d == 0) {
                run = (uint32_t)e;
                return true;
            }
            if (d > 0 || clock64() > t_end) return false;  // overwritten / ran out
            __nanosleep(64);
            e = *slot;
        }
    };
    auto grab = [&]() -> unsigned long long {
        const unsigned long long tot = BATCH ? __ldg(p.offsets + p.ntexts) : p.total;
        if (p.chunk_ctr == nullptr) {
            const unsigned long long ts = st_next;
            st_next += (unsigned long long)gridDim.x * (blockDim.x >> 5) * p.tile;
            return ts < tot ? ts : kNoTile;
        }
        const uint32_t j = atomicAdd(&s_tick, 1u);
        const uint32_t m = j / PM_CHUNK_TILES, o = j % PM_CHUNK_TILES;
        unsigned long long run;
        if (o == 0) {
            if (!run_of(m + 1, run)) return kFailTile;
            const uint32_t g = atomicAdd(p.chunk_ctr, 1u);
            *(volatile unsigned long long *)(s_run + (m + 2) % kChunkRing) =
                ((unsigned long long)(m + 2) << 32) | g;
        }
        if (!run_of(m, run)) return kFailTile;
        const unsigned long long ts = (run * PM_CHUNK_TILES + o) * p.tile;
        return ts < tot ? ts : kNoTile;
    };

    {
        uint8_t *wsm = smem + p.off_warp + (size_t)warp * p.warp_bytes;
        uint64_t *bars = reinterpret_cast<uint64_t *>(wsm);
        unsigned long long *qpos = reinterpret_cast<unsigned long long *>(wsm + p.off_queue);
        uint32_t *qcode = reinterpret_cast<uint32_t *>(wsm + p.off_queue + 8 * kQueue);
        uint8_t *stages = wsm + p.off_stages;
        const uint32_t below = (1u << lane) - 1u;

        // the warp's walk queue: entries qh .. qh + qn (mod kQueue)
        uint32_t qh = 0, qn = 0;
        auto round = [&](uint32_t n) {  // run the first n (<= 32) queued walks
            if (lane < n) {
                const uint32_t idx = (qh + lane) & (kQueue - 1);
                run_walk<BATCH, MODE>(p, qpos[idx], qcode[idx], end, pol, acc, look, nwalk);
            }
            qh += n;
            qn -= n;
            __syncwarp();
        };

        bool failed = false;
        // start byte of stage s's tile, held by lane s (kNoTile: none); a
        // register, not shared memory (the shared bytes per CTA decide the
        // L1 the SM keeps beside them)
        unsigned long long my_ts = kNoTile;
        // (whole warp) lane 0 takes the next tile into stage s and starts its
        // copy; lane s keeps the tile's start
        auto refill = [&](uint32_t s) {
            unsigned long long ts = kNoTile;
            if (lane == 0) {
                ts = grab();
                if (ts == kFailTile) {
                    record_error(PM_ERR_TIMEOUT);
                    ts = kNoTile;
                }
                if (ts != kNoTile) issue_tile(p, stages, bars, s, ts, end);
            }
            ts = __shfl_sync(kFull, ts, 0);
            if (lane == s) my_ts = ts;
        };
        if (lane == 0) {
            for (uint32_t s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncwarp();  // the initialised barriers, before any lane tests them
        for (uint32_t s = 0; s < p.stages; ++s) refill(s);

        const uint32_t lw = p.lw;
        // byte alphabet, exact levels: filter bit index = low 8k+lw bits of
        // the little-endian window
        constexpr uint32_t KFU = KF > 0 ? (uint32_t)KF : 0u;
        const uint32_t imask = KF >= 0 ? (uint32_t)((1ull << (8 * KFU + lw)) - 1ull) : 0u;
        // byte classes: bits of one lane's chunk, code shifts
        const uint32_t cb = CB ? (uint32_t)CB : p.cb, Pcb = P * cb;
        const uint32_t Fv = FIXED ? (uint32_t)FC : p.F, Dv = FIXED ? (uint32_t)DC : p.D;
        const uint32_t nnb = FIXED ? NNBC : p.nnb;
        // four letters with a telling 3-bit field (fixed shapes only)
        const bool sw = FIXED && t.sw_shift != kNoSwar;
        const uint32_t shF = 32u - cb * Fv, shD = 32u - cb * Dv;  // used only when F, D > 0
        const uint32_t span = (p.gram > 1 ? p.gram : 1u) - 1u;  // bytes a position's filter reads past it

        // the stages hold the warp's tiles in the order taken; the first
        // stage without one ends the warp's work
        uint32_t s = 0, phase = 0;  // stage and its mbarrier phase
        while (!failed) {
            const unsigned long long t0 = __shfl_sync(kFull, my_ts, s);  // the current tile
            if (t0 == kNoTile) break;
            const uint32_t nbytes = (uint32_t)tile_bytes(p, t0, end);
            uint8_t *st = stages + (size_t)s * p.stage_bytes;

            const bool ok = __all_sync(kFull, mbar_wait_bounded(&bars[s], phase, p.wait_budget));
            if (!ok) {
                // copies still in flight: every stage holding a tile
                const uint32_t held = __ballot_sync(kFull, lane < p.stages && my_ts != kNoTile);
                if (lane == 0) {
                    record_error(PM_ERR_TIMEOUT);
                    for (uint32_t j = 0; j < p.stages; ++j) {  // (full budget)
                        const uint32_t sj = (s + j) % p.stages;
                        if ((held >> sj) & 1u)
                            mbar_wait_bounded(&bars[sj], phase ^ (uint32_t)((s + j) >= p.stages),
                                              kWaitBudget);
                    }
                }
                failed = true;
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
                cur = find_text(p.offsets, p.ntexts, t0 + P * lane < total ? t0 + P * lane : t0);
                text_end = __ldg(p.offsets + cur + 1);
            }
            uint32_t rel_end = rel_end_of(text_end, t0);
            // groups [lp0, lp0+P) with lp0 + P <= fast_n take the fast path
            auto fast_bound = [&]() -> uint32_t {
                const uint32_t r = rel_end >= span ? rel_end - span : 0u;
                return r < tile_n ? r : tile_n;
            };
            uint32_t fast_n = fast_bound();
            int32_t *idt = p.ids + t0;  // this tile's ids

            // byte classes: the lane's chunk of the current group (carried
            // from the previous group's look-ahead)
            uint32_t cur_c = 0, cur_o = 0;
            if (!IDENT)
                cur_c = sw ? classify4<P>(st + P * lane, t.sw_shift, t.sw_cls[0], t.sw_cls[1],
                                          t.sw_sym[0], t.sw_sym[1], cur_o)
                           : classify<P>(st + P * lane, s_lut, lane, cb, cur_o);

            const uint32_t iters = (tile_n + GP - 1) / GP;
            for (uint32_t i = 0; i < iters; ++i) {
                const uint32_t lp0 = i * GP + P * lane;
                if (BATCH && lp0 < tile_n && t0 + lp0 >= text_end) {
                    while (t0 + lp0 >= text_end) {
                        ++cur;
                        text_end = __ldg(p.offsets + cur + 1);
                    }
                    rel_end = rel_end_of(text_end, t0);
                    fast_n = fast_bound();
                }
                const uint32_t cur0 = cur;  // text of position lp0
                uint32_t need = 0;   // bit q: position lp0+q starts a walk at level k / D
                uint32_t rootm = 0;  // bit q: position lp0+q is walked from the root
                uint32_t nxt_c = 0, nxt_o = 0;
                uint64_t X = 0;      // byte classes: packed classes from byte lp0 on
                bool fast = MODE != MODE_LOOKUPS && lp0 + P <= fast_n;
                if (!IDENT) {
                    // look ahead: the lane's chunk of the next group (read
                    // within the stage buffer; bytes past the staged ones
                    // only reach codes of positions that take the slow path)
                    if (lp0 + GP + P <= p.stage_bytes)
                        nxt_c = sw ? classify4<P>(st + lp0 + GP, t.sw_shift, t.sw_cls[0], t.sw_cls[1],
                                                  t.sw_sym[0], t.sw_sym[1], nxt_o)
                                   : classify<P>(st + lp0 + GP, s_lut, lane, cb, nxt_o);
                    X = (uint64_t)cur_c << (64u - Pcb);
#pragma unroll
                    for (int d = 1; d <= kMaxNeighbours; ++d) {
                        if ((uint32_t)d > nnb) break;
                        const uint32_t src = (lane + d) & 31u;
                        const uint32_t a = __shfl_sync(kFull, cur_c, src);
                        const uint32_t b = __shfl_sync(kFull, nxt_c, src);
                        X |= (uint64_t)(lane + d < 32 ? a : b) << (64u - (d + 1) * Pcb);
                    }
                    if (t.other_check &&
                        __any_sync(kFull, cur_o != 0 || (lane < nnb && nxt_o != 0)))
                        fast = false;  // a byte of no pattern: decide per position
                }
                if (fast) {
                    if (IDENT) {
                        // bytes lp0 .. lp0 + P + 3 (staged)
                        // (a lane's bytes start on a P-byte boundary of the
                        // 16-byte-aligned stage: one 16- or 8-byte load per
                        // 16 or 8 bytes, a quarter of the wavefronts of
                        // 4-byte loads at that lane stride)
                        uint32_t w[P / 4 + 1];
                        load_words<P>(st + lp0, w);
#define PM_WIN(q) ((q) % 4 == 0 ? w[(q) / 4] : __funnelshift_r(w[(q) / 4], w[(q) / 4 + 1], 8 * ((q) % 4)))
                        if (KF >= (int)kBloomK) {
                            // blocked Bloom test of the g-gram at each position
                            const uint32_t sh = 32u - (8u * KFU + lw - 5u);
                            const uint32_t gsh = G > 0 ? 32u - 8u * G : 32u - 8u * p.gram;
                            uint32_t acc_f = 0;  // see funnel_in
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const uint32_t win = PM_WIN(q);
                                // bytes q .. q+g-1, shifted to the top
                                const uint32_t h = __umulhi(G == 4 ? win : win << gsh, kBloomMul);
                                const uint32_t word = h >> sh;
                                uint32_t r = 0;
                                if (MODE == MODE_CHECKED && word >= p.filt_words) {
                                    record_error(PM_ERR_BOUNDS);
                                } else {
                                    // both Bloom bits, each rotated down to bit 0 (the
                                    // funnel shift takes its amount mod 32)
                                    const uint32_t val = s_filt[word];
                                    r = __funnelshift_r(val, val, h) & __funnelshift_r(val, val, h >> 5);
                                }
                                acc_f = funnel_in(acc_f, r);
                            }
                            need = acc_f >> (32 - P);
                        } else if (KF >= 0) {
                            uint32_t acc_f = 0;
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const uint32_t idx = PM_WIN(q) & imask;
                                const uint32_t word = idx >> 5;
                                uint32_t r = 0;
                                if (MODE == MODE_CHECKED && word >= p.filt_words) {
                                    record_error(PM_ERR_BOUNDS);
                                } else {
                                    const uint32_t val = s_filt[word];
                                    r = __funnelshift_r(val, val, idx);
                                }
                                acc_f = funnel_in(acc_f, r);
                            }
                            need = acc_f >> (32 - P);
                        }
                        if (KF == 0) {  // no dense level: passing positions walk from the root
                            rootm = need;
                            need = 0;
                        }
                    } else if (FIXED) {
                        // byte classes, shapes fixed at compile time: every
                        // code is a constant shift of the window
                        // (a code's low 5 bits, the bit in its word, are the
                        // low bits of the shifted window: the rotations below
                        // take their amount mod 32)
                        constexpr uint32_t FM = (1u << (CB * FC)) - 1u, DM = (1u << (CB * DC)) - 1u;
                        uint32_t acc_f = 0;
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const uint32_t a = (uint32_t)(X >> (64 - CB * (q + FC)));
                            uint32_t r = 0;
                            if (MODE == MODE_CHECKED && ((a & FM) >> 5) >= p.filt_words) {
                                record_error(PM_ERR_BOUNDS);
                            } else {
                                const uint32_t val = s_filt[(a & FM) >> 5];
                                r = __funnelshift_r(val, val, a);
                            }
                            acc_f = funnel_in(acc_f, r);
                        }
                        need = acc_f >> (32 - P);
                        if (need) {
                            if (lp0 + (P - 1) + DC > rel_end) {
                                // positions whose D-gram leaves the text walk
                                // from the root
#pragma unroll
                                for (int q = 0; q < P; ++q)
                                    if (((need >> q) & 1u) && lp0 + q + DC > rel_end) {
                                        need &= ~(1u << q);
                                        rootm |= 1u << q;
                                    }
                            }
                            if (DC > FC && need) {
                                // the D-gram's bit in the deep level (L2):
                                // eight loads issued, then tested (a position
                                // not tested keeps word 0: bit clear); with
                                // sixteen positions, in two halves
                                constexpr int H = P < 8 ? P : 8;
                                uint32_t acc_d = 0;
#pragma unroll
                                for (int h0 = 0; h0 < P; h0 += H) {
                                    uint32_t dw[H];
#pragma unroll
                                    for (int k = 0; k < H; ++k) {
                                        const int q = h0 + k;
                                        dw[k] = 0;
                                        if (!((need >> q) & 1u)) continue;
                                        const uint32_t code = (uint32_t)(X >> (64 - CB * (q + DC))) & DM;
                                        if (MODE == MODE_CHECKED && (code >> 5) >= t.deep_words) {
                                            record_error(PM_ERR_BOUNDS);
                                            continue;
                                        }
                                        dw[k] = ld_trie_u32(t.deep + (code >> 5), pol);
                                    }
#pragma unroll
                                    for (int k = 0; k < H; ++k) {
                                        const uint32_t a = (uint32_t)(X >> (64 - CB * (h0 + k + DC)));
                                        acc_d = funnel_in(acc_d, __funnelshift_r(dw[k], dw[k], a));
                                    }
                                }
                                need = acc_d >> (32 - P);
                            }
                        }
                    } else {
                        // byte classes: the F-gram at each position in the
                        // exact shared-memory bitmap
                        if (p.F == 0) {
                            need = (uint32_t)((1ull << P) - 1ull);
                        } else {
                            uint64_t Xq = X;
                            uint32_t acc_f = 0;
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const uint32_t code = (uint32_t)(Xq >> 32) >> shF;
                                Xq <<= cb;
                                uint32_t r = 0;
                                if (MODE == MODE_CHECKED && (code >> 5) >= p.filt_words) {
                                    record_error(PM_ERR_BOUNDS);
                                } else {
                                    const uint32_t val = s_filt[code >> 5];
                                    r = __funnelshift_r(val, val, code);
                                }
                                acc_f = funnel_in(acc_f, r);
                            }
                            need = acc_f >> (32 - P);
                        }
                        if (need) {
                            if (p.D == 0) {
                                rootm = need;  // no deep level: walk from the root
                                need = 0;
                            } else {
                                // positions whose D-gram leaves the text walk
                                // from the root
                                if (lp0 + (P - 1) + p.D > rel_end) {
#pragma unroll
                                    for (int q = 0; q < P; ++q)
                                        if (((need >> q) & 1u) && lp0 + q + p.D > rel_end) {
                                            need &= ~(1u << q);
                                            rootm |= 1u << q;
                                        }
                                }
                                if (p.D > p.F && need) {
                                    // the D-gram's bit in the deep level (L2):
                                    // all loads issued, then tested (a
                                    // position not tested keeps word 0)
                                    uint32_t dw[P];
#pragma unroll
                                    for (int q = 0; q < P; ++q) {
                                        dw[q] = 0;
                                        if (!((need >> q) & 1u)) continue;
                                        const uint32_t code = (uint32_t)((X << (cb * q)) >> 32) >> shD;
                                        if (MODE == MODE_CHECKED && (code >> 5) >= t.deep_words) {
                                            record_error(PM_ERR_BOUNDS);
                                            continue;
                                        }
                                        dw[q] = ld_trie_u32(t.deep + (code >> 5), pol);
                                    }
                                    uint32_t acc_d = 0;
#pragma unroll
                                    for (int q = 0; q < P; ++q) {
                                        const uint32_t code = (uint32_t)((X << (cb * q)) >> 32) >> shD;
                                        acc_d = funnel_in(acc_d, __funnelshift_r(dw[q], dw[q], code));
                                    }
                                    need = acc_d >> (32 - P);
                                }
                            }
                        }
                    }
                } else {
                    // ragged group (tile end, text boundary, last bytes of a
                    // text, a byte of no pattern): every position that passes
                    // the filter, or that is too close to its text end to
                    // test, is walked from the root
                    for (uint32_t q = 0; q < P; ++q) {
                        const uint32_t lp = lp0 + q;
                        if (lp >= tile_n) break;
                        if (BATCH) {
                            while (t0 + lp >= text_end) {
                                ++cur;
                                text_end = __ldg(p.offsets + cur + 1);
                            }
                            rel_end = rel_end_of(text_end, t0);
                            fast_n = fast_bound();
                        }
                        if (MODE == MODE_LOOKUPS || lp + p.gram > rel_end) {
                            rootm |= 1u << q;
                            continue;
                        }
                        uint32_t word = 0, bits = 0;
                        if (IDENT && KF >= (int)kBloomK) {
                            uint32_t x = 0;
                            for (uint32_t j = 0; j < p.gram; ++j) x |= (uint32_t)st[lp + j] << (8 * j);
                            const BloomProbe b = bloom_probe(x, p.gram, 8u * KFU + lw - 5u);
                            word = b.word;
                            bits = b.mask;
                        } else if (IDENT && KF >= 0) {
                            uint32_t x = 0;
                            for (uint32_t j = 0; j <= KFU; ++j) x |= (uint32_t)st[lp + j] << (8 * j);
                            const uint32_t idx = x & imask;
                            word = idx >> 5;
                            bits = 1u << (idx & 31u);
                        } else {
                            if (p.F == 0) {
                                rootm |= 1u << q;
                                continue;
                            }
                            uint32_t code = 0, oth = 0;
                            for (uint32_t j = 0; j < p.F; ++j) {
                                const uint32_t b = st[lp + j];
                                const uint32_t v = (s_lut[(b >> 2) * 32 + lane] >> ((b & 3u) * 8u)) & 0xFFu;
                                code = (code << cb) | (v & ((1u << cb) - 1u));
                                oth |= v & 0x80u;
                            }
                            if (t.other_check && oth) continue;  // a byte of no pattern: no match here
                            word = code >> 5;
                            bits = 1u << (code & 31u);
                        }
                        if (MODE == MODE_CHECKED && word >= p.filt_words) {
                            record_error(PM_ERR_BOUNDS);
                            continue;
                        }
                        if ((s_filt[word] & bits) == bits) rootm |= 1u << q;
                    }
                }
                // every position gets -1 now; the walks patch the matches
                if (BATCH && p.out_ids) {
                    // per-text output buffers: each position to its own text's
                    uint32_t c2 = cur0;
                    unsigned long long e2 = __ldg(p.offsets + c2 + 1);
                    for (uint32_t q = 0; q < P && lp0 + q < tile_n; ++q) {
                        const unsigned long long pos = t0 + lp0 + q;
                        while (pos >= e2) {
                            ++c2;
                            e2 = __ldg(p.offsets + c2 + 1);
                        }
                        __stcs(p.out_ids[c2] + (pos - __ldg(p.offsets + c2)), -1);
                    }
                } else if (p.ids_aligned && i * GP + GP <= tile_n) {
                    // every id of the group is -1: the warp writes the
                    // group's 32P ids as P/4 fully coalesced 512-byte rows,
                    // whichever lane owns the positions
#pragma unroll
                    for (int j = 0; j < P / 4; ++j)
                        __stcs(reinterpret_cast<int4 *>(idt + i * GP) + 32 * j + lane,
                               make_int4(-1, -1, -1, -1));
                } else if (p.ids_aligned && lp0 + P <= tile_n) {
#pragma unroll
                    for (int j = 0; j < P / 4; ++j)
                        __stcs(reinterpret_cast<int4 *>(idt + lp0) + j, make_int4(-1, -1, -1, -1));
                } else {
#pragma unroll
                    for (int q = 0; q < P; ++q)
                        if (lp0 + q < tile_n) __stcs(idt + lp0 + q, -1);
                }
                // the group's walks into the warp's queue (ballot/popc
                // compaction), or, when more than the queue holds, walked at
                // once by the lanes that own them
                const uint32_t work = need | rootm;
                if (__any_sync(kFull, work != 0)) {
                    const uint32_t c = __popc(work);
                    uint32_t pre, tot;
                    if (!__any_sync(kFull, c > 1u)) {
                        const uint32_t b1 = __ballot_sync(kFull, c != 0u);
                        pre = __popc(b1 & below);
                        tot = __popc(b1);
                    } else {
                        uint32_t x = c;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, x, o);
                            if (lane >= (uint32_t)o) x += y;
                        }
                        pre = x - c;
                        tot = __shfl_sync(kFull, x, 31);
                    }
                    if (qn + tot > kQueue)
                        while (qn) round(qn < 32u ? qn : 32u);
                    // entry of position lp0 + q: kind and code
                    auto entry = [&](uint32_t q, uint32_t &code) -> unsigned long long {
                        const unsigned long long pos = t0 + lp0 + q;
                        code = 0;
                        if ((rootm >> q) & 1u) return pos;
                        if (IDENT) {
                            code = KF == 1 ? (uint32_t)st[lp0 + q]
                                           : ((uint32_t)st[lp0 + q] << 8) | st[lp0 + q + 1];
                            return pos | ((unsigned long long)WALK_DENSE << 61);
                        }
                        code = (uint32_t)((X << (cb * q)) >> 32) >> shD;
                        return pos | ((unsigned long long)WALK_DEEP << 61);
                    };
                    if (tot > kQueue) {
                        __syncwarp();  // the group's -1 stores (any lane's) first
                        uint32_t wk = work;
                        while (wk) {
                            const uint32_t q = __ffs(wk) - 1;
                            wk &= wk - 1;
                            uint32_t code;
                            const unsigned long long e = entry(q, code);
                            run_walk<BATCH, MODE>(p, e, code, end, pol, acc, look, nwalk);
                        }
                        __syncwarp();
                    } else {
                        uint32_t wk = work, slot = qh + qn + pre;
                        while (wk) {
                            const uint32_t q = __ffs(wk) - 1;
                            wk &= wk - 1;
                            uint32_t code;
                            const unsigned long long e = entry(q, code);
                            const uint32_t idx = slot++ & (kQueue - 1);
                            qpos[idx] = e;
                            qcode[idx] = code;
                        }
                        qn += tot;
                        __syncwarp();
                        while (qn >= 32u) round(32u);
                    }
                }
                cur_c = nxt_c;
                cur_o = nxt_o;
            }

            __syncwarp();  // stage s fully consumed by this warp
            if (lane == 0) fence_proxy_async();
            refill(s);
            if (++s == p.stages) {
                s = 0;
                phase ^= 1u;
            }
        }
        if (!failed)
            while (qn) round(qn < 32u ? qn : 32u);
    }

    // warp reductions: single-text count, lookups and walks
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(kFull, acc, o);
        look += __shfl_xor_sync(kFull, look, o);
        nwalk += __shfl_xor_sync(kFull, nwalk, o);
    }
    if (lane == 0) {
        if (!BATCH && acc) atomicAdd(reinterpret_cast<unsigned long long *>(p.counts), acc);
        if (MODE == MODE_LOOKUPS && look && p.lookups) atomicAdd(p.lookups, look);
        if (p.walks && nwalk) atomicAdd(p.walks, nwalk);
    }
}
#undef PM_WIN

typedef void (*KernelFn)(KParams);

template <int KF, int G, bool IDENT, int P, int CB = 0, int FC = 0, int DC = 0>
KernelFn pick_mode(bool batch, int mode)
{
    if (batch) {
        switch (mode) {
        case MODE_CHECKED: return pfac_scan_kernel<KF, G, IDENT, true, MODE_CHECKED, P, CB, FC, DC>;
        case MODE_LOOKUPS: return pfac_scan_kernel<KF, G, IDENT, true, MODE_LOOKUPS, 4>;
        default: return pfac_scan_kernel<KF, G, IDENT, true, MODE_FAST, P, CB, FC, DC>;
        }
    }
    switch (mode) {
    case MODE_CHECKED: return pfac_scan_kernel<KF, G, IDENT, false, MODE_CHECKED, P, CB, FC, DC>;
    case MODE_LOOKUPS: return pfac_scan_kernel<KF, G, IDENT, false, MODE_LOOKUPS, 4>;
    default: return pfac_scan_kernel<KF, G, IDENT, false, MODE_FAST, P, CB, FC, DC>;
    }
}

template <int P>
KernelFn pick_kernel_p(const TrieDev &t, uint32_t k, uint32_t gram, uint32_t D, bool batch,
                       int mode)
{
    if (t.C == 256) {
        if (k == 0) return pick_mode<0, 0, true, P>(batch, mode);
        if (k == 1) return pick_mode<1, 0, true, P>(batch, mode);
        if (gram == 4) return pick_mode<2, 4, true, P>(batch, mode);
        return pick_mode<2, 3, true, P>(batch, mode);
    }
    // four-letter alphabets (two bits a class) with every pattern at least
    // 13 long, e.g. DNA: the deepest filter and deep level, fixed
    if (t.cb == 2 && k == 10 && D == 13) return pick_mode<-1, 0, false, P, 2, 10, 13>(batch, mode);
    return pick_mode<-1, 0, false, P>(batch, mode);
}

// Byte alphabet (C = 256): k is 0, 1 or 2 and fixed at compile time, and so
// is the Bloom gram length at k = 2. The instrumented lookup-counting kernel
// always takes four positions per lane.
KernelFn pick_kernel(const TrieDev &t, uint32_t k, uint32_t gram, uint32_t D, bool batch,
                     int mode, int positions)
{
    // sixteen positions a lane: the byte alphabet's Bloom level only (the
    // configuration check admits nothing else); a group is then 512
    // positions, which halves the per-position share of the group's fixed
    // work (its -1 rows, queue test and loop) against eight
    if (positions == 16 && mode != MODE_LOOKUPS && t.C == 256 && k == 2)
        return gram == 4 ? pick_mode<2, 4, true, 16>(batch, mode) : pick_mode<2, 3, true, 16>(batch, mode);
    // and the four-letter fixed shapes: 16 two-bit classes and one 32-bit
    // neighbour chunk hold the 28 classes a lane's positions and their
    // 13-grams need
    if (positions == 16 && mode != MODE_LOOKUPS && t.cb == 2 && k == 10 && D == 13)
        return pick_mode<-1, 0, false, 16, 2, 10, 13>(batch, mode);
    if (positions == 8 && mode != MODE_LOOKUPS)
        return pick_kernel_p<8>(t, k, gram, D, batch, mode);
    return pick_kernel_p<4>(t, k, gram, D, batch, mode);
}

// Light form for short single texts: no shared-memory tables, no staging,
// kLightThreads threads a CTA, four positions per thread. A thread loads its
// bytes, then the filter words of its four positions (global memory,
// L2-resident) all at once, writes -1, and walks at once where the filter
// cannot rule a position out: the same filters, start nodes and walks as
// the persistent kernel, so the same bits. A text that one CTA covers gets
// its count written by that CTA (no separate zeroing of the count);
// launching it costs a few microseconds where the persistent kernel loads
// up to 128 KiB of tables into every CTA first.
constexpr uint32_t kLightThreads = 512;
constexpr uint32_t kLightP = 4;

template <int KF, int G, bool IDENT, int MODE>
__global__ void __launch_bounds__(kLightThreads) pfac_light_kernel(const KParams p)
{
    constexpr int P = (int)kLightP;
    __shared__ unsigned long long s_red[kLightThreads / 32];
    const TrieDev &t = p.t;
    const uint64_t pol = policy_evict_last();
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long acc = 0, look = 0, nwalk = 0;
    const unsigned long long i0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * P;
    constexpr uint32_t KFU = KF > 0 ? (uint32_t)KF : 0u;
    const uint32_t cb = p.cb;
    if (i0 < p.total) {
        const uint8_t *tp = p.text + i0;
        const unsigned long long left0 = p.limit - i0;  // readable bytes from i0
        unsigned long long e[P];
        uint32_t code[P];
        uint32_t walk = 0;  // bit q: position i0+q is walked
#pragma unroll
        for (int q = 0; q < P; ++q) {
            e[q] = i0 + q;
            code[q] = 0;
        }
        if (IDENT && MODE != MODE_LOOKUPS) {
            // bytes i0 .. i0 + P + 2 (those inside the readable text)
            uint32_t b[P + 3];
#pragma unroll
            for (int j = 0; j < P + 3; ++j) b[j] = (unsigned long long)j < left0 ? __ldg(tp + j) : 0u;
            uint32_t word[P], bits[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const uint32_t x = b[q] | (b[q + 1] << 8) | (b[q + 2] << 16) | (b[q + 3] << 24);
                if (KF >= (int)kBloomK) {
                    const BloomProbe pr = bloom_probe(x, p.gram, 8u * KFU + p.lw - 5u);
                    word[q] = pr.word;
                    bits[q] = pr.mask;
                } else {
                    const uint32_t idx = x & (uint32_t)((1ull << (8 * KFU + p.lw)) - 1ull);
                    word[q] = idx >> 5;
                    bits[q] = 1u << (idx & 31u);
                }
                if (MODE == MODE_CHECKED && word[q] >= p.filt_words) {
                    record_error(PM_ERR_BOUNDS);
                    word[q] = 0;
                    bits[q] = 0;
                }
                if (KF >= 1) code[q] = KF == 1 ? b[q] : (b[q] << 8) | b[q + 1];
            }
            uint32_t fw[P];
#pragma unroll
            for (int q = 0; q < P; ++q) fw[q] = ld_trie_u32(p.filter + word[q], pol);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                if (i0 + q >= p.total) break;
                if ((unsigned long long)q + p.gram > left0) {
                    walk |= 1u << q;  // too close to the end to test: from the root
                } else if ((fw[q] & bits[q]) == bits[q]) {
                    walk |= 1u << q;
                    if (KF >= 1) e[q] |= (unsigned long long)WALK_DENSE << 61;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                if (i0 + q >= p.total) break;
                const unsigned long long left = left0 - q;
                if (MODE == MODE_LOOKUPS || p.F == 0 || p.gram > left) {
                    walk |= 1u << q;
                    continue;
                }
                const uint8_t *pq = tp + q;
                uint32_t c = 0, oth = 0;
                for (uint32_t j = 0; j < p.F; ++j) {
                    const uint32_t v = __ldg(t.cls + __ldg(pq + j));
                    c = (c << cb) | (v & ((1u << cb) - 1u));
                    oth |= v & 0x80u;
                }
                if (t.other_check && oth) continue;  // a byte of no pattern: no match
                if (MODE == MODE_CHECKED && (c >> 5) >= p.filt_words) {
                    record_error(PM_ERR_BOUNDS);
                    continue;
                }
                if (!((ld_trie_u32(p.filter + (c >> 5), pol) >> (c & 31u)) & 1u)) continue;
                walk |= 1u << q;
                if (p.D > 0 && p.D <= left) {
                    for (uint32_t j = p.F; j < p.D; ++j) {
                        const uint32_t v = __ldg(t.cls + __ldg(pq + j));
                        c = (c << cb) | (v & ((1u << cb) - 1u));
                        oth |= v & 0x80u;
                    }
                    if (t.other_check && oth) {
                        walk &= ~(1u << q);
                        continue;
                    }
                    code[q] = c;
                    e[q] |= (unsigned long long)WALK_DEEP << 61;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q)
            if (i0 + q < p.total) __stcs(p.ids + i0 + q, -1);
#pragma unroll
        for (int q = 0; q < P; ++q)
            if ((walk >> q) & 1u) run_walk<false, MODE>(p, e[q], code[q], p.limit, pol, acc, look, nwalk);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(kFull, acc, o);
        look += __shfl_xor_sync(kFull, look, o);
        nwalk += __shfl_xor_sync(kFull, nwalk, o);
    }
    if (gridDim.x == 1) {
        // one CTA: it writes the count (and adds the lookups and walks) itself
        if (lane == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) tot += s_red[w];
            if (p.light_add) *p.counts += (int64_t)tot;
            else *p.counts = (int64_t)tot;
        }
        acc = 0;
    }
    if (lane == 0) {
        if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(p.counts), acc);
        if (MODE == MODE_LOOKUPS && look && p.lookups) atomicAdd(p.lookups, look);
        if (p.walks && nwalk) atomicAdd(p.walks, nwalk);
    }
}

template <int KF, int G, bool IDENT>
KernelFn pick_light_mode(int mode)
{
    switch (mode) {
    case MODE_CHECKED: return pfac_light_kernel<KF, G, IDENT, MODE_CHECKED>;
    case MODE_LOOKUPS: return pfac_light_kernel<KF, G, IDENT, MODE_LOOKUPS>;
    default: return pfac_light_kernel<KF, G, IDENT, MODE_FAST>;
    }
}

KernelFn pick_light(const TrieDev &t, uint32_t k, uint32_t gram, int mode)
{
    if (t.C == 256) {
        if (k == 0) return pick_light_mode<0, 0, true>(mode);
        if (k == 1) return pick_light_mode<1, 0, true>(mode);
        if (gram == 4) return pick_light_mode<2, 4, true>(mode);
        return pick_light_mode<2, 3, true>(mode);
    }
    return pick_light_mode<-1, 0, false>(mode);
}

// Per-text count finalisation: counts[t] to the caller's *out[t].
__global__ void pm_counts_scatter_kernel(const int64_t *counts, int64_t *const *out, uint32_t n)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) *out[t] = counts[t];
}

uint32_t round16(uint64_t x) { return (uint32_t)((x + 15) & ~15ull); }

int width_index(int32_t bits) { return bits == 8 ? 0 : bits == 16 ? 1 : 2; }

}  // namespace

// Shared memory: [filter][class table] shared by the CTA, then one block per
// warp: [mbarriers][walk queue][stages x (tile + halo + pad)].
ScanLayout scan_layout(const TrieDev &t, const pm_config &cfg)
{
    ScanLayout L{};
    const uint32_t k = (uint32_t)cfg.dense_k;
    const bool ident = t.C == 256;
    L.filt_words = ident ? t.filter_words[k][width_index(cfg.filter_bits)]
                         : (k > 0 ? t.filter_words[k][0] : 0u);
    L.filt_u4 = L.filt_words / 4;
    uint32_t off = round16((uint64_t)L.filt_words * 4);
    L.off_lut = off;
    if (!ident) off += 64 * 32 * 4;
    L.off_warp = off;
    L.halo = round16(t.max_len > 16 ? t.max_len : 16);
    L.stage_bytes = (uint32_t)cfg.tile + L.halo + kStagePad;
    L.off_queue = kWarpHeader;
    L.off_stages = kWarpHeader + kQueue * 12;
    L.warp_bytes = L.off_stages + (uint32_t)cfg.stages * L.stage_bytes;
    L.off_sched = off + (uint32_t)(cfg.threads / 32) * L.warp_bytes;
    L.total = L.off_sched + 8 * kChunkRing + 16;
    // byte classes: neighbour chunks a lane's window needs
    uint32_t dmax = k;
    if (!ident && cfg.deep && t.deep_k > dmax) dmax = t.deep_k;
    const uint32_t P = (uint32_t)cfg.positions;
    L.nnb = dmax > 1 ? (dmax - 1 + P - 1) / P : 0;
    return L;
}

namespace {

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

// Stream-ordered pool per device for the dynamic schedule's run counters
// (4 bytes a launch); freed blocks stay in the pool for the next launch.
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;  // guarded by g_pool_mu

bool run_pool(int dev, cudaMemPool_t &pool)
{
    std::lock_guard<std::mutex> g(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        pool = it->second;
        return true;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools.emplace(dev, pool);
    return true;
}

// A zeroed run counter for one launch on st, or null (static schedule):
// never while st is being captured into a graph.
unsigned int *run_counter(int dev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemPool_t pool;
    if (cs != cudaStreamCaptureStatusNone || !run_pool(dev, pool)) return nullptr;
    void *ctr = nullptr;
    if (cudaMallocFromPoolAsync(&ctr, sizeof(unsigned int), pool, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned int), st) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(ctr, st);
        return nullptr;
    }
    return static_cast<unsigned int *>(ctr);
}

}  // namespace

uint64_t scan_smem_bytes(const TrieDev &t, const pm_config &cfg)
{
    return scan_layout(t, cfg).total;
}

int launch_scan(const TrieDev &t, const pm_config &cfg, const ScanArgs &a, void *stream,
                int device_sms, std::string &msg)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool batch = a.offsets != nullptr;
    const uint32_t ncount = batch ? a.ntexts : 1;
    // the light form on a text one CTA covers writes its count itself
    const bool light1 = !batch && cfg.light_max > 0 && a.len > 0 &&
                        a.len <= (uint64_t)cfg.light_max &&
                        a.len <= (uint64_t)kLightThreads * kLightP && !a.lookups;
    if (ncount && !a.keep_counts && !light1) {
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
    pm_config c = cfg;
    if (mode == MODE_LOOKUPS) c.positions = 4;
    const bool ident = t.C == 256;
    const uint32_t deep_d = !ident && c.deep && t.deep_k > 0 ? t.deep_k : 0u;
    KernelFn fn = pick_kernel(t, (uint32_t)c.dense_k, ident ? t.gram[c.dense_k] : 0u, deep_d,
                              batch, mode, c.positions);
    const ScanLayout L = scan_layout(t, c);

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
    p.match_bits = batch ? nullptr : a.match_bits;
    p.walks = a.walks;
    p.tile = (uint32_t)c.tile;
    p.halo = L.halo;
    p.k = (uint32_t)c.dense_k;
    p.lw = c.filter_bits == 8 ? 3u : c.filter_bits == 16 ? 4u : 5u;
    if (ident) {
        p.filter = t.filter[c.dense_k][width_index(c.filter_bits)];
        p.dense = c.dense_k > 0 ? t.dense[c.dense_k] : nullptr;
        p.first_k = t.first[c.dense_k];
        p.gram = t.gram[c.dense_k];
    } else {
        p.filter = c.dense_k > 0 ? t.filter[c.dense_k][0] : nullptr;
        p.cb = t.cb;
        p.F = (uint32_t)c.dense_k;
        p.D = c.deep && t.deep_k > 0 ? t.deep_k : 0u;
        p.gram = p.F;
        p.nnb = L.nnb;
    }
    p.binary = c.row_search ? 1u : 0u;
    p.bitmap = c.layout == 1 ? 1u : 0u;
    p.stages = (uint32_t)c.stages;
    p.aligned = ((uintptr_t)a.text & 15u) == 0;
    p.ids_aligned = ((uintptr_t)a.ids & 15u) == 0;
    p.wait_budget = c.wait_clocks > 0 ? (long long)c.wait_clocks : kWaitBudget;
    p.off_lut = L.off_lut;
    p.off_warp = L.off_warp;
    p.warp_bytes = L.warp_bytes;
    p.off_queue = L.off_queue;
    p.off_stages = L.off_stages;
    p.off_sched = L.off_sched;
    p.stage_bytes = L.stage_bytes;
    p.filt_u4 = L.filt_u4;
    p.filt_words = L.filt_words;

    cudaError_t e;
    if (!batch && c.light_max > 0 && a.len <= (uint64_t)c.light_max) {
        const uint32_t threads = kLightThreads;
        const unsigned long long per = (unsigned long long)kLightP * threads;
        const unsigned long long grid = light1 ? 1ull : (a.len + per - 1) / per;
        p.light_add = a.keep_counts ? 1u : 0u;
        KernelFn lf = pick_light(t, (uint32_t)c.dense_k, ident ? t.gram[c.dense_k] : 0u, mode);
        lf<<<(unsigned)grid, threads, 0, st>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            msg = std::string("light scan launch: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
        return PM_OK;
    }
    int occ = 0;
    int dev = -1;
    {
        // the shared-memory attribute and the occupancy of each (kernel,
        // shared bytes, threads, device) are set and queried once
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) {
            msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
        const LaunchKey key{reinterpret_cast<const void *>(fn), L.total, (uint32_t)c.threads, dev};
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
                &occ, reinterpret_cast<const void *>(fn), c.threads, L.total);
            if (e != cudaSuccess || occ < 1) {
                msg = "configuration does not fit on an SM (threads " +
                      std::to_string(c.threads) + ", shared " + std::to_string(L.total) + ")";
                return PM_ERR_INVAL;
            }
            g_occ.emplace(key, occ);
        }
    }
    if (c.ctas_per_sm > 0 && c.ctas_per_sm < occ) occ = c.ctas_per_sm;
    unsigned long long grid = (unsigned long long)device_sms * occ;
    const unsigned long long known = batch ? a.total_hint : a.len;
    if (known) {
        const unsigned long long warps = c.threads / 32;
        const unsigned long long ntiles = (known + c.tile - 1) / c.tile;
        const unsigned long long need = (ntiles + warps - 1) / warps;
        if (need < grid) grid = need;
    }
    // the dynamic schedule's run counter (none: the static schedule)
    p.chunk_ctr = c.schedule == PM_SCHED_DYNAMIC ? run_counter(dev, st) : nullptr;
    fn<<<(unsigned)grid, c.threads, L.total, st>>>(p);
    e = cudaGetLastError();
    if (p.chunk_ctr) cudaFreeAsync(p.chunk_ctr, st);
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
