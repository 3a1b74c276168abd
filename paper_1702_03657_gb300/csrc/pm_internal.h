// Internal types shared by the libpm translation units (host builder, CUDA
// scan, C ABI). Not installed; the public interface is include/pm.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <vector_types.h>

#include "pm.h"

namespace pm {

// Deepest filter level: the byte alphabet's levels k (k <= 2), or the
// filter depth F of a byte-class trie (F * bits per class <= 20).
constexpr int kMaxDenseK = 20;
// Shared-memory budget of one filter table.
constexpr uint64_t kFilterBudget = 128u * 1024u;
// Byte classes: bits of a packed filter code (2^20 bits = 128 KiB) and of a
// deep-level code (2^26 codes, a 16 MiB bitmap with ranks read from L2).
constexpr uint32_t kFilterCodeBits = 20;
constexpr uint32_t kDeepCodeBits = 26;
// All-matches: positions per tile of the match-count table.
constexpr uint32_t kMatchTileShift = 10;
// Filter widths: W = 8, 16, 32 bits per k-gram (index 0, 1, 2).
constexpr int kFilterWidths = 3;

// Device view of a built trie; passed by value to the scan kernels.
//
// CRS (Section III): row v's edges are row_ptr[v] .. row_ptr[v+1]-1, each with
// its byte col[e] (ascending) and child next[e]. Nodes are numbered in BFS
// order with children in ascending byte order.
//
// emit[v] = {best, nfinal}: best is the id of the deepest pattern ending on
// the root path of v (v included), -1 if none; nfinal the number of patterns
// ending on that path. A walk that stops at v has found exactly the nfinal
// patterns on its path and its longest match is best.
//
// Byte classes: the bytes used by some pattern, in ascending byte order, then
// one class for every other byte (none when all 256 are used: class = byte).
//
// Byte alphabet (C = 256). Dense table of level k (global memory): bit
// `code` (the k-gram, first byte most significant) is set iff the k-gram
// spells a root path, and then the depth-k node it reaches is
//   first[k] + base(word) + popc(word & lower bits),
// because BFS numbers the depth-k nodes contiguously in code order. Stored
// as uint2 {bits, base} per 32 codes.
//
// With k >= kBloomK the shared-memory filter is a blocked Bloom filter over
// 2^(8k + log2 W) bits of the root paths of length g (g = k+2 when every
// pattern is longer than k+1, else k+1), each read as the little-endian
// integer x = sum_j b_j << 8j. One multiplicative hash
// h = hi32((x << (32 - 8g)) * M) picks a 32-bit word (its top bits) and two
// bits in it (h mod 32 and (h >> 5) mod 32); both are set for every such
// path. A clear bit proves that the g-gram is not a root path, so the walk
// stops at depth <= g-1 < shortest pattern. The depth-k node of a passing
// position is then looked up in the dense table, which also tells whether
// the k-gram itself is a path.
//
// Byte-class tries (C < 256). The U used classes take cb = ceil(log2 U)
// bits each (at least 1); a d-gram's packed code is its classes
// concatenated, the first one in the most significant bits, so packed codes
// sort like the paths and BFS numbers the depth-d nodes in code order. A byte
// of the "other" class gets the code U when U < 2^cb (no path contains it),
// else a separate flag (other_check). Tables:
//  - filter of depth F (shared memory): bit `code` set iff the F-gram spells
//    a root path; F <= shortest pattern, so a clear bit proves that nothing
//    matches at that position;
//  - deep level of depth D (global memory, read through L2): the root paths
//    of depth D as uint2 {bits, base} per 32 packed codes; D <= shortest
//    pattern, so a D-gram that is not a path rules the position out, and
//    otherwise the walk starts at node deep_first + base + popc(...).
constexpr uint32_t kBloomK = 2;
constexpr uint32_t kBloomMul = 0x9E3779B1u;  // Knuth's golden-ratio multiplier
struct BloomProbe {
    uint32_t word, mask;
};
__host__ __device__ inline uint32_t bloom_mask(uint32_t h)
{
    return (1u << (h & 31u)) | (1u << ((h >> 5) & 31u));
}
__host__ __device__ inline BloomProbe bloom_probe(uint32_t x, uint32_t gram, uint32_t word_bits)
{
    const uint32_t h = (uint32_t)(((uint64_t)(x << (32u - 8u * gram)) * kBloomMul) >> 32);
    return {h >> (32u - word_bits), bloom_mask(h)};
}

// Filter of level k and width W (byte alphabet, k < kBloomK; shared
// memory): a bitset of 256^k * W bits. For a k-gram spelling a root path and
// a next byte c_k, the bit ((c_k mod W) << 8k) | sum_j b_j << 8j (the path
// read little-endian) is set iff the depth-k node has a child of some byte
// congruent to c_k mod W; bits of k-grams that are not root paths are clear.
// It is exact when W >= 256. With k < shortest pattern, a clear bit proves
// that the walk from this start position stops at depth <= k without a
// match.
//
// Device form of the CRS matrix. BFS numbering makes the next state of
// non-zero e equal to e + 1, so the value array is implicit, and each row is
// described by one 16-byte record read in a single load per walk step:
//   x: index of the row's first non-zero (row_ptr[v])
//   y: row length (bits 0..8) | 1 << 31 when a pattern ends on v's path
//   z, w: the row's first eight column bytes, ascending (zero padded)
// col holds every row's bytes for rows longer than eight.
constexpr uint32_t kNoSwar = 0xFFu;  // no 3-bit field tells the four letters apart

struct TrieDev {
    const uint4 *row;
    const uint8_t *col;
    const int2 *emit;
    const uint8_t *cls;                                   // byte -> class
    const uint2 *dense[kMaxDenseK + 1];                   // index k (0 unused)
    const uint32_t *filter[kMaxDenseK + 1][kFilterWidths];
    uint32_t filter_words[kMaxDenseK + 1][kFilterWidths]; // u32 words
    uint32_t dense_words[kMaxDenseK + 1];                 // uint2 entries of table k
    uint32_t first[kMaxDenseK + 1];                       // BFS id of the first depth-k node
    uint32_t nlevel[kMaxDenseK + 1];                      // number of depth-k nodes
    uint32_t gram[kMaxDenseK + 1];                        // bytes a level-k filter tests
    uint32_t C;                                           // classes
    uint32_t n_nodes;
    uint32_t nnz;
    uint32_t min_len;                                     // shortest pattern (>= 1)
    uint32_t max_len;
    uint32_t dense_k_max;                                 // deepest filter level
    uint32_t cb;                                          // byte classes: bits per class
    uint32_t other_check;                                 // byte classes: U == 2^cb
    // byte classes, four letters: the class of a byte read from an 8-entry
    // byte table by a 3-bit field of the byte (see HostTrie)
    uint32_t sw_shift;                                    // field (b >> sw_shift) & 7, or kNoSwar
    uint32_t sw_cls[2];                                   // field -> class
    uint32_t sw_sym[2];                                   // field -> the letter with that field
    const uint2 *deep;                                    // deep level {bits, base} (or null)
    uint32_t deep_k;                                      // its depth D (0: none)
    uint32_t deep_first;                                  // BFS id of the first depth-D node
    uint32_t deep_words;                                  // uint2 entries
    const int4 *minfo;                                    // per pattern id (all-matches)
    // Unary chains (see HostTrie): labels and, per chain position, the emit
    // {best, nfinal} of the node there, or {end node, 0} at a chain's end
    const uint8_t *ch_lab;
    const int2 *ch_info;
    uint32_t ch_len;                                      // chain positions
    // Bitmapped nodes (Section III, Fig. 3): node v's children as a 256-bit
    // bitmap over bytes (two uint4 at bm[2v]) and the id of its first child;
    // the child on byte b is first + (set bits below b)
    const uint4 *bm;
    const uint32_t *bm_first;
    uint32_t n_ids;                                       // pattern id space (input count)
};

// Host-side trie: the CRS arrays plus the derived tables.
struct HostTrie {
    std::vector<uint32_t> row_ptr;
    std::vector<uint8_t> col;
    std::vector<int32_t> next;
    std::vector<int32_t> final_id;
    std::vector<int32_t> best;
    std::vector<int32_t> nfinal;
    std::vector<uint32_t> depth;
    uint8_t cls[256];
    // byte classes: per byte its packed class; a byte of the "other" class
    // gets U, or 0x80 (flag, class bits 0) with other_check
    uint8_t lut[256];
    uint32_t cb = 0, other_check = 0;
    // four letters (U == 4): a shift s such that (b >> s) & 7 differs for
    // the four letters, and two 8-byte tables over that field: the letter's
    // class, and the letter itself (a field no letter has holds a byte whose
    // field differs, so that no byte matches it). A byte is a letter iff it
    // equals the table's letter at its field. kNoSwar: no such shift.
    uint32_t sw_shift = kNoSwar;
    uint8_t sw_cls[8] = {}, sw_sym[8] = {};
    uint32_t C = 0;
    uint32_t min_len = 0, max_len = 0;
    uint64_t n_patterns = 0, n_duplicates = 0;
    uint32_t dense_k_max = 0;
    uint32_t deep_k = 0, deep_first = 0;
    std::vector<uint32_t> deep;  // interleaved {bits, base} over 2^(cb * deep_k) codes
    // all-matches: per input pattern id (distinct patterns only, others -1/0):
    // the next shorter pattern on its root path, its length, and the number
    // of patterns on its root path (itself included)
    std::vector<int32_t> chain, plen, mcnt;
    std::vector<uint32_t> dense[kMaxDenseK + 1];     // interleaved {bits, base}
    // byte alphabet: filter of level k and width index w; byte classes: the
    // packed filter of depth F in filter[F][0]
    std::vector<uint32_t> filter[kMaxDenseK + 1][kFilterWidths];
    uint32_t first[kMaxDenseK + 1] = {};
    uint32_t nlevel[kMaxDenseK + 1] = {};
    std::vector<uint32_t> level_nodes;  // nodes per depth, every depth
    // Unary chains: each maximal run u_0 -> u_1 -> ... -> u_L of nodes with
    // exactly one child (u_0's parent has another number of children, u_L
    // has none or several) is stored at positions o .. o+L: ch_lab[o+j] is
    // the byte of the edge u_j -> u_{j+1}; ch_info[o+j] = {best, nfinal} of
    // u_j for j < L, and {u_L, 0} at o+L. A one-child node u_j has
    // ch_pos = o+j and ch_rem = L-j (edges forced from it); other nodes have
    // ch_rem = 0. ch_lab is padded with 32 zero bytes.
    std::vector<uint8_t> ch_lab;
    std::vector<int32_t> ch_info;       // interleaved pairs
    std::vector<uint32_t> ch_pos, ch_rem;
    uint32_t gram[kMaxDenseK + 1] = {};  // bytes a level-k filter tests: k+1 or k+2
};

// Builds the host trie. Returns PM_OK or an error code (msg filled).
int build_host_trie(const uint8_t *const *patterns, const uint32_t *lengths,
                    uint32_t n, HostTrie &t, std::string &msg);

// Launch parameters resolved from a pm_config for one scan.
struct ScanArgs {
    const uint8_t *text;
    const uint64_t *offsets;  // nullptr: one text of `len` bytes
    uint32_t ntexts;
    uint64_t len;             // start positions when offsets == nullptr
    uint64_t limit;           // readable bytes (>= len) of the single text;
                              // walks may read up to here (chunk overlap)
    int32_t *ids;
    int64_t *counts;
    unsigned long long *lookups;  // optional
    // batch only, optional: per-text output buffers (device arrays of device
    // pointers); ids of text t go to out_ids[t][0 .. len_t), and counts[t]
    // (still required, internal) is copied to *out_counts[t] at the end
    int32_t *const *out_ids;
    int64_t *const *out_counts;
    // batch only, optional: total text bytes when the host knows it (sizes
    // the persistent grid to the work; 0: one CTA per SM)
    uint64_t total_hint;
    // single text only, optional: matches per tile of 2^kMatchTileShift
    // start positions, added to (zeroed by the caller)
    uint32_t *tile_counts;
    // with tile_counts: one bit per start position, set where a pattern
    // occurs (zeroed by the caller)
    uint32_t *match_bits;
    // add to the counts instead of overwriting them
    bool keep_counts;
    // optional: number of walks queued (positions the filter, dense and deep
    // levels could not settle), added to
    unsigned long long *walks;
};

// All-matches listing after a single-text scan with tile_counts and
// match_bits (same stream): lists every occurrence into out[0 .. capacity)
// in position order, longest pattern first, positions offset by pos_base.
// work (match_work_bytes(len) bytes): the tile counts and the match bits
// (both zeroed before the scan, zero_bytes from the start), then the block
// sums and offsets.
struct MatchWork {
    uint64_t bits;        // byte offset of the match bits
    uint64_t bsum, boff;  // byte offsets of the block sums and offsets
    uint64_t zero_bytes;  // bytes to zero before the scan
    uint64_t total;
};
MatchWork match_work_layout(uint64_t len);
uint64_t match_work_bytes(uint64_t len);
int launch_matches(const TrieDev &t, const int32_t *ids, uint64_t len, void *work,
                   pm_match *out, uint64_t capacity, void *stream, std::string &msg,
                   uint64_t pos_base = 0);

// Enqueues the scan (counts zeroed first). Returns PM_OK / PM_ERR_CUDA.
int launch_scan(const TrieDev &t, const pm_config &cfg, const ScanArgs &a,
                void *stream, int device_sms, std::string &msg);

// Shared-memory layout of the scan kernel for a configuration (byte
// offsets), and the neighbour chunks a lane's window takes (byte classes).
struct ScanLayout {
    uint32_t off_lut, off_warp, warp_bytes, off_queue, off_stages, stage_bytes, total;
    uint32_t off_sched;  // dynamic schedule: the CTA's ticket counter and run ring
    uint32_t filt_u4, filt_words, halo, nnb;
};
ScanLayout scan_layout(const TrieDev &t, const pm_config &cfg);

// Dynamic shared memory the scan needs for a configuration.
uint64_t scan_smem_bytes(const TrieDev &t, const pm_config &cfg);

// Stream push preparation: dst = carry[0 .. nc) || chunk[0 .. len); bytes
// [keep_from, keep_from + nkeep) of dst also to carry_out (which must not
// overlap carry); *count = 0. Asynchronous on `stream`.
int launch_gather(const uint8_t *carry, uint64_t nc, const uint8_t *chunk, uint64_t len,
                  uint8_t *dst, uint8_t *carry_out, uint64_t keep_from, uint64_t nkeep,
                  int64_t *count, void *stream, std::string &msg);

// Reads and clears the device error word.
int read_device_error(int *code, std::string &msg);

// Records `code` and `msg` as this thread's last error and returns `code`.
int set_last_error(int code, const std::string &msg);

}  // namespace pm

// Opaque handle (C ABI type).
struct pm_trie {
    pm::HostTrie host;
    pm::TrieDev dev{};
    void *d_arena = nullptr;
    uint64_t device_bytes = 0;
    int device = -1;
    int sms = 0;
    pm_config cfg{};
    // pm_scan_host staging (allocated on first use)
    void *h_streams[2] = {nullptr, nullptr};
    uint8_t *d_hbuf_text = nullptr;
    int32_t *d_hbuf_ids = nullptr;
    int64_t *d_hbuf_counts = nullptr;
    int64_t *h_hbuf_counts = nullptr;  // pinned
    uint64_t hbuf_chunk = 0;
    // pm_scan_all_host: per slot, the listing workspace and the match list
    void *d_hbuf_work = nullptr;
    pm_match *d_hbuf_match = nullptr;
    uint64_t hbuf_work_bytes = 0, hbuf_mcap = 0;
};
