// Internal types shared by the libpm translation units (host builder, CUDA
// scan, C ABI). Not installed; the public interface is include/pm.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "pm.h"

namespace pm {

// Deepest dense prefix table (trie levels resolved by one table lookup).
constexpr int kMaxDenseK = 12;
// Shared-memory budget of one dense table (bitmap + rank words).
constexpr uint64_t kDenseBudget = 144u * 1024u;
// Shared-memory budget of one child-filter table (u32 per depth-k node).
constexpr uint64_t kChildMaskBudget = 96u * 1024u;

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
// Dense prefix table of level k: the first k trie levels expanded over the
// byte classes. A k-gram of classes (c_0..c_{k-1}) has code
// sum_j c_j * C^(k-1-j); bit `code` of the table is set iff the k-gram spells
// a root path, and then the depth-k node it reaches is
//   first[k] + rank(code) = first[k] + base(word) + popc(word & lower bits),
// because BFS numbers the depth-k nodes contiguously in code order. The table
// is stored as uint2 {bits, base} per 32 codes.
struct TrieDev {
    const uint32_t *row_ptr;
    const uint8_t *col;
    const int32_t *next;
    const int2 *emit;
    const uint8_t *cls;                    // byte -> class, 256 entries
    const uint2 *dense[kMaxDenseK + 1];    // index k (0 unused)
    const uint32_t *childmask[kMaxDenseK + 1];
    uint32_t dense_words[kMaxDenseK + 1];  // uint2 entries of table k
    uint32_t first[kMaxDenseK + 1];        // BFS id of the first depth-k node
    uint32_t nlevel[kMaxDenseK + 1];       // number of depth-k nodes
    uint32_t C;                            // classes
    uint32_t n_nodes;
    uint32_t nnz;
    uint32_t min_len;                      // shortest pattern (>= 1)
    uint32_t max_len;
    uint32_t dense_k_max;
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
    uint32_t C = 0;
    uint32_t min_len = 0, max_len = 0;
    uint64_t n_patterns = 0, n_duplicates = 0;
    uint32_t dense_k_max = 0;
    std::vector<uint32_t> dense[kMaxDenseK + 1];     // interleaved {bits, base}
    std::vector<uint32_t> childmask[kMaxDenseK + 1];
    uint32_t first[kMaxDenseK + 1] = {};
    uint32_t nlevel[kMaxDenseK + 1] = {};
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
};

// Enqueues the scan (counts zeroed first). Returns PM_OK / PM_ERR_CUDA.
int launch_scan(const TrieDev &t, const pm_config &cfg, const ScanArgs &a,
                void *stream, int device_sms, std::string &msg);

// Dynamic shared memory the scan needs for a configuration.
uint64_t scan_smem_bytes(const TrieDev &t, const pm_config &cfg);

// Reads and clears the device error word.
int read_device_error(int *code, std::string &msg);

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
};
