// Host-side trie construction and CRS compression (Section III).
//
// Steps, in the paper's order where they apply to an exact scan:
//  I   breadth-first, level-by-level construction;
//  II  pointer-free storage in BFS (row-major) order, children of a node in
//      ascending byte order;
//  VI  the node x byte sparse matrix of next states;
//  CRS that matrix compressed row by row: row_ptr (n+1), col (the byte of
//      each non-zero, ascending in a row), next (the child node).
// Truncation and suffix/end-node merging (steps III-V) change the result
// (prefix matches, shared end nodes without pattern ids) and are not used.
//
// Construction works on the lexicographically sorted, deduplicated pattern
// list: the patterns below a node at depth d form a contiguous range of that
// list, and its children are the runs of equal byte d inside the range, in
// ascending byte order. Processing nodes in creation order (a FIFO) therefore
// numbers them breadth-first, and the depth-d nodes come out sorted by their
// path, which the dense prefix tables rely on.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "pm_internal.h"

namespace pm {

namespace {

struct PatView {
    const uint8_t *p;
    uint32_t len;
};

bool less_str(const PatView &a, const PatView &b)
{
    uint32_t m = std::min(a.len, b.len);
    int r = m ? std::memcmp(a.p, b.p, m) : 0;
    if (r != 0) return r < 0;
    return a.len < b.len;
}

bool equal_str(const PatView &a, const PatView &b)
{
    return a.len == b.len && (a.len == 0 || std::memcmp(a.p, b.p, a.len) == 0);
}

// C^k, or 0 when it exceeds `cap`.
uint64_t ipow_capped(uint64_t C, int k, uint64_t cap)
{
    uint64_t r = 1;
    for (int i = 0; i < k; ++i) {
        if (r > cap / C) return 0;
        r *= C;
    }
    return r;
}

}  // namespace

int build_host_trie(const uint8_t *const *patterns, const uint32_t *lengths,
                    uint32_t n, HostTrie &t, std::string &msg)
{
    if (n > 0 && (!patterns || !lengths)) {
        msg = "patterns or lengths is NULL";
        return PM_ERR_INVAL;
    }
    uint64_t total_len = 0;
    for (uint32_t j = 0; j < n; ++j) {
        if (lengths[j] == 0) {
            msg = "pattern " + std::to_string(j) + " is empty";
            return PM_ERR_EMPTY_PATTERN;
        }
        if (lengths[j] > PM_MAX_PATTERN_LEN) {
            msg = "pattern " + std::to_string(j) + " is longer than PM_MAX_PATTERN_LEN";
            return PM_ERR_PATTERN_TOO_LONG;
        }
        if (!patterns[j]) {
            msg = "pattern " + std::to_string(j) + " is NULL";
            return PM_ERR_INVAL;
        }
        total_len += lengths[j];
    }
    if (total_len + 1 >= (1ull << 31)) {
        msg = "total pattern length exceeds 2^31 - 2 trie nodes";
        return PM_ERR_NOMEM;
    }

    // Sort by (string, input index) and keep the first of each equal run: a
    // pattern's id is the index of its first occurrence in the input.
    std::vector<uint32_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0u);
    auto view = [&](uint32_t j) { return PatView{patterns[j], lengths[j]}; };
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
        PatView va = view(a), vb = view(b);
        if (less_str(va, vb)) return true;
        if (less_str(vb, va)) return false;
        return a < b;
    });
    std::vector<uint32_t> uq;
    uq.reserve(n);
    for (uint32_t k = 0; k < n; ++k) {
        if (!uq.empty() && equal_str(view(uq.back()), view(ord[k]))) {
            ++t.n_duplicates;
            continue;
        }
        uq.push_back(ord[k]);
    }
    const uint32_t m = (uint32_t)uq.size();
    t.n_patterns = m;
    t.min_len = 0;
    t.max_len = 0;
    for (uint32_t k = 0; k < m; ++k) {
        uint32_t L = lengths[uq[k]];
        t.max_len = std::max(t.max_len, L);
        t.min_len = k ? std::min(t.min_len, L) : L;
    }

    // Byte classes: the bytes used by some pattern in ascending order, then
    // one class for every other byte (no trie edge carries it). With all 256
    // bytes in use the classes are the bytes themselves.
    bool used[256] = {};
    for (uint32_t k = 0; k < m; ++k) {
        const uint8_t *p = patterns[uq[k]];
        for (uint32_t d = 0; d < lengths[uq[k]]; ++d) used[p[d]] = true;
    }
    uint32_t u = 0;
    for (int b = 0; b < 256; ++b)
        if (used[b]) t.cls[b] = (uint8_t)u++;
    if (u == 256) {
        t.C = 256;
    } else {
        for (int b = 0; b < 256; ++b)
            if (!used[b]) t.cls[b] = (uint8_t)u;
        t.C = u + 1;
    }

    // Steps I, II, VI and CRS: BFS over pattern ranges.
    struct Range { uint32_t lo, hi; };
    std::vector<Range> rng;
    rng.reserve(total_len + 1);
    t.row_ptr.clear();
    t.col.clear();
    t.next.clear();
    t.final_id.clear();
    t.best.clear();
    t.nfinal.clear();
    t.depth.clear();
    rng.push_back({0, m});
    t.chain.assign(n, -1);
    t.plen.assign(n, 0);
    t.mcnt.assign(n, 0);
    t.final_id.push_back(-1);
    t.best.push_back(-1);
    t.nfinal.push_back(0);
    t.depth.push_back(0);
    t.row_ptr.push_back(0);
    for (size_t v = 0; v < rng.size(); ++v) {
        uint32_t lo = rng[v].lo, hi = rng[v].hi, d = t.depth[v];
        // the pattern spelling exactly this node's path sorts first
        if (lo < hi && lengths[uq[lo]] == d) ++lo;
        uint32_t k = lo;
        while (k < hi) {
            uint8_t b = patterns[uq[k]][d];
            uint32_t e = k + 1;
            while (e < hi && patterns[uq[e]][d] == b) ++e;
            uint32_t c = (uint32_t)rng.size();
            rng.push_back({k, e});
            t.col.push_back(b);
            t.next.push_back((int32_t)c);
            int32_t fid = lengths[uq[k]] == d + 1 ? (int32_t)uq[k] : -1;
            t.final_id.push_back(fid);
            t.nfinal.push_back(t.nfinal[v] + (fid >= 0 ? 1 : 0));
            if (fid >= 0) {
                t.chain[fid] = t.best[v];  // deepest pattern strictly above
                t.plen[fid] = (int32_t)(d + 1);
                t.mcnt[fid] = t.nfinal.back();
            }
            t.best.push_back(fid >= 0 ? fid : t.best[v]);
            t.depth.push_back(d + 1);
            k = e;
        }
        t.row_ptr.push_back((uint32_t)t.col.size());
    }
    const uint32_t nn = (uint32_t)rng.size();
    t.level_nodes.assign(t.max_len + 1, 0);
    for (uint32_t v = 0; v < nn; ++v) ++t.level_nodes[t.depth[v]];

    // Top-level tables for k = 0 .. K, K < shortest pattern, so that no
    // pattern ends within the levels a table resolves.
    for (int k = 0; k <= kMaxDenseK; ++k) {
        t.dense[k].clear();
        for (int w = 0; w < kFilterWidths; ++w) t.filter[k][w].clear();
        t.first[k] = t.nlevel[k] = 0;
    }
    const uint32_t kcap = m ? std::min<uint32_t>(t.min_len - 1, kMaxDenseK) : 0;
    const uint64_t max_codes = kFilterBudget;  // C^k * 8 bits <= budget
    uint32_t K = 0;
    for (uint32_t k = 1; k <= kcap; ++k) {
        if (ipow_capped(t.C, (int)k, max_codes) == 0) break;
        K = k;
    }
    t.dense_k_max = K;

    // code: base-C code of a node's path (first byte most significant), the
    // order in which BFS numbers each level. With the byte alphabet the
    // filter is indexed instead by the little-endian path (first byte least
    // significant), which the kernel reads straight from the text.
    const bool le = t.C == 256;
    // depth of the paths the filters are built from: up to K+2 (Bloom)
    const uint32_t D = le ? K + 2 : K + 1;
    std::vector<uint64_t> code(nn, 0), fcode(nn, 0);
    for (uint32_t v = 0; v < nn; ++v) {
        if (t.depth[v] >= D) break;  // BFS: depths never decrease
        for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e) {
            code[t.next[e]] = code[v] * t.C + t.cls[t.col[e]];
            fcode[t.next[e]] = le ? fcode[v] | ((uint64_t)t.col[e] << (8 * t.depth[v]))
                                  : code[t.next[e]];
        }
    }
    std::vector<uint32_t> lvl_begin(K + 3, nn), lvl_count(K + 3, 0);
    for (uint32_t v = 0; v < nn; ++v) {
        uint32_t d = t.depth[v];
        if (d > K + 2) break;
        if (lvl_count[d]++ == 0) lvl_begin[d] = v;
    }
    for (uint32_t k = 0; k <= K; ++k) {
        const uint64_t codes = ipow_capped(t.C, (int)k, ~0ull);
        t.first[k] = lvl_count[k] ? lvl_begin[k] : 0;
        t.nlevel[k] = lvl_count[k];
        // a Bloom level may test k+2 bytes only if no pattern ends at k+1
        t.gram[k] = (le && k >= kBloomK && k + 2 <= 4 && t.min_len >= k + 2) ? k + 2 : k + 1;
        if (k >= 1) {
            uint64_t words = (codes + 31) / 32;
            words += words & 1;  // even: copied in 16-byte units
            std::vector<uint32_t> &tab = t.dense[k];
            tab.assign(2 * words, 0);
            uint64_t prev = 0;
            for (uint32_t i = 0; i < lvl_count[k]; ++i) {
                const uint64_t c = code[lvl_begin[k] + i];
                if (i > 0 && c <= prev) {
                    msg = "internal: depth-k nodes not in code order";
                    return PM_ERR_INVAL;
                }
                prev = c;
                tab[2 * (c >> 5)] |= 1u << (c & 31);
            }
            uint32_t run = 0;
            for (uint64_t w = 0; w < words; ++w) {
                tab[2 * w + 1] = run;
                run += (uint32_t)__builtin_popcount(tab[2 * w]);
            }
        }
        for (int wi = 0; wi < kFilterWidths; ++wi) {
            const uint32_t W = 8u << wi;
            const uint64_t bits = codes * W;
            if (bits / 8 > kFilterBudget) continue;
            uint64_t words = (bits + 31) / 32;
            words = (words + 3) & ~3ull;  // 16-byte units
            std::vector<uint32_t> &f = t.filter[k][wi];
            f.assign(words, 0);
            if (le && k >= kBloomK) {
                // byte alphabet, k >= 2: blocked Bloom filter of the root
                // paths of length g (read little-endian) over 2^(8k + log2 W)
                // bits; g = k+2 when no pattern ends at depth k+1
                const uint32_t g = t.gram[k];
                const uint32_t word_bits = 8 * k + (3 + wi) - 5;
                for (uint32_t i = 0; i < lvl_count[g]; ++i) {
                    const BloomProbe b = bloom_probe((uint32_t)fcode[lvl_begin[g] + i], g, word_bits);
                    f[b.word] |= b.mask;
                }
                continue;
            }
            for (uint32_t i = 0; i < lvl_count[k]; ++i) {
                const uint32_t v = lvl_begin[k] + i;
                const uint64_t c = fcode[v];
                for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e) {
                    const uint64_t h = t.cls[t.col[e]] % W;
                    // byte alphabet: bit (h << 8k) | path; else: path * W + h
                    const uint64_t bit = le ? (h << (8 * k)) | c : c * W + h;
                    f[bit >> 5] |= 1u << (bit & 31);
                }
            }
        }
    }

    // Deep level (byte classes): the root paths of depth D2, K + 2 <= D2 <
    // shortest pattern, as a bitmap with ranks over base-U codes, U = the
    // used classes (a byte of the "other" class is on no path). A position
    // whose D2-gram is not a root path cannot match (D2 < shortest
    // pattern); one that is starts its walk at depth D2.
    t.deep_k = t.deep_U = t.deep_first = 0;
    t.deep.clear();
    if (!le && m > 0) {
        const uint32_t U = t.C - 1;
        uint32_t D2 = 0;
        for (uint32_t d = K + 2; d <= std::min<uint32_t>(t.min_len - 1, kDeepMaxK); ++d) {
            if (ipow_capped(U, (int)d, kDeepCodes) == 0) break;
            D2 = d;
        }
        if (D2) {
            std::vector<uint64_t> code2(nn, 0);
            uint32_t first2 = 0;
            for (uint32_t d = 0; d < D2; ++d) first2 += t.level_nodes[d];
            for (uint32_t v = 0; v < first2; ++v)  // BFS: nodes above depth D2
                for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e)
                    code2[t.next[e]] = code2[v] * U + t.cls[t.col[e]];
            const uint64_t codes = ipow_capped(U, (int)D2, ~0ull);
            uint64_t words = (codes + 31) / 32;
            words += words & 1;
            t.deep.assign(2 * words, 0);
            uint64_t prev = 0;
            for (uint32_t i = 0; i < t.level_nodes[D2]; ++i) {
                const uint64_t c = code2[first2 + i];
                if (t.depth[first2 + i] != D2 || (i > 0 && c <= prev)) {
                    msg = "internal: deep level not in code order";
                    return PM_ERR_INVAL;
                }
                prev = c;
                t.deep[2 * (c >> 5)] |= 1u << (c & 31);
            }
            uint32_t run = 0;
            for (uint64_t w = 0; w < words; ++w) {
                t.deep[2 * w + 1] = run;
                run += (uint32_t)__builtin_popcount(t.deep[2 * w]);
            }
            t.deep_k = D2;
            t.deep_U = U;
            t.deep_first = first2;
        }
    }
    return PM_OK;
}

}  // namespace pm
