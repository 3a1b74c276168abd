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

// Byte alphabet: the shared-memory filters and dense tables of levels
// k = 0 .. K, K < shortest pattern, so that no pattern ends within the
// levels a table resolves (at most two levels: 256^k codes fit the budget).
int build_byte_tables(HostTrie &t, uint32_t nn, const std::vector<uint32_t> &lvl_begin,
                      const std::vector<uint32_t> &lvl_count, std::string &msg)
{
    const uint32_t m = (uint32_t)t.n_patterns;
    const uint32_t kcap = m ? std::min<uint32_t>(t.min_len - 1, kMaxDenseK) : 0;
    uint32_t K = 0;
    for (uint32_t k = 1; k <= kcap; ++k) {
        if (ipow_capped(256, (int)k, kFilterBudget) == 0) break;
        K = k;
    }
    t.dense_k_max = K;
    // code: the path's bytes, first byte most significant (the order in which
    // BFS numbers each level); fcode: the same path read little-endian (first
    // byte least significant), as the kernel reads it straight from the text
    const uint32_t D = K + 2;  // deepest path a filter is built from (Bloom)
    std::vector<uint64_t> code(nn, 0), fcode(nn, 0);
    for (uint32_t v = 0; v < nn; ++v) {
        if (t.depth[v] >= D) break;  // BFS: depths never decrease
        for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e) {
            code[t.next[e]] = code[v] * 256 + t.col[e];
            fcode[t.next[e]] = fcode[v] | ((uint64_t)t.col[e] << (8 * t.depth[v]));
        }
    }
    auto begin = [&](uint32_t d) { return d < lvl_begin.size() ? lvl_begin[d] : nn; };
    auto count = [&](uint32_t d) { return d < lvl_count.size() ? lvl_count[d] : 0u; };
    for (uint32_t k = 0; k <= K; ++k) {
        const uint64_t codes = ipow_capped(256, (int)k, ~0ull);
        t.first[k] = count(k) ? begin(k) : 0;
        t.nlevel[k] = count(k);
        // a Bloom level may test k+2 bytes only if no pattern ends at k+1
        t.gram[k] = (k >= kBloomK && k + 2 <= 4 && t.min_len >= k + 2) ? k + 2 : k + 1;
        if (k >= 1) {
            uint64_t words = (codes + 31) / 32;
            words += words & 1;  // even: 16-byte units
            std::vector<uint32_t> &tab = t.dense[k];
            tab.assign(2 * words, 0);
            uint64_t prev = 0;
            for (uint32_t i = 0; i < count(k); ++i) {
                const uint64_t c = code[begin(k) + i];
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
            if (k >= kBloomK) {
                // blocked Bloom filter of the root paths of length g (read
                // little-endian) over 2^(8k + log2 W) bits
                const uint32_t g = t.gram[k];
                const uint32_t word_bits = 8 * k + (3 + wi) - 5;
                for (uint32_t i = 0; i < count(g); ++i) {
                    const BloomProbe b = bloom_probe((uint32_t)fcode[begin(g) + i], g, word_bits);
                    f[b.word] |= b.mask;
                }
                continue;
            }
            for (uint32_t i = 0; i < count(k); ++i) {
                const uint32_t v = begin(k) + i;
                for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e) {
                    const uint64_t h = t.col[e] % W;
                    const uint64_t bit = (h << (8 * k)) | fcode[v];
                    f[bit >> 5] |= 1u << (bit & 31);
                }
            }
        }
    }
    return PM_OK;
}

// Byte classes: the packed filters of depths F = 1 .. F_max and the deep
// level of depth D (see pm_internal.h). Both depths are at most the shortest
// pattern; F_max * cb <= 20 bits (a 128 KiB filter), D * cb <= 26 bits.
int build_class_tables(HostTrie &t, uint32_t nn, const std::vector<uint32_t> &lvl_begin,
                       const std::vector<uint32_t> &lvl_count, std::string &msg)
{
    const uint32_t m = (uint32_t)t.n_patterns;
    const uint32_t U = t.C - 1;  // used classes (the last class is "other")
    uint32_t cb = 1;
    while ((1u << cb) < U) ++cb;
    t.cb = cb;
    t.other_check = U == (1u << cb) ? 1u : 0u;
    // a byte of no pattern gets the code U when it fits in cb bits (then no
    // path contains it); otherwise (U == 2^cb, so cb <= 7) bit 7 flags it
    for (int b = 0; b < 256; ++b) {
        const uint32_t c = t.cls[b];
        t.lut[b] = c < U ? (uint8_t)c : (uint8_t)(t.other_check ? 0x80u : U);
    }
    if (cb == 2 && U == 4) {
        for (uint32_t s = 0; s <= 5 && t.sw_shift == kNoSwar; ++s) {
            uint32_t seen = 0;
            bool ok = true;
            for (int b = 0; b < 256 && ok; ++b)
                if (t.cls[b] < U) {
                    const uint32_t f = ((uint32_t)b >> s) & 7u;
                    ok = !((seen >> f) & 1u);
                    seen |= 1u << f;
                }
            if (!ok) continue;
            t.sw_shift = s;
            for (uint32_t f = 0; f < 8; ++f) {
                t.sw_cls[f] = 0;
                t.sw_sym[f] = (uint8_t)((f ^ 1u) << s);  // field f ^ 1: matches no byte of field f
            }
            for (int b = 0; b < 256; ++b)
                if (t.cls[b] < U) {
                    const uint32_t f = ((uint32_t)b >> s) & 7u;
                    t.sw_cls[f] = (uint8_t)t.cls[b];
                    t.sw_sym[f] = (uint8_t)b;
                }
        }
    }
    const uint32_t FM = m ? std::min<uint32_t>({t.min_len, kFilterCodeBits / cb, (uint32_t)kMaxDenseK}) : 0;
    const uint32_t D = m ? std::min<uint32_t>(t.min_len, kDeepCodeBits / cb) : 0;
    t.dense_k_max = FM;
    // packed path codes of the nodes down to depth D
    std::vector<uint32_t> pc(nn, 0);
    for (uint32_t v = 0; v < nn; ++v) {
        if (t.depth[v] >= D) break;
        for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e)
            pc[t.next[e]] = (pc[v] << cb) | t.cls[t.col[e]];
    }
    auto begin = [&](uint32_t d) { return d < lvl_begin.size() ? lvl_begin[d] : nn; };
    auto count = [&](uint32_t d) { return d < lvl_count.size() ? lvl_count[d] : 0u; };
    for (uint32_t F = 1; F <= FM; ++F) {
        const uint64_t bits = 1ull << (cb * F);
        uint64_t words = (bits + 31) / 32;
        words = (words + 3) & ~3ull;  // 16-byte units
        std::vector<uint32_t> &f = t.filter[F][0];
        f.assign(words, 0);
        for (uint32_t i = 0; i < count(F); ++i) {
            const uint32_t c = pc[begin(F) + i];
            f[c >> 5] |= 1u << (c & 31);
        }
        t.gram[F] = F;
        t.first[F] = count(F) ? begin(F) : 0;
        t.nlevel[F] = count(F);
    }
    if (D) {
        const uint64_t codes = 1ull << (cb * D);
        uint64_t words = (codes + 31) / 32;
        words += words & 1;
        t.deep.assign(2 * words, 0);
        uint64_t prev = 0;
        for (uint32_t i = 0; i < count(D); ++i) {
            const uint64_t c = pc[begin(D) + i];
            if (i > 0 && c <= prev) {
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
        t.deep_k = D;
        t.deep_first = count(D) ? begin(D) : 0;
    }
    return PM_OK;
}


// Unary chains (see pm_internal.h). BFS order visits a chain's first node
// before the rest of it, so a one-child node not yet on a chain starts one.
void build_chains(HostTrie &t, uint32_t nn)
{
    t.ch_lab.clear();
    t.ch_info.clear();
    t.ch_pos.assign(nn, 0);
    t.ch_rem.assign(nn, 0);
    std::vector<uint32_t> nodes;
    for (uint32_t v = 0; v < nn; ++v) {
        if (t.row_ptr[v + 1] - t.row_ptr[v] != 1 || t.ch_rem[v] != 0) continue;
        const uint32_t o = (uint32_t)t.ch_lab.size();
        nodes.clear();
        uint32_t u = v;
        while (t.row_ptr[u + 1] - t.row_ptr[u] == 1) {
            nodes.push_back(u);
            t.ch_lab.push_back(t.col[t.row_ptr[u]]);
            t.ch_info.push_back(t.best[u]);
            t.ch_info.push_back(t.nfinal[u]);
            u = (uint32_t)t.next[t.row_ptr[u]];
        }
        t.ch_lab.push_back(0);
        t.ch_info.push_back((int32_t)u);
        t.ch_info.push_back(0);
        const uint32_t L = (uint32_t)nodes.size();
        for (uint32_t j = 0; j < L; ++j) {
            t.ch_pos[nodes[j]] = o + j;
            t.ch_rem[nodes[j]] = L - j;
        }
    }
    t.ch_lab.resize(t.ch_lab.size() + 32, 0);
}

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
    build_chains(t, nn);

    for (int k = 0; k <= kMaxDenseK; ++k) {
        t.dense[k].clear();
        for (int w = 0; w < kFilterWidths; ++w) t.filter[k][w].clear();
        t.first[k] = t.nlevel[k] = t.gram[k] = 0;
    }
    t.deep_k = t.deep_first = 0;
    t.deep.clear();
    t.cb = t.other_check = 0;
    std::memset(t.lut, 0, sizeof(t.lut));
    t.sw_shift = kNoSwar;
    std::memset(t.sw_cls, 0, sizeof(t.sw_cls));
    std::memset(t.sw_sym, 0, sizeof(t.sw_sym));
    std::vector<uint32_t> lvl_begin(t.max_len + 2, nn), lvl_count(t.max_len + 2, 0);
    for (uint32_t v = 0; v < nn; ++v)
        if (lvl_count[t.depth[v]]++ == 0) lvl_begin[t.depth[v]] = v;
    return t.C == 256 ? build_byte_tables(t, nn, lvl_begin, lvl_count, msg)
                      : build_class_tables(t, nn, lvl_begin, lvl_count, msg);
}

}  // namespace pm
