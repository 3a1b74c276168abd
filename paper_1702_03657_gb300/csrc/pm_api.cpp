// C ABI of libpm (include/pm.h): handle management, device upload, argument
// checks and error reporting around the host builder and the scan kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "pm_internal.h"

namespace {

thread_local int t_last = PM_OK;
thread_local std::string t_msg;

int fail(int code, const std::string &msg)
{
    t_last = code;
    t_msg = msg;
    return code;
}

int ok()
{
    t_last = PM_OK;
    t_msg.clear();
    return PM_OK;
}

int cuda_fail(const char *what, cudaError_t e)
{
    return fail(PM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

uint64_t csr_bytes(const pm::HostTrie &h)
{
    uint64_t n = h.final_id.size(), nnz = h.col.size();
    return 4 * (n + 1) + nnz + 4 * nnz + 4 * n;
}

// Shared memory a CTA may use on this device (opt-in limit).
int max_smem_optin(int device)
{
    int v = 0;
    if (device < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
                          cudaSuccess)
        v = 227 * 1024;
    return v;
}

int width_index(int32_t bits) { return bits == 8 ? 0 : bits == 16 ? 1 : bits == 32 ? 2 : -1; }

bool have_filter(const pm_trie *h, int32_t k, int32_t bits)
{
    const int wi = width_index(bits);
    return k >= 0 && (uint32_t)k <= h->host.dense_k_max && wi >= 0 && !h->host.filter[k][wi].empty();
}

// Narrowest filter that is exact at this level (C <= W), else the widest
// that exists, else 0.
int32_t pick_bits(const pm_trie *h, int32_t k)
{
    for (int32_t b : {8, 16, 32})
        if ((uint32_t)b >= h->host.C && have_filter(h, k, b)) return b;
    for (int32_t b : {8, 16, 32})
        if (have_filter(h, k, b)) return b;
    return 0;
}

// Single texts up to this size take the light launch form by default.
constexpr int32_t kLightMax = 64 * 1024;

// Thread counts tried for a CTA, largest first (one CTA per SM).
const int32_t kThreadChoices[] = {1024, 992, 960, 928, 896, 768, 512, 384, 256, 128};

// Byte classes: whether a lane's window of packed classes (its chunk of
// `positions` classes and the neighbour chunks covering the deepest gram it
// reads) fits the kernel's 64-bit window.
bool window_fits(const pm_trie *h, const pm_config &c)
{
    if (h->host.C == 256) return true;
    const pm::ScanLayout L = pm::scan_layout(h->dev, c);
    const uint32_t pcb = (uint32_t)c.positions * h->host.cb;
    return pcb <= 32 && (1 + L.nnb) * pcb <= 64 && L.nnb <= 8;
}

// Default launch configuration: one CTA per SM, 1 KiB tiles double-buffered
// with as many warps as the shared memory allows, sixteen positions per lane
// at the byte alphabet's Bloom level and for four-letter classes at the
// fixed shapes, eight elsewhere where the window allows, and the deepest
// filter level that fits. For
// the byte alphabet's Bloom filter the wider filter comes first (fewer
// walks); byte-class tries look up the deep level behind their filter. An
// autotuner may refine it.
//
// The shared memory a CTA takes decides how much of the SM's 256 KiB of
// L1/shared storage stays L1: the driver picks the smallest carveout that
// holds it (plus 1 KiB per CTA it keeps), in steps ending at 196 and 228
// KiB. Byte-class tries behind a deep level read the deep level, the trie
// and the text through L1 for a walk at about one position in a hundred, and
// measured much faster with the 56 KiB of L1 that the 196 KiB carveout leaves
// than with the 28 KiB of the 228 KiB one (ACGT, 1 GiB: 2.10 ms with 31
// warps under 196 KiB, 2.86 ms with 32 warps over it); their configurations
// stay within it.
constexpr uint64_t kCarveout196 = 196 * 1024;

pm_config default_config(const pm_trie *h, int smem_limit)
{
    pm_config c{};
    c.row_search = 0;
    c.ctas_per_sm = 0;
    c.stages = 2;
    c.checked = 0;
    c.layout = 0;
    c.wait_clocks = 0;
    c.light_max = kLightMax;
    c.schedule = PM_SCHED_AUTO;
    const bool ident = h->host.C == 256;
    c.deep = !ident && h->host.deep_k > 0 ? 1 : 0;
    const uint64_t limit = (uint64_t)smem_limit - 1024;
    const uint64_t deep_limit = std::min<uint64_t>(limit, kCarveout196 - 1024);
    struct Pref {
        int32_t bits, tile;
    };
    for (int32_t k = (int32_t)h->host.dense_k_max; k >= 0; --k) {
        c.dense_k = k;
        std::vector<Pref> prefs;
        if (ident && k >= 2) prefs = {{16, 1024}, {8, 2048}, {8, 1024}};
        const int32_t exact = ident ? pick_bits(h, k) : 8;
        // byte classes behind a deep level: 512-byte tiles (a warp spends more
        // of its time on L2 round trips per tile, shorter tiles keep more
        // warps streaming)
        if (c.deep)
            for (int32_t tile : {512, 1024, 256}) prefs.push_back({exact, tile});
        else
            for (int32_t tile : {1024, 2048, 512, 256}) prefs.push_back({exact, tile});
        for (const Pref &pf : prefs) {
            for (int32_t threads : kThreadChoices) {
                for (int32_t pos : {16, 8, 4}) {
                    // sixteen positions a lane: the byte alphabet's Bloom
                    // level (paper scale, 256 MiB: 0.236 ms against 0.256
                    // with eight) and the four-letter fixed shapes (ACGT,
                    // 1 GiB: 1.987 ms against 2.094)
                    const bool fixed16 = !ident && c.deep && h->host.cb == 2 && k == 10 &&
                                         h->host.deep_k == 13;
                    if (pos == 16 && !(ident && k == 2) && !fixed16) continue;
                    if (ident ? !have_filter(h, k, pf.bits) : pf.bits != 8) continue;
                    if (pf.tile % (32 * pos) != 0) continue;
                    c.threads = threads;
                    c.tile = pf.tile;
                    c.filter_bits = pf.bits;
                    c.positions = pos;
                    if (!window_fits(h, c)) continue;
                    if (pm::scan_smem_bytes(h->dev, c) <= (c.deep ? deep_limit : limit)) return c;
                }
            }
        }
    }
    c.dense_k = 0;
    c.filter_bits = 8;
    c.threads = 128;
    c.tile = 128;
    c.positions = 4;
    c.light_max = kLightMax;
    c.schedule = PM_SCHED_AUTO;
    return c;
}

int validate_config(const pm_trie *h, const pm_config &c, std::string &why)
{
    const bool ident = h->host.C == 256;
    if (c.threads < 128 || c.threads > 1024 || c.threads % 32 != 0) {
        why = "threads must be a multiple of 32 in [128, 1024]";
        return PM_ERR_INVAL;
    }
    if (c.positions == 16 &&
        !(h->host.C == 256 && c.dense_k == 2) &&
        !(h->host.C != 256 && h->host.cb == 2 && c.dense_k == 10 && c.deep && h->host.deep_k == 13)) {
        why = "16 positions per lane only for the byte alphabet at dense_k 2 and for 2-bit "
              "classes at filter depth 10 with the deep level of depth 13";
        return PM_ERR_INVAL;
    }
    if (c.positions != 4 && c.positions != 8 && c.positions != 16) {
        why = "positions must be 4, 8 or 16";
        return PM_ERR_INVAL;
    }
    if (c.tile < 32 * c.positions || c.tile > 32768 || c.tile % (32 * c.positions) != 0) {
        why = "tile must be a multiple of 32 * positions in [32 * positions, 32768]";
        return PM_ERR_INVAL;
    }
    if (c.dense_k < 0 || (uint32_t)c.dense_k > h->host.dense_k_max) {
        why = "dense_k must be in 0..dense_k_max";
        return PM_ERR_INVAL;
    }
    if (ident ? !have_filter(h, c.dense_k, c.filter_bits) : c.filter_bits != 8) {
        why = ident ? "no filter of this width at this dense_k (widths 8, 16, 32)"
                    : "byte-class tries take filter_bits 8";
        return PM_ERR_INVAL;
    }
    if (c.stages < 2 || c.stages > 4) {
        why = "stages must be 2..4";
        return PM_ERR_INVAL;
    }
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32) {
        why = "ctas_per_sm must be 0..32";
        return PM_ERR_INVAL;
    }
    if (c.row_search < 0 || c.row_search > 1 || c.checked < 0 || c.checked > 1) {
        why = "row_search and checked are 0 or 1";
        return PM_ERR_INVAL;
    }
    if (c.layout < 0 || c.layout > 1) {
        why = "layout is 0 (CRS row records) or 1 (bitmapped nodes)";
        return PM_ERR_INVAL;
    }
    if (c.deep < 0 || c.deep > 1 || (c.deep == 1 && (ident || h->host.deep_k == 0))) {
        why = "deep is 0, or 1 when the trie has a deep level (byte classes)";
        return PM_ERR_INVAL;
    }
    if (c.wait_clocks < 0) {
        why = "wait_clocks must be >= 0";
        return PM_ERR_INVAL;
    }
    if (c.light_max < 0) {
        why = "light_max must be >= 0";
        return PM_ERR_INVAL;
    }
    if (c.schedule < PM_SCHED_AUTO || c.schedule > PM_SCHED_DYNAMIC) {
        why = "schedule must be PM_SCHED_AUTO, PM_SCHED_STATIC or PM_SCHED_DYNAMIC";
        return PM_ERR_INVAL;
    }
    if (!window_fits(h, c)) {
        why = "positions x bits per class too wide for the window at this filter and deep level";
        return PM_ERR_INVAL;
    }
    uint64_t need = pm::scan_smem_bytes(h->dev, c);
    if (need + 1024 > (uint64_t)max_smem_optin(h->device)) {
        why = "configuration needs " + std::to_string(need) + " bytes of shared memory";
        return PM_ERR_INVAL;
    }
    return PM_OK;
}

// Host-side view for TrieDev fields that do not depend on the device.
void fill_dev_sizes(pm_trie *h)
{
    pm::TrieDev &d = h->dev;
    const pm::HostTrie &t = h->host;
    d.C = t.C;
    d.n_nodes = (uint32_t)t.final_id.size();
    d.nnz = (uint32_t)t.col.size();
    d.min_len = t.n_patterns ? t.min_len : 0xFFFFFFFFu;
    d.max_len = t.max_len;
    d.dense_k_max = t.dense_k_max;
    d.cb = t.cb;
    d.other_check = t.other_check;
    d.sw_shift = t.sw_shift;
    for (int w = 0; w < 2; ++w) {
        d.sw_cls[w] = d.sw_sym[w] = 0;
        for (int j = 0; j < 4; ++j) {
            d.sw_cls[w] |= (uint32_t)t.sw_cls[4 * w + j] << (8 * j);
            d.sw_sym[w] |= (uint32_t)t.sw_sym[4 * w + j] << (8 * j);
        }
    }
    d.deep_k = t.deep_k;
    d.deep_first = t.deep_first;
    d.deep_words = (uint32_t)(t.deep.size() / 2);
    d.n_ids = (uint32_t)t.chain.size();
    d.ch_len = (uint32_t)(t.ch_info.size() / 2);
    for (int k = 0; k <= pm::kMaxDenseK; ++k) {
        d.dense_words[k] = (uint32_t)(t.dense[k].size() / 2);
        d.first[k] = t.first[k];
        d.nlevel[k] = t.nlevel[k];
        d.gram[k] = t.gram[k];
        for (int w = 0; w < pm::kFilterWidths; ++w)
            d.filter_words[k][w] = (uint32_t)t.filter[k][w].size();
    }
}

int upload(pm_trie *h)
{
    const pm::HostTrie &t = h->host;
    const uint64_t n = t.final_id.size(), nnz = t.col.size();
    struct Part {
        const void *src;
        uint64_t bytes;
        uint64_t off;
    };
    std::vector<int2> emit(n);
    for (uint64_t v = 0; v < n; ++v) emit[v] = make_int2(t.best[v], t.nfinal[v]);
    // row records (first non-zero, length | has-match, first eight bytes);
    // the device derives the next state e + 1 from the non-zero's index
    std::vector<uint4> row(n);
    for (uint64_t v = 0; v < n; ++v) {
        const uint32_t r0 = t.row_ptr[v], deg = t.row_ptr[v + 1] - r0;
        uint32_t lab[2] = {0, 0};
        for (uint32_t i = 0; i < deg && i < 8; ++i) lab[i >> 2] |= (uint32_t)t.col[r0 + i] << (8 * (i & 3));
        if (deg == 1 && t.ch_rem[v] >= 2) {
            // one child, on a unary chain: the edges forced from here and
            // the chain position ride in the unused label bytes
            lab[0] |= t.ch_rem[v] << 8;
            lab[1] = t.ch_pos[v];
        }
        row[v] = make_uint4(r0, deg | (t.nfinal[v] > 0 ? 1u << 31 : 0u), lab[0], lab[1]);
    }
    for (uint64_t e = 0; e < nnz; ++e)
        if (t.next[e] != (int32_t)(e + 1)) return fail(PM_ERR_INVAL, "internal: next state is not BFS order");
    std::vector<Part> parts;
    uint64_t off = 0;
    auto add = [&](const void *src, uint64_t bytes) {
        parts.push_back({src, bytes, off});
        off = align256(off + std::max<uint64_t>(bytes, 16));
        return parts.size() - 1;
    };
    size_t i_row = add(row.data(), 16 * n);
    size_t i_col = add(t.col.data(), nnz);
    size_t i_emit = add(emit.data(), 8 * n);
    size_t i_cls = add(t.lut, 256);  // byte classes: packed class | "other" flag per byte
    const size_t i_deep = t.deep.empty() ? (size_t)-1 : add(t.deep.data(), 4 * t.deep.size());
    std::vector<int4> minfo(t.chain.size());
    for (size_t i = 0; i < minfo.size(); ++i) minfo[i] = make_int4(t.chain[i], t.plen[i], t.mcnt[i], 0);
    const size_t i_minfo = minfo.empty() ? (size_t)-1 : add(minfo.data(), 16 * minfo.size());
    // bitmapped nodes: 256-bit child bitmap + first child id per node
    std::vector<uint32_t> bm(8 * n, 0), bm_first(n);
    for (uint64_t v = 0; v < n; ++v) {
        bm_first[v] = t.row_ptr[v] + 1;  // BFS: the child of non-zero e is node e + 1
        for (uint32_t e = t.row_ptr[v]; e < t.row_ptr[v + 1]; ++e)
            bm[8 * v + (t.col[e] >> 5)] |= 1u << (t.col[e] & 31);
    }
    const size_t i_chl = add(t.ch_lab.data(), t.ch_lab.size());
    const size_t i_chi = add(t.ch_info.data(), 4 * t.ch_info.size());
    const size_t i_bm = add(bm.data(), 32 * n);
    const size_t i_bmf = add(bm_first.data(), 4 * n);
    const size_t none = (size_t)-1;
    size_t i_dense[pm::kMaxDenseK + 1];
    size_t i_f[pm::kMaxDenseK + 1][pm::kFilterWidths];
    for (int k = 0; k <= pm::kMaxDenseK; ++k) {
        i_dense[k] = t.dense[k].empty() ? none : add(t.dense[k].data(), 4 * t.dense[k].size());
        for (int w = 0; w < pm::kFilterWidths; ++w)
            i_f[k][w] = t.filter[k][w].empty() ? none
                                               : add(t.filter[k][w].data(), 4 * t.filter[k][w].size());
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute", e);
    void *arena = nullptr;
    e = cudaMalloc(&arena, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PM_ERR_NOMEM, "cudaMalloc of " + std::to_string(off) + " bytes failed");
    }
    h->d_arena = arena;
    h->device_bytes = off;
    uint8_t *base = static_cast<uint8_t *>(arena);
    for (const Part &p : parts) {
        if (!p.bytes) continue;
        e = cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail("cudaMemcpy", e);
    }
    pm::TrieDev &d = h->dev;
    d.row = reinterpret_cast<const uint4 *>(base + parts[i_row].off);
    d.col = base + parts[i_col].off;
    d.emit = reinterpret_cast<const int2 *>(base + parts[i_emit].off);
    d.cls = base + parts[i_cls].off;
    d.deep = i_deep == (size_t)-1 ? nullptr : reinterpret_cast<const uint2 *>(base + parts[i_deep].off);
    d.minfo = i_minfo == (size_t)-1 ? nullptr : reinterpret_cast<const int4 *>(base + parts[i_minfo].off);
    d.ch_lab = base + parts[i_chl].off;
    d.ch_info = reinterpret_cast<const int2 *>(base + parts[i_chi].off);
    d.bm = reinterpret_cast<const uint4 *>(base + parts[i_bm].off);
    d.bm_first = reinterpret_cast<const uint32_t *>(base + parts[i_bmf].off);
    for (int k = 0; k <= pm::kMaxDenseK; ++k) {
        d.dense[k] = i_dense[k] == none ? nullptr
                                        : reinterpret_cast<const uint2 *>(base + parts[i_dense[k]].off);
        for (int w = 0; w < pm::kFilterWidths; ++w)
            d.filter[k][w] = i_f[k][w] == none
                                 ? nullptr
                                 : reinterpret_cast<const uint32_t *>(base + parts[i_f[k][w]].off);
    }
    return PM_OK;
}

int build_common(const uint8_t *const *patterns, const uint32_t *lengths, uint32_t n,
                 pm_trie **out, uint64_t *footprint, bool device)
{
    if (!out) return fail(PM_ERR_INVAL, "out is NULL");
    *out = nullptr;
    pm_trie *h = new (std::nothrow) pm_trie();
    if (!h) return fail(PM_ERR_NOMEM, "handle allocation failed");
    std::string msg;
    int rc;
    try {
        rc = pm::build_host_trie(patterns, lengths, n, h->host, msg);
    } catch (const std::bad_alloc &) {
        rc = PM_ERR_NOMEM;
        msg = "host allocation failed while building the trie";
    }
    if (rc != PM_OK) {
        delete h;
        return fail(rc, msg);
    }
    fill_dev_sizes(h);
    if (device) {
        rc = upload(h);
        if (rc != PM_OK) {
            std::string keep = t_msg;
            pm_free(h);
            return fail(rc, keep);
        }
    }
    h->cfg = default_config(h, max_smem_optin(h->device));
    if (footprint) *footprint = csr_bytes(h->host);
    *out = h;
    return ok();
}

int scan_common(const pm_trie *h, const uint8_t *d_texts, const uint64_t *d_offsets,
                uint32_t ntexts, uint64_t len, uint64_t limit, int32_t *d_ids, int64_t *d_counts,
                uint64_t *d_lookups, const pm_config *cfg, pm_stream stream,
                uint32_t *tile_counts = nullptr, uint64_t *d_walks = nullptr,
                uint32_t *match_bits = nullptr)
{
    if (!h) return fail(PM_ERR_INVAL, "handle is NULL");
    if (!h->d_arena) return fail(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    const bool batch = d_offsets != nullptr;
    if (!d_counts) return fail(PM_ERR_INVAL, "counts is NULL");
    if (batch ? ntexts > 0 && (!d_texts || !d_ids) : len > 0 && (!d_texts || !d_ids))
        return fail(PM_ERR_INVAL, "text or ids is NULL");
    if (!batch && len >= (1ull << 40)) return fail(PM_ERR_INVAL, "text of 2^40 bytes or more");
    pm_config c = cfg ? *cfg : h->cfg;
    if (cfg) {
        std::string why;
        if (validate_config(h, c, why) != PM_OK) return fail(PM_ERR_INVAL, why);
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    if (dev != h->device)
        return fail(PM_ERR_INVAL, "current device differs from the device the trie was built on");
    pm::ScanArgs a{};
    a.text = d_texts;
    a.offsets = d_offsets;
    a.ntexts = batch ? ntexts : 1;
    a.len = len;
    a.limit = limit;
    a.ids = d_ids;
    a.counts = d_counts;
    a.lookups = reinterpret_cast<unsigned long long *>(d_lookups);
    a.tile_counts = tile_counts;
    a.match_bits = match_bits;
    a.walks = reinterpret_cast<unsigned long long *>(d_walks);
    std::string msg;
    int rc = pm::launch_scan(h->dev, c, a, stream, h->sms, msg);
    if (rc != PM_OK) return fail(rc, msg);
    return ok();
}


// Host-buffer scans: chunks of kHostChunk start positions, two slots.
constexpr uint64_t kHostChunk = 32ull << 20;

// The staging buffers and streams of pm_scan_host / pm_scan_all_host,
// allocated on first use: per slot the chunk's text (+ max_len - 1 bytes),
// its ids and count; pinned counts on the host.
int host_staging(pm_trie *h)
{
    const uint64_t overlap = h->host.max_len ? h->host.max_len - 1 : 0;
    const uint64_t slot = (kHostChunk + overlap + 255) & ~255ull;
    cudaError_t e;
    if (!h->h_streams[0]) {
        for (void *&s : h->h_streams) {
            cudaStream_t st;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail("cudaStreamCreate", e);
            s = st;
        }
    }
    if (h->hbuf_chunk != slot) {
        if (h->d_hbuf_text) cudaFree(h->d_hbuf_text);
        if (h->d_hbuf_ids) cudaFree(h->d_hbuf_ids);
        if (h->d_hbuf_counts) cudaFree(h->d_hbuf_counts);
        if (h->h_hbuf_counts) cudaFreeHost(h->h_hbuf_counts);
        h->d_hbuf_text = nullptr;
        h->d_hbuf_ids = nullptr;
        h->d_hbuf_counts = nullptr;
        h->h_hbuf_counts = nullptr;
        h->hbuf_chunk = 0;
        if (cudaMalloc(&h->d_hbuf_text, 2 * slot) != cudaSuccess ||
            cudaMalloc(&h->d_hbuf_ids, 2 * 4 * kHostChunk) != cudaSuccess ||
            cudaMalloc(&h->d_hbuf_counts, 2 * 8) != cudaSuccess ||
            cudaMallocHost(&h->h_hbuf_counts, 8 * 4096) != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ERR_NOMEM, "host-buffer scan staging buffers");
        }
        h->hbuf_chunk = slot;
    }
    return PM_OK;
}

// pm_scan_all on one device text at `pos_base` of a longer one: the scan
// with per-tile match counts, then the listing (positions + pos_base).
int scan_all_common(const pm_trie *h, const uint8_t *d_text, uint64_t len, uint64_t limit,
                    int32_t *d_ids, int64_t *d_count, pm_match *d_matches, uint64_t capacity,
                    void *d_work, pm_stream stream, uint64_t pos_base)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const pm::MatchWork W = pm::match_work_layout(len);
    if (len > 0) {
        cudaError_t e = cudaMemsetAsync(d_work, 0, W.zero_bytes, st);
        if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync", e);
    }
    uint8_t *w = static_cast<uint8_t *>(d_work);
    int rc = scan_common(h, d_text, nullptr, 1, len, limit, d_ids, d_count, nullptr, nullptr,
                         stream, len > 0 ? reinterpret_cast<uint32_t *>(w) : nullptr, nullptr,
                         len > 0 ? reinterpret_cast<uint32_t *>(w + W.bits) : nullptr);
    if (rc != PM_OK || len == 0) return rc;
    std::string msg;
    rc = pm::launch_matches(h->dev, d_ids, len, d_work, d_matches, capacity, stream, msg, pos_base);
    if (rc != PM_OK) return fail(rc, msg);
    return PM_OK;
}

}  // namespace

namespace pm {
int set_last_error(int code, const std::string &msg)
{
    t_last = code;
    t_msg = msg;
    return code;
}
}  // namespace pm

extern "C" {

int pm_build(const uint8_t *const *patterns, const uint32_t *lengths, uint32_t n, pm_trie **out,
             uint64_t *footprint_bytes)
{
    return build_common(patterns, lengths, n, out, footprint_bytes, true);
}

int pm_build_host(const uint8_t *const *patterns, const uint32_t *lengths, uint32_t n,
                  pm_trie **out, uint64_t *footprint_bytes)
{
    return build_common(patterns, lengths, n, out, footprint_bytes, false);
}

void pm_free(pm_trie *h)
{
    if (!h) return;
    for (void *&s : h->h_streams)
        if (s) {
            cudaStreamDestroy(reinterpret_cast<cudaStream_t>(s));
            s = nullptr;
        }
    if (h->d_hbuf_text) cudaFree(h->d_hbuf_text);
    if (h->d_hbuf_ids) cudaFree(h->d_hbuf_ids);
    if (h->d_hbuf_counts) cudaFree(h->d_hbuf_counts);
    if (h->h_hbuf_counts) cudaFreeHost(h->h_hbuf_counts);
    if (h->d_hbuf_work) cudaFree(h->d_hbuf_work);
    if (h->d_hbuf_match) cudaFree(h->d_hbuf_match);
    if (h->d_arena) cudaFree(h->d_arena);
    delete h;
}

int pm_stats(const pm_trie *h, pm_trie_stats *s)
{
    if (!h || !s) return fail(PM_ERR_INVAL, "handle or stats is NULL");
    const pm::HostTrie &t = h->host;
    std::memset(s, 0, sizeof(*s));
    const uint64_t n = t.final_id.size(), nnz = t.col.size();
    s->n_patterns = t.n_patterns;
    s->n_duplicates = t.n_duplicates;
    s->n_nodes = n;
    s->nnz = nnz;
    s->min_len = t.min_len;
    s->max_len = t.max_len;
    s->alphabet = t.C;
    s->dense_k_max = t.dense_k_max;
    s->crs_elements = 2 * nnz + n + 1;
    s->csr_bytes = csr_bytes(t);
    s->dense256_bytes = 256ull * 4 * n;
    s->bitmap36_bytes = 36ull * n;
    s->device_bytes = h->device_bytes;
    s->deep_bytes = 4ull * t.deep.size();
    s->deep_k = t.deep_k;
    return ok();
}

int pm_export_csr(const pm_trie *h, uint32_t *row_ptr, uint8_t *col, int32_t *next,
                  int32_t *final_id)
{
    if (!h) return fail(PM_ERR_INVAL, "handle is NULL");
    const pm::HostTrie &t = h->host;
    if (row_ptr) std::memcpy(row_ptr, t.row_ptr.data(), 4 * t.row_ptr.size());
    if (col && !t.col.empty()) std::memcpy(col, t.col.data(), t.col.size());
    if (next && !t.next.empty()) std::memcpy(next, t.next.data(), 4 * t.next.size());
    if (final_id) std::memcpy(final_id, t.final_id.data(), 4 * t.final_id.size());
    return ok();
}

int pm_get_config(const pm_trie *h, pm_config *cfg)
{
    if (!h || !cfg) return fail(PM_ERR_INVAL, "handle or config is NULL");
    *cfg = h->cfg;
    return ok();
}

int pm_set_config(pm_trie *h, const pm_config *cfg)
{
    if (!h || !cfg) return fail(PM_ERR_INVAL, "handle or config is NULL");
    std::string why;
    if (validate_config(h, *cfg, why) != PM_OK) return fail(PM_ERR_INVAL, why);
    h->cfg = *cfg;
    return ok();
}

int pm_scan(const pm_trie *h, const uint8_t *d_text, uint64_t len, pm_result out, pm_stream stream)
{
    return scan_common(h, d_text, nullptr, 1, len, len, out.ids, out.count, nullptr, nullptr,
                       stream);
}

int pm_scan_range(const pm_trie *h, const uint8_t *d_text, uint64_t start, uint64_t end,
                  uint64_t limit, pm_result out, pm_stream stream)
{
    if (start > end || end > limit)
        return fail(PM_ERR_INVAL, "range must satisfy start <= end <= limit");
    if (limit - start >= (1ull << 40)) return fail(PM_ERR_INVAL, "range of 2^40 bytes or more");
    if (end > start && !d_text) return fail(PM_ERR_INVAL, "text is NULL");
    return scan_common(h, d_text ? d_text + start : nullptr, nullptr, 1, end - start,
                       limit - start, out.ids, out.count, nullptr, nullptr, stream);
}

int pm_scan_walks(const pm_trie *h, const uint8_t *d_text, uint64_t len, int32_t *d_ids,
                  int64_t *d_count, uint64_t *d_walks, const pm_config *cfg, pm_stream stream)
{
    if (!d_walks) return fail(PM_ERR_INVAL, "walks is NULL");
    if (h && h->d_arena) {
        const cudaError_t e =
            cudaMemsetAsync(d_walks, 0, sizeof(uint64_t), reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync", e);
    }
    return scan_common(h, d_text, nullptr, 1, len, len, d_ids, d_count, nullptr, cfg, stream,
                       nullptr, d_walks);
}

uint64_t pm_scan_all_work_bytes(uint64_t len) { return pm::match_work_bytes(len); }

int pm_scan_all(const pm_trie *h, const uint8_t *d_text, uint64_t len, pm_result out,
                pm_match *d_matches, uint64_t capacity, void *d_work, uint64_t work_bytes,
                pm_stream stream)
{
    if (!h) return fail(PM_ERR_INVAL, "handle is NULL");
    if (capacity > 0 && !d_matches) return fail(PM_ERR_INVAL, "matches is NULL with capacity > 0");
    if (len >= (1ull << 40)) return fail(PM_ERR_INVAL, "text of 2^40 bytes or more");
    const uint64_t need = pm::match_work_bytes(len);
    if (len > 0 && (!d_work || work_bytes < need))
        return fail(PM_ERR_INVAL, "workspace of " + std::to_string(need) + " bytes needed");
    if (((uintptr_t)d_work & 255u) != 0) return fail(PM_ERR_INVAL, "workspace not 256-byte aligned");
    if (!h->d_arena) return fail(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    const int rc = scan_all_common(h, d_text, len, len, out.ids, out.count, d_matches, capacity,
                                   d_work, stream, 0);
    return rc != PM_OK ? rc : ok();
}

int pm_scan_all_host(pm_trie *h, const uint8_t *h_text, uint64_t len, pm_match *h_matches,
                     uint64_t capacity, uint64_t *h_count)
{
    if (!h) return fail(PM_ERR_INVAL, "handle is NULL");
    if (!h->d_arena) return fail(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    if (!h_count || (len > 0 && !h_text) || (capacity > 0 && !h_matches))
        return fail(PM_ERR_INVAL, "text, matches or count is NULL");
    *h_count = 0;
    if (len == 0) return ok();
    int rc = host_staging(h);
    if (rc != PM_OK) return rc;
    const uint64_t CH = kHostChunk;
    const uint64_t overlap = h->host.max_len ? h->host.max_len - 1 : 0;
    const uint64_t slot = h->hbuf_chunk;
    const uint64_t wbytes = (pm::match_work_bytes(CH) + 255) & ~255ull;
    cudaError_t e;
    if (h->hbuf_work_bytes != wbytes) {
        if (h->d_hbuf_work) cudaFree(h->d_hbuf_work);
        h->d_hbuf_work = nullptr;
        h->hbuf_work_bytes = 0;
        if (cudaMalloc(&h->d_hbuf_work, 2 * wbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ERR_NOMEM, "pm_scan_all_host workspace");
        }
        h->hbuf_work_bytes = wbytes;
    }
    auto grow = [&](uint64_t need) -> int {
        uint64_t cap = h->hbuf_mcap ? h->hbuf_mcap : (1ull << 16);
        while (cap < need) cap *= 2;
        if (cap == h->hbuf_mcap && h->d_hbuf_match) return PM_OK;
        for (void *s : h->h_streams) cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s));
        if (h->d_hbuf_match) cudaFree(h->d_hbuf_match);
        h->d_hbuf_match = nullptr;
        h->hbuf_mcap = 0;
        if (cudaMalloc(&h->d_hbuf_match, 2 * sizeof(pm_match) * cap) != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ERR_NOMEM, "pm_scan_all_host match buffers");
        }
        h->hbuf_mcap = cap;
        return PM_OK;
    };
    rc = grow(1);
    if (rc != PM_OK) return rc;
    const uint64_t nchunks = (len + CH - 1) / CH;
    // Chunk c runs on slot c & 1: text in, scan, listing, count out. Its list
    // is copied out once its count is known (two chunks in flight); a chunk
    // whose list outgrew the buffers is run again with larger ones.
    auto enqueue = [&](uint64_t c) -> int {
        const int b = (int)(c & 1);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(h->h_streams[b]);
        const uint64_t s0 = c * CH;
        const uint64_t npos = std::min(CH, len - s0);
        const uint64_t nread = std::min(npos + overlap, len - s0);
        uint8_t *dt = h->d_hbuf_text + b * slot;
        e = cudaMemcpyAsync(dt, h_text + s0, nread, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync H2D", e);
        int r = scan_all_common(h, dt, npos, nread, h->d_hbuf_ids + b * CH, h->d_hbuf_counts + b,
                                h->d_hbuf_match + b * h->hbuf_mcap, h->hbuf_mcap,
                                static_cast<uint8_t *>(h->d_hbuf_work) + b * wbytes,
                                reinterpret_cast<pm_stream>(st), s0);
        if (r != PM_OK) return r;
        e = cudaMemcpyAsync(h->h_hbuf_counts + b, h->d_hbuf_counts + b, 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync D2H", e);
        return PM_OK;
    };
    uint64_t c_next = 0, c_done = 0, total = 0;
    while (c_done < nchunks) {
        while (c_next < nchunks && c_next < c_done + 2) {
            rc = enqueue(c_next++);
            if (rc != PM_OK) return rc;
        }
        const int b = (int)(c_done & 1);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(h->h_streams[b]);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
        const uint64_t cnt = (uint64_t)h->h_hbuf_counts[b];
        if (cnt > h->hbuf_mcap) {
            rc = grow(cnt);
            if (rc != PM_OK) return rc;
            c_next = c_done;  // run this chunk (and the next) again
            continue;
        }
        if (total < capacity && cnt) {
            const uint64_t n = std::min(cnt, capacity - total);
            e = cudaMemcpyAsync(h_matches + total, h->d_hbuf_match + b * h->hbuf_mcap,
                                sizeof(pm_match) * n, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync D2H", e);
        }
        total += cnt;
        ++c_done;
    }
    for (void *s : h->h_streams) {
        e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s));
        if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
    }
    *h_count = total;
    return ok();
}

int pm_scan_batch(const pm_trie *h, const uint8_t *d_texts, const uint64_t *d_offsets,
                  uint32_t ntexts, int32_t *d_ids, int64_t *d_counts, pm_stream stream)
{
    if (!d_offsets) return fail(PM_ERR_INVAL, "offsets is NULL");
    return scan_common(h, d_texts, d_offsets, ntexts, 0, 0, d_ids, d_counts, nullptr, nullptr,
                       stream);
}

int pm_scan_ex(const pm_trie *h, const uint8_t *d_texts, const uint64_t *d_offsets,
               uint32_t ntexts, uint64_t len, int32_t *d_ids, int64_t *d_counts,
               uint64_t *d_lookups, const pm_config *cfg, pm_stream stream)
{
    return scan_common(h, d_texts, d_offsets, ntexts, len, len, d_ids, d_counts, d_lookups, cfg,
                       stream);
}

int pm_scan_host(pm_trie *h, const uint8_t *h_text, uint64_t len, int32_t *h_ids,
                 int64_t *h_count)
{
    if (!h) return fail(PM_ERR_INVAL, "handle is NULL");
    if (!h->d_arena) return fail(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    if (!h_count || (len > 0 && (!h_text || !h_ids)))
        return fail(PM_ERR_INVAL, "text, ids or count is NULL");
    *h_count = 0;
    if (len == 0) return ok();
    // Chunks of CH start positions; each chunk also copies the next
    // overlap = max_len - 1 bytes so that its last walks can finish.
    const uint64_t CH = kHostChunk;
    const uint64_t overlap = h->host.max_len ? h->host.max_len - 1 : 0;
    int rc0 = host_staging(h);
    if (rc0 != PM_OK) return rc0;
    const uint64_t slot = h->hbuf_chunk;
    cudaError_t e;
    const uint64_t nchunks = (len + CH - 1) / CH;
    int64_t total = 0;
    for (uint64_t c0 = 0; c0 < nchunks; c0 += 4096) {
        const uint64_t c1 = std::min(nchunks, c0 + 4096);
        for (uint64_t c = c0; c < c1; ++c) {
            const int b = (int)(c & 1);
            cudaStream_t st = reinterpret_cast<cudaStream_t>(h->h_streams[b]);
            const uint64_t s = c * CH;
            const uint64_t npos = std::min(CH, len - s);
            const uint64_t nread = std::min(npos + overlap, len - s);
            uint8_t *dt = h->d_hbuf_text + b * slot;
            int32_t *di = h->d_hbuf_ids + b * CH;
            int64_t *dc = h->d_hbuf_counts + b;
            e = cudaMemcpyAsync(dt, h_text + s, nread, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync H2D", e);
            int rc = scan_common(h, dt, nullptr, 1, npos, nread, di, dc, nullptr, nullptr,
                                 reinterpret_cast<pm_stream>(st));
            if (rc != PM_OK) return rc;
            e = cudaMemcpyAsync(h_ids + s, di, 4 * npos, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync D2H", e);
            e = cudaMemcpyAsync(h->h_hbuf_counts + (c - c0), dc, 8, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync D2H", e);
        }
        for (void *s : h->h_streams) {
            e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s));
            if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
        }
        for (uint64_t c = c0; c < c1; ++c) total += h->h_hbuf_counts[c - c0];
    }
    *h_count = total;
    return ok();
}

int pm_device_error(int *code)
{
    if (!code) return fail(PM_ERR_INVAL, "code is NULL");
    std::string msg;
    int rc = pm::read_device_error(code, msg);
    if (rc != PM_OK) return fail(rc, msg);
    return ok();
}

const char *pm_strerror(int code)
{
    switch (code) {
    case PM_OK: return "success";
    case PM_ERR_INVAL: return "invalid argument";
    case PM_ERR_NOMEM: return "out of memory";
    case PM_ERR_EMPTY_PATTERN: return "empty pattern";
    case PM_ERR_PATTERN_TOO_LONG: return "pattern longer than PM_MAX_PATTERN_LEN";
    case PM_ERR_CUDA: return "CUDA error";
    case PM_ERR_TIMEOUT: return "bounded wait timed out";
    case PM_ERR_BOUNDS: return "index out of bounds (checked scan)";
    case PM_ERR_BUSY: return "no slot or arena space available";
    case PM_ERR_NOT_FOUND: return "unknown request";
    case PM_ERR_HOST_ONLY: return "handle has no device copy";
    default: return "unknown error";
    }
}

int pm_last_error(void) { return t_last; }

const char *pm_last_error_msg(void) { return t_msg.c_str(); }

}  // extern "C"
