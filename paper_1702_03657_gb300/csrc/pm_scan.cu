// PFAC scan kernels for sm_103a (Section II-C: one failure-less walk per
// start position over the CRS trie of Section III).
//
// One persistent kernel serves the single-text scan and the batched scan.
// Each CTA owns every gridDim.x-th tile of the (concatenated) text:
//
//  a1 staging   thread 0 streams tile + halo (>= longest pattern) into one of
//               `stages` shared-memory buffers with a 1-D TMA bulk copy
//               completing on an mbarrier, `stages` tiles ahead (text whose
//               base is not 16-byte aligned is staged with plain loads);
//  a2 dense     the first k trie levels are resolved by one lookup of the
//               k-gram of byte classes in a shared-memory bitmap with rank
//               words (the depth-k node = first + rank);
//  a3 CRS walk  deeper levels walk the CRS rows in global memory (read-only
//               path, L2-resident) until the first mismatch or the text end;
//               an optional 32-bit child filter of the depth-k node skips
//               the first row search when the next byte cannot follow;
//  a4 emit      ids[i] = best[v], count += nfinal[v] of the deepest node v;
//               four consecutive positions per thread give one 16-byte store;
//  a5 reduce    per-text counts are summed in registers and flushed with one
//               atomic per (thread, text) that saw a match, or per CTA for a
//               single text after a warp/CTA reduction.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the CTA
// records PM_ERR_TIMEOUT in a device word, waits (bounded) for its copies in
// flight and returns. The checked variant bounds-checks every shared and
// global index and records PM_ERR_BOUNDS instead of touching memory out of
// range.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>

#include "pm_internal.h"

namespace pm {

__device__ int g_pm_dev_error;

namespace {

constexpr long long kWaitBudget = 4000000000LL;  // SM clocks (~2 s)
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
    int64_t *counts;
    unsigned long long *lookups;
    uint32_t tile;
    uint32_t halo;
    uint32_t k;
    uint32_t use_cm;
    uint32_t binary;
    uint32_t stages;
    uint32_t aligned;
    uint32_t ids_aligned;
    // shared-memory layout (byte offsets)
    uint32_t off_cm, off_lut, off_bar, off_stage, stage_bytes;
    uint32_t dense_u4, cm_u4;   // table sizes in 16-byte units
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

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
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

// Bytes staged for the tile at t0: tile + halo, clipped to the readable end
// (the total in batch mode, the single text's limit otherwise).
__device__ __forceinline__ unsigned long long tile_bytes(const KParams &p, unsigned long long t0,
                                                         unsigned long long end)
{
    unsigned long long want = (unsigned long long)p.tile + p.halo;
    unsigned long long left = end - t0;
    return left < want ? left : want;
}

// Issue the TMA copy of tile `tile_idx` into stage `s` (thread 0 only).
__device__ __forceinline__ void issue_tile(const KParams &p, uint8_t *smem, uint64_t *bars,
                                           uint32_t s, unsigned long long tile_idx,
                                           unsigned long long end)
{
    unsigned long long t0 = tile_idx * p.tile;
    uint32_t nb = (uint32_t)tile_bytes(p, t0, end);
    uint32_t nb16 = nb & ~15u;
    if (p.aligned && nb16) {
        mbar_arrive_tx(&bars[s], nb16);
        tma_load_1d(smem + p.off_stage + (size_t)s * p.stage_bytes, p.text + t0, nb16, &bars[s]);
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

template <int KC, bool IDENT, bool BATCH, int MODE>
__global__ void __launch_bounds__(512) pfac_scan_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const TrieDev &t = p.t;
    const uint32_t tid = threadIdx.x, T = blockDim.x, lane = tid & 31;

    const unsigned long long total = BATCH ? __ldg(p.offsets + p.ntexts) : p.total;
    const unsigned long long end = BATCH ? total : p.limit;
    const unsigned long long ntiles = (total + p.tile - 1) / p.tile;
    if (blockIdx.x >= ntiles) return;
    const unsigned long long my_tiles = (ntiles - 1 - blockIdx.x) / gridDim.x + 1;

    uint2 *s_dense = reinterpret_cast<uint2 *>(smem);
    uint32_t *s_cm = reinterpret_cast<uint32_t *>(smem + p.off_cm);
    uint32_t *s_lut = reinterpret_cast<uint32_t *>(smem + p.off_lut);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + p.off_bar);
    __shared__ uint32_t s_text0;
    __shared__ unsigned long long s_red[32];

    // Tables into shared memory (once per CTA).
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(t.dense[p.k]);
        uint4 *dst = reinterpret_cast<uint4 *>(s_dense);
        for (uint32_t i = tid; i < p.dense_u4; i += T) dst[i] = __ldg(src + i);
        if (p.use_cm) {
            const uint4 *cs = reinterpret_cast<const uint4 *>(t.childmask[p.k]);
            uint4 *cd = reinterpret_cast<uint4 *>(s_cm);
            for (uint32_t i = tid; i < p.cm_u4; i += T) cd[i] = __ldg(cs + i);
        }
        if (!IDENT) {
            // class LUT replicated per lane: word (b/4)*32 + lane holds the
            // classes of bytes 4*(b/4) .. +3, so lane l always hits bank l.
            for (uint32_t i = tid; i < 64 * 32; i += T) {
                uint32_t w = i >> 5;
                uint32_t v = (uint32_t)__ldg(t.cls + 4 * w) | ((uint32_t)__ldg(t.cls + 4 * w + 1) << 8) |
                             ((uint32_t)__ldg(t.cls + 4 * w + 2) << 16) |
                             ((uint32_t)__ldg(t.cls + 4 * w + 3) << 24);
                s_lut[i] = v;
            }
        }
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long pre = my_tiles < p.stages ? my_tiles : p.stages;
        for (unsigned long long i = 0; i < pre; ++i)
            issue_tile(p, smem, bars, (uint32_t)i, blockIdx.x + i * gridDim.x, end);
    }

    auto cls_of = [&](uint32_t b) -> uint32_t {
        if (IDENT) return b;
        return (s_lut[(b >> 2) * 32 + lane] >> ((b & 3) * 8)) & 0xFFu;
    };

    const uint32_t k = p.k;
    const uint32_t C = t.C;
    const uint32_t first_k = t.first[k];
    const uint32_t min_len = t.min_len;
    unsigned long long acc = 0;       // matches of the current text
    unsigned long long look = 0;      // lookups (MODE_LOOKUPS)
    uint32_t cur = 0;                 // current text (batch mode)

    for (unsigned long long it = 0; it < my_tiles; ++it) {
        const uint32_t s = (uint32_t)(it % p.stages);
        const uint32_t phase = (uint32_t)((it / p.stages) & 1);
        const unsigned long long tile_idx = blockIdx.x + it * gridDim.x;
        const unsigned long long t0 = tile_idx * p.tile;
        const uint32_t nbytes = (uint32_t)tile_bytes(p, t0, end);
        uint8_t *st = smem + p.off_stage + (size_t)s * p.stage_bytes;

        if (BATCH && tid == 0) s_text0 = find_text(p.offsets, p.ntexts, t0);
        bool ok = mbar_wait_bounded(&bars[s], phase);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (tid == 0) {
                record_error(PM_ERR_TIMEOUT);
                // copies still in flight: tiles it .. it+stages-1
                for (unsigned long long j = it; j < my_tiles && j < it + p.stages; ++j)
                    mbar_wait_bounded(&bars[j % p.stages], (uint32_t)((j / p.stages) & 1));
            }
            return;
        }
        const uint32_t nb16 = p.aligned ? (nbytes & ~15u) : 0u;
        if (nb16 < nbytes) {
            for (uint32_t i = nb16 + tid; i < nbytes; i += T) st[i] = __ldg(p.text + t0 + i);
            __syncthreads();
        }

        const uint32_t tile_n = (uint32_t)(total - t0 < p.tile ? total - t0 : p.tile);
        unsigned long long text_end;
        if (BATCH) {
            cur = s_text0;
            text_end = __ldg(p.offsets + cur + 1);
        } else {
            text_end = end;
        }

        for (uint32_t li = 4 * tid; li < tile_n; li += 4 * T) {
            uint32_t c[16];
            {
                const uint32_t *wp = reinterpret_cast<const uint32_t *>(st + li);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (w * 4 < KC + 4) {  // bytes li .. li+3+KC
                        uint32_t word;
                        if (MODE == MODE_CHECKED && li + 4 * w + 4 > p.stage_bytes) {
                            record_error(PM_ERR_BOUNDS);
                            word = 0;
                        } else {
                            word = wp[w];
                        }
#pragma unroll
                        for (int b = 0; b < 4; ++b) c[4 * w + b] = (word >> (8 * b)) & 0xFFu;
                    }
                }
                if (!IDENT) {
#pragma unroll
                    for (int j = 0; j < KC + 4 && j < 16; ++j) c[j] = cls_of(c[j]);
                }
            }
            int32_t out[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                out[q] = -1;
                const uint32_t lp = li + q;
                if (lp >= tile_n) continue;
                const unsigned long long pos = t0 + lp;
                if (BATCH) {
                    while (pos >= text_end) {
                        if (acc) {
                            atomicAdd(reinterpret_cast<unsigned long long *>(p.counts + cur), acc);
                            acc = 0;
                        }
                        ++cur;
                        text_end = __ldg(p.offsets + cur + 1);
                    }
                }
                // walk limit inside the staged buffer
                const unsigned long long lim64 = text_end - t0;
                const uint32_t lim = lim64 < nbytes ? (uint32_t)lim64 : nbytes;

                uint32_t v = 0, depth = 0;
                bool walk = true;
                if (MODE != MODE_LOOKUPS && pos + k <= text_end) {
                    uint32_t code = 0;
#pragma unroll
                    for (int j = 0; j < KC; ++j)
                        if (j < (int)k) code = IDENT ? (code << 8) | c[q + j] : code * C + c[q + j];
                    uint32_t w = code >> 5, bit = code & 31u;
                    if (MODE == MODE_CHECKED && w >= t.dense_words[k]) {
                        record_error(PM_ERR_BOUNDS);
                        continue;
                    }
                    const uint2 e = s_dense[w];
                    if ((e.x >> bit) & 1u) {
                        v = first_k + e.y + __popc(e.x & ((1u << bit) - 1u));
                        depth = k;
                        if (p.use_cm && pos + k < text_end) {
                            uint32_t nc = 0;
#pragma unroll
                            for (int j = 1; j <= KC; ++j)
                                if (j == (int)k) nc = c[q + j];
                            if (MODE == MODE_CHECKED && v - first_k >= t.nlevel[k]) {
                                record_error(PM_ERR_BOUNDS);
                                continue;
                            }
                            if (!((s_cm[v - first_k] >> (nc & 31u)) & 1u)) walk = false;
                        }
                    } else {
                        walk = false;  // stopped above depth k <= shortest pattern
                    }
                }
                if (walk) {
                    uint32_t lj = lp + depth;
                    while (lj < lim) {
                        const uint32_t b = st[lj];
                        if (MODE == MODE_CHECKED && v >= t.n_nodes) {
                            record_error(PM_ERR_BOUNDS);
                            break;
                        }
                        const uint32_t r0 = __ldg(t.row_ptr + v), r1 = __ldg(t.row_ptr + v + 1);
                        if (MODE == MODE_CHECKED && (r1 < r0 || r1 > t.nnz)) {
                            record_error(PM_ERR_BOUNDS);
                            break;
                        }
                        if (MODE == MODE_LOOKUPS) ++look;
                        uint32_t e;
                        bool found = false;
                        if (p.binary) {
                            uint32_t lo = r0, hi = r1;
                            while (lo < hi) {
                                uint32_t mid = (lo + hi) >> 1;
                                if (__ldg(t.col + mid) < b) lo = mid + 1;
                                else hi = mid;
                            }
                            e = lo;
                            found = lo < r1 && __ldg(t.col + lo) == b;
                        } else {
                            for (e = r0; e < r1; ++e) {
                                const uint32_t cb = __ldg(t.col + e);
                                if (cb >= b) {
                                    found = cb == b;
                                    break;
                                }
                            }
                        }
                        if (!found) break;
                        v = (uint32_t)__ldg(t.next + e);
                        ++lj;
                    }
                    depth = lj - lp;
                }
                if (depth >= min_len) {
                    const int2 em = __ldg(t.emit + v);
                    out[q] = em.x;
                    acc += (unsigned)em.y;
                }
            }
            const unsigned long long pos0 = t0 + li;
            if (p.ids_aligned && li + 3 < tile_n) {
                __stcs(reinterpret_cast<int4 *>(p.ids + pos0), make_int4(out[0], out[1], out[2], out[3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (li + q < tile_n) __stcs(p.ids + pos0 + q, out[q]);
            }
        }
        if (BATCH && acc) {
            atomicAdd(reinterpret_cast<unsigned long long *>(p.counts + cur), acc);
            acc = 0;
        }
        __syncthreads();  // stage s fully consumed
        if (tid == 0 && it + p.stages < my_tiles) {
            fence_proxy_async();
            issue_tile(p, smem, bars, s, blockIdx.x + (it + p.stages) * gridDim.x, end);
        }
    }

    // CTA reductions: the single-text count, and lookups.
    if (!BATCH || MODE == MODE_LOOKUPS) {
        unsigned long long a = BATCH ? 0ull : acc;
        unsigned long long l = look;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            l += __shfl_xor_sync(0xffffffffu, l, o);
        }
        if (lane == 0) s_red[tid >> 5] = a;
        __syncthreads();
        if (tid < 32) {
            unsigned long long x = tid < (T >> 5) ? s_red[tid] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (tid == 0 && x && !BATCH) atomicAdd(reinterpret_cast<unsigned long long *>(p.counts), x);
        }
        __syncthreads();
        if (MODE == MODE_LOOKUPS) {
            if (lane == 0) s_red[tid >> 5] = l;
            __syncthreads();
            if (tid < 32) {
                unsigned long long x = tid < (T >> 5) ? s_red[tid] : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (tid == 0 && x && p.lookups) atomicAdd(p.lookups, x);
            }
        }
    }
}

typedef void (*KernelFn)(KParams);

template <int KC, bool IDENT>
KernelFn pick_mode(bool batch, int mode)
{
    if (batch) {
        switch (mode) {
        case MODE_CHECKED: return pfac_scan_kernel<KC, IDENT, true, MODE_CHECKED>;
        case MODE_LOOKUPS: return pfac_scan_kernel<KC, IDENT, true, MODE_LOOKUPS>;
        default: return pfac_scan_kernel<KC, IDENT, true, MODE_FAST>;
        }
    }
    switch (mode) {
    case MODE_CHECKED: return pfac_scan_kernel<KC, IDENT, false, MODE_CHECKED>;
    case MODE_LOOKUPS: return pfac_scan_kernel<KC, IDENT, false, MODE_LOOKUPS>;
    default: return pfac_scan_kernel<KC, IDENT, false, MODE_FAST>;
    }
}

KernelFn pick_kernel(uint32_t C, uint32_t k, bool batch, int mode)
{
    if (C == 256) return pick_mode<2, true>(batch, mode);  // k <= 2 at C = 256
    if (k <= 4) return pick_mode<4, false>(batch, mode);
    return pick_mode<12, false>(batch, mode);
}

uint32_t round16(uint64_t x) { return (uint32_t)((x + 15) & ~15ull); }

struct Layout {
    uint32_t off_cm, off_lut, off_bar, off_stage, stage_bytes, total;
    uint32_t dense_u4, cm_u4, halo;
};

Layout layout(const TrieDev &t, const pm_config &cfg)
{
    Layout L{};
    const uint32_t k = (uint32_t)cfg.dense_k;
    uint64_t dense_bytes = (uint64_t)t.dense_words[k] * 8;
    L.dense_u4 = (uint32_t)(dense_bytes / 16);
    uint32_t off = round16(dense_bytes);
    L.off_cm = off;
    if (cfg.childmask && t.childmask[k]) {
        uint64_t cm_bytes = (uint64_t)((t.nlevel[k] + 3) / 4) * 16;
        if (cm_bytes == 0) cm_bytes = 16;
        L.cm_u4 = (uint32_t)(cm_bytes / 16);
        off += (uint32_t)cm_bytes;
    }
    L.off_lut = off;
    if (t.C != 256) off += 64 * 32 * 4;
    L.off_bar = off;
    off += round16((uint64_t)kMaxStages * 8);
    L.off_stage = off;
    L.halo = round16(t.max_len > 16 ? t.max_len : 16);
    L.stage_bytes = (uint32_t)cfg.tile + L.halo;
    off += (uint32_t)cfg.stages * L.stage_bytes;
    L.total = off;
    return L;
}

std::mutex g_attr_mu;

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
    if (ncount) {
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
    KernelFn fn = pick_kernel(t.C, (uint32_t)cfg.dense_k, batch, mode);
    Layout L = layout(t, cfg);

    KParams p{};
    p.t = t;
    p.text = a.text;
    p.offsets = a.offsets;
    p.ntexts = a.ntexts;
    p.total = a.len;
    p.limit = a.limit > a.len ? a.limit : a.len;
    p.ids = a.ids;
    p.counts = a.counts;
    p.lookups = a.lookups;
    p.tile = (uint32_t)cfg.tile;
    p.halo = L.halo;
    p.k = (uint32_t)cfg.dense_k;
    p.use_cm = (cfg.childmask && t.childmask[cfg.dense_k]) ? 1u : 0u;
    p.binary = cfg.row_search ? 1u : 0u;
    p.stages = (uint32_t)cfg.stages;
    p.aligned = ((uintptr_t)a.text & 15u) == 0;
    p.ids_aligned = ((uintptr_t)a.ids & 15u) == 0;
    p.off_cm = L.off_cm;
    p.off_lut = L.off_lut;
    p.off_bar = L.off_bar;
    p.off_stage = L.off_stage;
    p.stage_bytes = L.stage_bytes;
    p.dense_u4 = L.dense_u4;
    p.cm_u4 = L.cm_u4;

    cudaError_t e;
    {
        std::lock_guard<std::mutex> g(g_attr_mu);
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    }
    if (e != cudaSuccess) {
        msg = std::string("shared memory ") + std::to_string(L.total) +
              " bytes: " + cudaGetErrorString(e);
        return PM_ERR_INVAL;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void *>(fn),
                                                      cfg.threads, L.total);
    if (e != cudaSuccess || occ < 1) {
        msg = "configuration does not fit on an SM (threads " + std::to_string(cfg.threads) +
              ", shared " + std::to_string(L.total) + ")";
        return PM_ERR_INVAL;
    }
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < occ) occ = cfg.ctas_per_sm;
    unsigned long long grid = (unsigned long long)device_sms * occ;
    if (!batch) {
        unsigned long long ntiles = (a.len + cfg.tile - 1) / cfg.tile;
        if (ntiles < grid) grid = ntiles;
    }
    fn<<<(unsigned)grid, cfg.threads, L.total, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        msg = std::string("scan launch: ") + cudaGetErrorString(e);
        return PM_ERR_CUDA;
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
