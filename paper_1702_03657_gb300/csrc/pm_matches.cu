// All-matches listing (Sections II-B and II-C ask for every occurrence of
// every pattern): after a single-text scan has written the longest-match id
// of every position and, per tile of 2^kMatchTileShift positions, the
// number of occurrences starting there and a bit per position that holds
// one, three kernels list every occurrence in position order, longest
// pattern first at a position:
//   1. the match count of each block of kTilesPerBlock tiles;
//   2. an exclusive scan of those block sums (one CTA);
//   3. per block, an exclusive scan of its tile counts gives each tile's
//      first output slot; warps take the tiles with matches, read the ids of
//      the positions marked in the match bits (not the whole id array), and
//      expand each into the chain of patterns on its walk (the longest
//      first, each pattern's next shorter one from the per-id table), at
//      offsets from a warp scan.
// The patterns occurring at a position are exactly the prefixes of its
// longest match that are patterns, so the ids and the chains determine the
// whole list.
#include "pm_internal.h"

namespace pm {
namespace {

constexpr uint32_t kTilesPerBlock = 1024;  // tiles per CTA of the listing kernels
constexpr uint32_t kFull = 0xffffffffu;

uint64_t round256(uint64_t x) { return (x + 255) & ~255ull; }

__device__ __forceinline__ unsigned long long warp_inclusive_scan(unsigned long long x,
                                                                  uint32_t lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the thread's exclusive prefix and sets *total.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                                   unsigned long long *ws,
                                                                   unsigned long long *total)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long x = warp_inclusive_scan(v, lane);
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) ws[lane] = warp_inclusive_scan(ws[lane], lane);
    __syncthreads();
    const unsigned long long pre = (warp ? ws[warp - 1] : 0ull) + x - v;
    *total = ws[31];
    __syncthreads();  // ws is reused by the caller's next scan
    return pre;
}

__global__ void __launch_bounds__(1024, 1) pm_tile_sums_kernel(const uint32_t *tc,
                                                               uint64_t ntiles,
                                                               unsigned long long *bsum)
{
    __shared__ unsigned long long ws[32];
    const uint64_t t = (uint64_t)blockIdx.x * kTilesPerBlock + threadIdx.x;
    unsigned long long s = t < ntiles ? tc[t] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024, 1) pm_block_scan_kernel(const unsigned long long *bsum,
                                                                uint32_t nb,
                                                                unsigned long long *boff)
{
    __shared__ unsigned long long ws[32];
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long pre = block_exclusive_scan(v, ws, &tot);
        if (i < nb) boff[i] = carry + pre;
        carry += tot;
    }
}

// One block of kTilesPerBlock tiles, one tile per thread for the scan of
// the tile counts; then each warp lists its tiles with matches, each lane
// 32 consecutive positions of the tile: one word of the match bits says
// which of them hold a match, and only their ids are read. Lanes are
// ordered by one warp scan of their record counts.
__global__ void __launch_bounds__(1024, 1) pm_matches_write_kernel(
    const int32_t *ids, const uint32_t *bits, uint64_t len, const uint32_t *tc, uint64_t ntiles,
    const unsigned long long *boff, const int4 *minfo, pm_match *out, uint64_t cap,
    uint64_t pos_base)
{
    __shared__ unsigned long long toff[kTilesPerBlock];
    __shared__ uint32_t tcs[kTilesPerBlock];
    __shared__ unsigned long long ws[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t b0 = (uint64_t)blockIdx.x * kTilesPerBlock;
    {
        const uint64_t t = b0 + threadIdx.x;
        const uint32_t c = t < ntiles ? tc[t] : 0u;
        tcs[threadIdx.x] = c;
        unsigned long long tot;
        toff[threadIdx.x] = boff[blockIdx.x] + block_exclusive_scan(c, ws, &tot);
    }
    __syncthreads();
    for (uint32_t i = warp; i < kTilesPerBlock; i += 32) {
        if (tcs[i] == 0) continue;
        const uint64_t q0 = ((b0 + i) << kMatchTileShift) + 32ull * lane;  // lane's positions
        // bit r: position q0 + r holds a match (only positions below len do)
        const uint32_t mask = q0 < len ? __ldg(bits + (q0 >> 5)) : 0u;
        unsigned long long m = 0;
        for (uint32_t w = mask; w; w &= w - 1)
            m += (unsigned long long)__ldg(&minfo[__ldg(ids + q0 + __ffs(w) - 1)].z);
        const unsigned long long x = warp_inclusive_scan(m, lane);
        unsigned long long slot = toff[i] + x - m;
        if (m == 0) continue;
        for (uint32_t w = mask; w; w &= w - 1) {
            const uint32_t r = __ffs(w) - 1;
            // the position's patterns, longest first, down the chain
            int32_t q = __ldg(ids + q0 + r);
            int4 mi = __ldg(minfo + q);
            const int32_t cnt = mi.z;
            for (int32_t k = 0; k < cnt; ++k) {
                if (slot < cap) {
                    pm_match e;
                    e.pos = pos_base + q0 + r;
                    e.id = q;
                    e.len = mi.y;
                    out[slot] = e;
                }
                ++slot;
                if (k + 1 < cnt) {
                    q = mi.x;  // next shorter pattern on the walk
                    mi = __ldg(minfo + q);
                }
            }
        }
    }
}

}  // namespace

MatchWork match_work_layout(uint64_t len)
{
    const uint64_t ntiles = (len + (1ull << kMatchTileShift) - 1) >> kMatchTileShift;
    const uint64_t nb = (ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    MatchWork W{};
    W.bits = round256(4 * ntiles);
    W.zero_bytes = W.bits + 4 * ((len + 31) / 32);
    W.bsum = round256(W.zero_bytes);
    W.boff = W.bsum + round256(8 * nb);
    W.total = W.boff + round256(8 * nb);
    return W;
}

uint64_t match_work_bytes(uint64_t len) { return match_work_layout(len).total; }

int launch_matches(const TrieDev &t, const int32_t *ids, uint64_t len, void *work,
                   pm_match *out, uint64_t capacity, void *stream, std::string &msg,
                   uint64_t pos_base)
{
    if (len == 0) return PM_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t ntiles = (len + (1ull << kMatchTileShift) - 1) >> kMatchTileShift;
    const uint64_t nb = (ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    const MatchWork W = match_work_layout(len);
    uint8_t *w = static_cast<uint8_t *>(work);
    uint32_t *tc = reinterpret_cast<uint32_t *>(w);
    const uint32_t *bits = reinterpret_cast<const uint32_t *>(w + W.bits);
    unsigned long long *bsum = reinterpret_cast<unsigned long long *>(w + W.bsum);
    unsigned long long *boff = reinterpret_cast<unsigned long long *>(w + W.boff);
    pm_tile_sums_kernel<<<(unsigned)nb, 1024, 0, st>>>(tc, ntiles, bsum);
    pm_block_scan_kernel<<<1, 1024, 0, st>>>(bsum, (uint32_t)nb, boff);
    pm_matches_write_kernel<<<(unsigned)nb, 1024, 0, st>>>(ids, bits, len, tc, ntiles, boff,
                                                           t.minfo, out, capacity, pos_base);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        msg = std::string("all-matches launch: ") + cudaGetErrorString(e);
        return PM_ERR_CUDA;
    }
    return PM_OK;
}

}  // namespace pm
