// Stream scans (Section II-B's overlap rule applied to a text arriving in
// chunks): one kernel prepares a push. It copies the held bytes (the carry)
// and the new chunk back to back into the scanner's buffer, keeps the bytes
// the next push will need as the new carry, and zeroes the push's count, so
// that a push is this launch plus one scan.
#include "pm_internal.h"

namespace pm {
namespace {

__global__ void pm_gather_kernel(const uint8_t *carry, uint64_t nc, const uint8_t *chunk,
                                 uint64_t len, uint8_t *dst, uint8_t *carry_out,
                                 uint64_t keep_from, uint64_t nkeep, int64_t *count)
{
    const uint64_t n = nc + len;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint8_t b = j < nc ? carry[j] : chunk[j - nc];
        dst[j] = b;
        if (j >= keep_from && j - keep_from < nkeep) carry_out[j - keep_from] = b;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0;
}

}  // namespace

int launch_gather(const uint8_t *carry, uint64_t nc, const uint8_t *chunk, uint64_t len,
                  uint8_t *dst, uint8_t *carry_out, uint64_t keep_from, uint64_t nkeep,
                  int64_t *count, void *stream, std::string &msg)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n = nc + len;
    const uint32_t threads = 256;
    uint64_t blocks = (n + threads * 16 - 1) / (threads * 16);
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    pm_gather_kernel<<<(unsigned)blocks, threads, 0, st>>>(carry, nc, chunk, len, dst, carry_out,
                                                          keep_from, nkeep, count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        msg = std::string("gather launch: ") + cudaGetErrorString(e);
        return PM_ERR_CUDA;
    }
    return PM_OK;
}

}  // namespace pm
