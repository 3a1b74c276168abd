// pm_scan_host_static: the host-buffer scan for callers that cannot allocate
// device memory.
//
// pm_scan_host allocates its device staging buffers on first use. Some
// callers cannot let a library call cudaMalloc:
//  - processes whose device memory is owned by one allocator (a framework's
//    caching allocator, or an arena reserved up front), where a raw
//    cudaMalloc/cudaFree would fragment or exceed that budget;
//  - latency-sensitive callers, for whom cudaMalloc/cudaFree add unbounded,
//    often device-synchronising, delays on the request path.
// This entry point stages the text, the ids and the count in one fixed,
// statically sized device array instead, and allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pm_internal.h"

namespace {

// Layout of the scratch array: [text: PM_STATIC_MAX_LEN][ids: 4 *
// PM_STATIC_MAX_LEN][count: 8], each part 256-byte aligned. A GPU holds this
// array (about 5 MiB) from the time this file's module is loaded there (its
// first use under lazy module loading, context creation under eager
// loading) until the process exits.
constexpr uint64_t kTextOff = 0;
constexpr uint64_t kIdsOff = PM_STATIC_MAX_LEN;
constexpr uint64_t kCountOff = kIdsOff + 4ull * PM_STATIC_MAX_LEN;
constexpr uint64_t kScratchBytes = kCountOff + 256;

static __device__ __align__(256) unsigned char g_pm_static_scratch[kScratchBytes];

// Device address of the scratch array, resolved once per device (with that
// device current) and cached for the life of the process: the array's name
// in host code is only a host stand-in for the symbol, not a device address.
// A cudaDeviceReset would leave the cached address stale; the header states
// that it is not supported after the first call.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

int scratch_address(int device, unsigned char **out, std::string &msg)
{
    if (device < 0 || device >= kMaxDevices) {
        msg = "device index out of range for the static scratch table";
        return PM_ERR_INVAL;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_pm_static_scratch);
        if (e != cudaSuccess || !ptr) {
            msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PM_ERR_CUDA;
        }
        g_addr[device] = ptr;
    }
    *out = static_cast<unsigned char *>(g_addr[device]);
    return PM_OK;
}

}  // namespace

extern "C" int pm_scan_host_static(const pm_trie *h, const uint8_t *h_text, uint64_t len,
                                   int32_t *h_ids, int64_t *h_count, pm_stream stream)
{
    if (!h) return pm::set_last_error(PM_ERR_INVAL, "handle is NULL");
    if (!h->d_arena) return pm::set_last_error(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    if (!h_count || (len > 0 && (!h_text || !h_ids)))
        return pm::set_last_error(PM_ERR_INVAL, "text, ids or count is NULL");
    if (len > PM_STATIC_MAX_LEN)
        return pm::set_last_error(PM_ERR_INVAL,
                                  "text of " + std::to_string(len) +
                                      " bytes exceeds PM_STATIC_MAX_LEN (" +
                                      std::to_string((unsigned long long)PM_STATIC_MAX_LEN) +
                                      "); use pm_scan_host");
    *h_count = 0;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return pm::set_last_error(PM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != h->device)
        return pm::set_last_error(PM_ERR_INVAL,
                                  "current device differs from the device the trie was built on");
    std::string msg;
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base, msg);
    if (rc != PM_OK) return pm::set_last_error(rc, msg);
    if (len == 0) return pm::set_last_error(PM_OK, "");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *d_text = base + kTextOff;
    int32_t *d_ids = reinterpret_cast<int32_t *>(base + kIdsOff);
    int64_t *d_count = reinterpret_cast<int64_t *>(base + kCountOff);
    e = cudaMemcpyAsync(d_text, h_text, len, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return pm::set_last_error(PM_ERR_CUDA, std::string("cudaMemcpyAsync H2D: ") + cudaGetErrorString(e));
    // The scan overwrites every id and zeroes the count before adding to it,
    // so nothing a previous call left in the array reaches this result.
    pm::ScanArgs a{};
    a.text = d_text;
    a.offsets = nullptr;
    a.ntexts = 1;
    a.len = len;
    a.limit = len;
    a.ids = d_ids;
    a.counts = d_count;
    a.lookups = nullptr;
    rc = pm::launch_scan(h->dev, h->cfg, a, st, h->sms, msg);
    if (rc != PM_OK) return pm::set_last_error(rc, msg);
    e = cudaMemcpyAsync(h_ids, d_ids, 4 * len, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_count, d_count, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return pm::set_last_error(PM_ERR_CUDA, std::string("pm_scan_host_static: ") + cudaGetErrorString(e));
    return pm::set_last_error(PM_OK, "");
}
