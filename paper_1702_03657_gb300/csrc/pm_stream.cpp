// Streams of chunks (Section II-B: a text too long for one pass is cut into
// pieces that overlap by the longest pattern's length minus one, so that no
// match straddling a cut is lost). A scanner holds the last H = max_len - 1
// bytes it has seen (the carry) and the positions whose walks may still
// reach bytes not yet pushed; each push resolves every position below
// (bytes seen) - H, so the concatenated outputs equal one scan of the whole
// stream.
//
// A push of chunk C (c bytes) onto a stream of L bytes with R positions
// resolved (L - R <= H):
//   R' = max(R, L + c - H);
//   held positions [R, min(L, R')) are scanned on S = carry || C[0, min(c, H))
//   (at most 2H bytes), reading up to the end of S;
//   positions [L, R') are scanned in C itself, reading up to its end;
//   the new carry is the bytes [R', L + c).
// A chunk of at most kCopyMax bytes is instead copied behind the carry into
// one device buffer and scanned once (one launch instead of two; the copy
// costs less than a launch at these sizes). That buffer grows, stream
// ordered, to the largest such chunk seen.
#include <algorithm>
#include <cstring>

#include "pm_internal.h"

struct pm_scanner {
    const pm_trie *h = nullptr;
    uint64_t H = 0;      // max_len - 1
    uint64_t L = 0;      // bytes pushed
    uint64_t R = 0;      // positions resolved
    uint8_t *d_carry[2] = {nullptr, nullptr};
    int cur = 0;         // carry buffer in use
    uint8_t *d_s = nullptr;  // carry || chunk head
    uint8_t *d_buf = nullptr;  // carry || whole chunk (chunks up to kCopyMax)
    uint64_t buf_cap = 0;
    cudaStream_t last = nullptr;  // stream of the last push or finish
};

namespace {

constexpr uint64_t kCopyMax = 16ull << 20;

int sfail(int code, const std::string &msg) { return pm::set_last_error(code, msg); }

int scuda(const char *what, cudaError_t e)
{
    return pm::set_last_error(PM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Scan positions [0, n) of text (readable to limit) into ids; add to *count
// when `add`, else overwrite it.
int scan_piece(const pm_trie *h, const uint8_t *text, uint64_t n, uint64_t limit, int32_t *ids,
               int64_t *count, bool add, cudaStream_t st)
{
    pm::ScanArgs a{};
    a.text = text;
    a.offsets = nullptr;
    a.ntexts = 1;
    a.len = n;
    a.limit = limit;
    a.ids = ids;
    a.counts = count;
    a.keep_counts = add;
    std::string msg;
    const int rc = pm::launch_scan(h->dev, h->cfg, a, st, h->sms, msg);
    return rc == PM_OK ? PM_OK : sfail(rc, msg);
}

}  // namespace

extern "C" {

int pm_scanner_open(const pm_trie *h, pm_scanner **out)
{
    if (!h || !out) return sfail(PM_ERR_INVAL, "handle or out is NULL");
    if (!h->d_arena) return sfail(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return scuda("cudaGetDevice", e);
    if (dev != h->device) return sfail(PM_ERR_INVAL, "current device is not the trie's device");
    pm_scanner *s = new (std::nothrow) pm_scanner;
    if (!s) return sfail(PM_ERR_NOMEM, "scanner allocation failed");
    s->h = h;
    s->H = h->host.max_len > 0 ? h->host.max_len - 1 : 0;
    const uint64_t cb = std::max<uint64_t>(s->H, 16);
    void *p = nullptr;
    e = cudaMalloc(&p, 4 * cb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(PM_ERR_NOMEM, "scanner device buffers");
    }
    uint8_t *b = static_cast<uint8_t *>(p);
    s->d_carry[0] = b;
    s->d_carry[1] = b + cb;
    s->d_s = b + 2 * cb;
    *out = s;
    return pm::set_last_error(PM_OK, "");
}

int pm_scanner_push(pm_scanner *s, const uint8_t *d_chunk, uint64_t len, int32_t *d_ids,
                    int64_t *d_count, uint64_t *n_ids, pm_stream stream)
{
    if (!s || !d_count || !n_ids) return sfail(PM_ERR_INVAL, "scanner, count or n_ids is NULL");
    if (len > 0 && !d_chunk) return sfail(PM_ERR_INVAL, "chunk is NULL");
    if (len >= (1ull << 40)) return sfail(PM_ERR_INVAL, "chunk of 2^40 bytes or more");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s->last = st;
    const uint64_t H = s->H, L = s->L, R = s->R, Ln = L + len;
    const uint64_t Rn = std::max(R, Ln > H ? Ln - H : 0);
    const uint64_t held = std::min(L, Rn) - R;  // held positions resolved now
    const uint64_t fresh = Rn > L ? Rn - L : 0; // the chunk's own positions
    if (held + fresh > 0 && !d_ids) return sfail(PM_ERR_INVAL, "ids is NULL");
    const uint64_t carry = L - R;
    const uint64_t head = std::min(len, H);
    cudaError_t e;
    if (len > 0 && len <= kCopyMax) {
        // one scan of carry || chunk
        if (s->buf_cap < H + len) {
            const uint64_t cap = std::max<uint64_t>(H + len, 2 * s->buf_cap);
            void *nb = nullptr;
            e = cudaMallocAsync(&nb, cap, st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return sfail(PM_ERR_NOMEM, "scanner buffer of " + std::to_string(cap) + " bytes");
            }
            if (s->d_buf) cudaFreeAsync(s->d_buf, st);
            s->d_buf = static_cast<uint8_t *>(nb);
            s->buf_cap = cap;
        }
        // one launch: carry || chunk into the buffer, the next carry (bytes
        // [Rn, Ln) of the stream) saved, the count zeroed; then one scan
        // that adds to the count
        const uint64_t nc = Ln - Rn;
        std::string msg;
        int rc = pm::launch_gather(s->d_carry[s->cur], carry, d_chunk, len, s->d_buf,
                                   s->d_carry[s->cur ^ 1], Rn - R, nc, d_count, st, msg);
        if (rc != PM_OK) return sfail(rc, msg);
        if (held + fresh > 0) {
            rc = scan_piece(s->h, s->d_buf, held + fresh, carry + len, d_ids, d_count, true, st);
            if (rc != PM_OK) return rc;
        }
        s->cur ^= 1;
        s->L = Ln;
        s->R = Rn;
        *n_ids = held + fresh;
        return pm::set_last_error(PM_OK, "");
    }
    if (carry > 0) {
        e = cudaMemcpyAsync(s->d_s, s->d_carry[s->cur], carry, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return scuda("cudaMemcpyAsync", e);
        if (head) {
            e = cudaMemcpyAsync(s->d_s + carry, d_chunk, head, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return scuda("cudaMemcpyAsync", e);
        }
    }
    bool have = false;
    if (held > 0) {
        const int rc = scan_piece(s->h, s->d_s, held, carry + head, d_ids, d_count, false, st);
        if (rc != PM_OK) return rc;
        have = true;
    }
    if (fresh > 0) {
        const int rc = scan_piece(s->h, d_chunk, fresh, len, d_ids + held, d_count, have, st);
        if (rc != PM_OK) return rc;
        have = true;
    }
    if (!have) {
        e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return scuda("cudaMemsetAsync", e);
    }
    // new carry: bytes [Rn, Ln), from the chunk or (short chunk) from S
    const uint64_t nc = Ln - Rn;
    if (nc > 0) {
        const uint8_t *src = Rn >= L ? d_chunk + (Rn - L) : s->d_s + (Rn - R);
        e = cudaMemcpyAsync(s->d_carry[s->cur ^ 1], src, nc, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return scuda("cudaMemcpyAsync", e);
    }
    s->cur ^= 1;
    s->L = Ln;
    s->R = Rn;
    *n_ids = held + fresh;
    return pm::set_last_error(PM_OK, "");
}

int pm_scanner_finish(pm_scanner *s, int32_t *d_ids, int64_t *d_count, uint64_t *n_ids,
                      pm_stream stream)
{
    if (!s || !d_count || !n_ids) return sfail(PM_ERR_INVAL, "scanner, count or n_ids is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s->last = st;
    const uint64_t held = s->L - s->R;
    if (held > 0) {
        if (!d_ids) return sfail(PM_ERR_INVAL, "ids is NULL");
        const int rc = scan_piece(s->h, s->d_carry[s->cur], held, held, d_ids, d_count, false, st);
        if (rc != PM_OK) return rc;
    } else {
        const cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return scuda("cudaMemsetAsync", e);
    }
    s->L = s->R = 0;
    *n_ids = held;
    return pm::set_last_error(PM_OK, "");
}

int pm_scanner_close(pm_scanner *s)
{
    if (!s) return pm::set_last_error(PM_OK, "");
    // the stream-ordered buffer is freed once the scanner's work is done
    cudaError_t e = cudaStreamSynchronize(s->last);
    if (s->d_buf) {
        const cudaError_t e2 = cudaFree(s->d_buf);
        if (e == cudaSuccess) e = e2;
    }
    if (s->d_carry[0]) {
        const cudaError_t e2 = cudaFree(s->d_carry[0]);
        if (e == cudaSuccess) e = e2;
    }
    delete s;
    if (e != cudaSuccess) return scuda("cudaFree", e);
    return pm::set_last_error(PM_OK, "");
}

}  // extern "C"
