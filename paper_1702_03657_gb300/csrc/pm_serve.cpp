// Serving: continuous batching of scan requests on one GPU.
//
// Clients submit host texts with caller-owned device outputs. A scheduler
// thread owns the GPU side:
//  - admission: requests are taken in arrival order while a batch slot is
//    free and the device arena has room for the batch's texts (first-fit
//    over the arena); otherwise they wait until memory and slots free up;
//  - batching: everything admitted at that moment (up to max_batch requests
//    and max_batch_bytes) becomes one persistent-kernel launch over a device
//    offset table; ids are written straight into each request's own buffer;
//  - overlap: each batch runs on its own stream, up to max_inflight at once,
//    so requests that arrive while others are on the GPU start right away;
//  - completion: the batch's event is polled; its requests are marked done
//    and its arena block and slot are released.
// The trie stays resident on the device for the server's lifetime.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pm_internal.h"

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    uint64_t id;
    const uint8_t *h_text;
    uint64_t len;
    int32_t *d_ids;
    int64_t *d_count;
};

struct ReqState {
    int done = 0;   // 1 when the results are in the caller's buffers
    int error = 0;  // PM_OK or the error that failed the request
    uint64_t t_submit = 0, t_done = 0;
};

// First-fit allocator over [0, size), 256-byte granularity.
class Arena {
public:
    void init(uint64_t size) { free_.clear(); free_[0] = size; }
    bool alloc(uint64_t n, uint64_t *off)
    {
        n = std::max<uint64_t>((n + 255) & ~255ull, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const uint64_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t n)
    {
        n = std::max<uint64_t>((n + 255) & ~255ull, 256);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<uint64_t, uint64_t> free_;
};

// Requests up to this size are gathered on the host into one pinned staging
// buffer per slot and copied with a single DMA per batch.
constexpr uint64_t kSmallReq = 64ull << 10;
constexpr uint64_t kStageBytes = 8ull << 20;

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    uint8_t *h_stage = nullptr;  // pinned gather buffer for small requests
    uint64_t *h_off = nullptr;   // pinned tables for the batch in flight
    int32_t **h_ids = nullptr;
    int64_t **h_cnt = nullptr;
    uint64_t *d_off = nullptr;   // device copies
    int32_t **d_ids = nullptr;
    int64_t **d_cnt = nullptr;
    int64_t *d_counts = nullptr;  // per-text counts of the batch
    std::vector<uint64_t> reqs;
    uint64_t arena_off = 0, arena_len = 0;
    bool busy = false;
};

}  // namespace

struct pm_server {
    const pm_trie *trie = nullptr;
    pm_server_config cfg{};
    int device = -1;
    uint8_t *d_arena = nullptr;
    Arena arena;  // scheduler thread only
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv;       // new submissions, or stop
    std::condition_variable done_cv;  // completions
    std::deque<Req> incoming;         // submitted, not yet seen by the scheduler
    std::unordered_map<uint64_t, ReqState> table;
    std::atomic<uint64_t> next_id{1};
    std::atomic<bool> stop{false};
    std::atomic<int> fatal{PM_OK};
    std::string fatal_msg;
    pm_server_stats stats{};
    std::thread thr;

    std::deque<Req> pending;  // scheduler thread only
};

namespace {

void finish_requests(pm_server *s, const std::vector<uint64_t> &ids, int err)
{
    const uint64_t t = now_ns();
    {
        std::lock_guard<std::mutex> g(s->mu);
        for (uint64_t id : ids) {
            auto it = s->table.find(id);
            if (it == s->table.end()) continue;
            it->second.done = 1;
            it->second.error = err;
            it->second.t_done = t;
        }
        s->stats.completed += ids.size();
    }
    s->done_cv.notify_all();
}

void fail_server(pm_server *s, const std::string &msg)
{
    if (s->fatal.load() == PM_OK) {
        std::lock_guard<std::mutex> g(s->mu);
        s->fatal_msg = msg;
    }
    s->fatal.store(PM_ERR_CUDA);
}

// Launch the first n pending requests as one batch on slot `sl`. Inside the
// batch the small requests come first: they are gathered into the slot's
// pinned staging buffer and copied with one DMA; larger requests are copied
// straight from the caller's buffers.
bool issue_batch(pm_server *s, Slot &sl, size_t n, uint64_t bytes, uint64_t aoff)
{
    cudaStream_t st = sl.stream;
    uint64_t o = 0;
    size_t t = 0;
    sl.reqs.clear();
    // classify once: small requests while the staging buffer has room
    std::vector<char> small_req(n, 0);
    uint64_t staged = 0;
    for (size_t i = 0; i < n; ++i) {
        const uint64_t L = s->pending[i].len;
        if (L <= kSmallReq && staged + L <= kStageBytes) {
            small_req[i] = 1;
            staged += L;
        }
    }
    for (int pass = 0; pass < 2; ++pass) {
        for (size_t i = 0; i < n; ++i) {
            const Req &r = s->pending[i];
            const bool small = small_req[i] != 0;
            if ((pass == 0) != small) continue;
            if (small) {
                if (r.len) std::memcpy(sl.h_stage + o, r.h_text, r.len);
            } else if (r.len && cudaMemcpyAsync(s->d_arena + aoff + o, r.h_text, r.len,
                                                cudaMemcpyHostToDevice, st) != cudaSuccess) {
                return false;
            }
            sl.h_off[t] = o;
            sl.h_ids[t] = r.d_ids;
            sl.h_cnt[t] = r.d_count;
            sl.reqs.push_back(r.id);
            o += r.len;
            ++t;
        }
        if (pass == 0 && o &&
            cudaMemcpyAsync(s->d_arena + aoff, sl.h_stage, o, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return false;
    }
    if (t != n || o != bytes) return false;  // every request placed exactly once
    sl.h_off[n] = o;
    if (cudaMemcpyAsync(sl.d_off, sl.h_off, 8 * (n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(sl.d_ids, sl.h_ids, sizeof(void *) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(sl.d_cnt, sl.h_cnt, sizeof(void *) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return false;
    pm::ScanArgs a{};
    a.text = s->d_arena + aoff;
    a.offsets = sl.d_off;
    a.ntexts = (uint32_t)n;
    a.ids = nullptr;
    a.counts = sl.d_counts;
    a.out_ids = sl.d_ids;
    a.out_counts = sl.d_cnt;
    a.total_hint = bytes ? bytes : 1;
    std::string msg;
    if (pm::launch_scan(s->trie->dev, s->trie->cfg, a, st, s->trie->sms, msg) != PM_OK) {
        fail_server(s, msg);
        return false;
    }
    if (cudaEventRecord(sl.ev, st) != cudaSuccess) return false;
    sl.arena_off = aoff;
    sl.arena_len = bytes;
    sl.busy = true;
    s->pending.erase(s->pending.begin(), s->pending.begin() + (long)n);
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stats.batches += 1;
        s->stats.bytes += bytes;
        s->stats.max_batch_seen = std::max<uint64_t>(s->stats.max_batch_seen, n);
    }
    return true;
}

void scheduler(pm_server *s)
{
    cudaSetDevice(s->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const bool idle = s->pending.empty() &&
                              std::none_of(s->slots.begin(), s->slots.end(),
                                           [](const Slot &x) { return x.busy; });
            if (idle && s->incoming.empty() && !s->stop.load())
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            while (!s->incoming.empty()) {
                s->pending.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        // completions
        uint32_t inflight = 0;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) {
                ++inflight;
                continue;
            }
            finish_requests(s, sl.reqs, q == cudaSuccess ? PM_OK : PM_ERR_CUDA);
            if (q != cudaSuccess) fail_server(s, std::string("batch: ") + cudaGetErrorString(q));
            s->arena.release(sl.arena_off, sl.arena_len);
            sl.busy = false;
        }
        // admission and launches, in arrival order
        bool blocked = false;
        for (Slot &sl : s->slots) {
            if (sl.busy || s->pending.empty() || s->fatal.load() != PM_OK) continue;
            size_t n = 0;
            uint64_t bytes = 0;
            while (n < s->pending.size() && n < s->cfg.max_batch) {
                const uint64_t L = s->pending[n].len;
                if (n > 0 && bytes + L > s->cfg.max_batch_bytes) break;
                bytes += L;
                ++n;
            }
            uint64_t aoff = 0;
            while (n > 0 && !s->arena.alloc(bytes, &aoff)) {
                // not enough device memory: admit fewer, or wait for frees
                bytes -= s->pending[n - 1].len;
                --n;
            }
            if (n == 0) {
                blocked = true;
                break;
            }
            if (!issue_batch(s, sl, n, bytes, aoff)) {
                s->arena.release(aoff, bytes);
                fail_server(s, "batch issue failed");
                break;
            }
            ++inflight;
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.max_inflight_seen = std::max<uint64_t>(s->stats.max_inflight_seen, inflight);
            if (blocked) s->stats.admission_waits += 1;
        }
        if (s->fatal.load() != PM_OK) {
            std::vector<uint64_t> ids;
            for (const Req &r : s->pending) ids.push_back(r.id);
            s->pending.clear();
            if (!ids.empty()) finish_requests(s, ids, PM_ERR_CUDA);
        }
        if (s->stop.load() && s->pending.empty() && inflight == 0) {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->incoming.empty()) break;
        }
        if (inflight) std::this_thread::yield();
    }
}

void destroy_slots(pm_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        if (sl.h_off) cudaFreeHost(sl.h_off);
        if (sl.h_ids) cudaFreeHost(sl.h_ids);
        if (sl.h_cnt) cudaFreeHost(sl.h_cnt);
        if (sl.d_off) cudaFree(sl.d_off);
        if (sl.d_ids) cudaFree(sl.d_ids);
        if (sl.d_cnt) cudaFree(sl.d_cnt);
        if (sl.d_counts) cudaFree(sl.d_counts);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

int pm_server_create(const pm_trie *h, const pm_server_config *cfg, pm_server **out)
{
    if (!out) return pm::set_last_error(PM_ERR_INVAL, "out is NULL");
    *out = nullptr;
    if (!h) return pm::set_last_error(PM_ERR_INVAL, "handle is NULL");
    if (!h->d_arena) return pm::set_last_error(PM_ERR_HOST_ONLY, "handle was built with pm_build_host");
    pm_server_config c{};
    if (cfg) c = *cfg;
    if (!c.arena_bytes) c.arena_bytes = 256ull << 20;
    if (!c.max_inflight) c.max_inflight = 4;
    if (!c.max_batch) c.max_batch = 1024;
    if (!c.max_batch_bytes) c.max_batch_bytes = 64ull << 20;
    if (!c.max_queue) c.max_queue = 1u << 16;
    if (c.max_inflight > 64 || c.max_batch > (1u << 20))
        return pm::set_last_error(PM_ERR_INVAL, "max_inflight <= 64 and max_batch <= 2^20");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
        return pm::set_last_error(PM_ERR_INVAL, "current device is not the trie's device");
    pm_server *s = new (std::nothrow) pm_server();
    if (!s) return pm::set_last_error(PM_ERR_NOMEM, "server allocation failed");
    s->trie = h;
    s->cfg = c;
    s->device = dev;
    bool ok = cudaMalloc(&s->d_arena, c.arena_bytes) == cudaSuccess;
    s->arena.init(c.arena_bytes);
    s->slots.resize(c.max_inflight);
    const uint32_t B = c.max_batch;
    for (Slot &sl : s->slots) {
        if (!ok) break;
        ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaMallocHost(&sl.h_stage, kStageBytes) == cudaSuccess &&
             cudaMallocHost(&sl.h_off, 8ull * (B + 1)) == cudaSuccess &&
             cudaMallocHost(&sl.h_ids, sizeof(void *) * B) == cudaSuccess &&
             cudaMallocHost(&sl.h_cnt, sizeof(void *) * B) == cudaSuccess &&
             cudaMalloc(&sl.d_off, 8ull * (B + 1)) == cudaSuccess &&
             cudaMalloc(&sl.d_ids, sizeof(void *) * B) == cudaSuccess &&
             cudaMalloc(&sl.d_cnt, sizeof(void *) * B) == cudaSuccess &&
             cudaMalloc(&sl.d_counts, 8ull * B) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        destroy_slots(s);
        if (s->d_arena) cudaFree(s->d_arena);
        delete s;
        return pm::set_last_error(PM_ERR_NOMEM, "server device or pinned allocation failed");
    }
    s->thr = std::thread(scheduler, s);
    *out = s;
    return pm::set_last_error(PM_OK, "");
}

int pm_submit(pm_server *s, const uint8_t *h_text, uint64_t len, pm_result out, uint64_t *req_id)
{
    if (!s || !req_id || !out.count || (len > 0 && (!h_text || !out.ids)))
        return pm::set_last_error(PM_ERR_INVAL, "server, text, outputs or req_id is NULL");
    if (len > s->cfg.arena_bytes)
        return pm::set_last_error(PM_ERR_INVAL, "request larger than the server's arena");
    if (s->fatal.load() != PM_OK) return pm::set_last_error(PM_ERR_CUDA, "server failed: " + s->fatal_msg);
    const uint64_t id = s->next_id.fetch_add(1);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->incoming.size() >= s->cfg.max_queue)
            return pm::set_last_error(PM_ERR_BUSY, "submission queue full");
        ReqState rs;
        rs.t_submit = now_ns();
        s->table.emplace(id, rs);
        s->incoming.push_back(Req{id, h_text, len, out.ids, out.count});
        s->stats.submitted += 1;
    }
    s->cv.notify_one();
    *req_id = id;
    return pm::set_last_error(PM_OK, "");
}

int pm_poll(pm_server *s, uint64_t req_id, int *done)
{
    if (!s || !done) return pm::set_last_error(PM_ERR_INVAL, "server or done is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->table.find(req_id);
    if (it == s->table.end()) return pm::set_last_error(PM_ERR_NOT_FOUND, "unknown request id");
    *done = it->second.done;
    if (it->second.done) {
        const int err = it->second.error;
        s->table.erase(it);  // a finished request is reported once
        if (err != PM_OK) return pm::set_last_error(err, "request failed");
    }
    return pm::set_last_error(PM_OK, "");
}

int pm_wait(pm_server *s, uint64_t req_id, uint32_t timeout_ms)
{
    if (!s) return pm::set_last_error(PM_ERR_INVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(req_id);
    if (it == s->table.end()) return pm::set_last_error(PM_ERR_NOT_FOUND, "unknown request id");
    const bool ok = s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto jt = s->table.find(req_id);
        return jt == s->table.end() || jt->second.done;
    });
    if (!ok) return pm::set_last_error(PM_ERR_TIMEOUT, "request not done within the timeout");
    it = s->table.find(req_id);
    if (it == s->table.end()) return pm::set_last_error(PM_ERR_NOT_FOUND, "request already reported");
    const int err = it->second.error;
    s->table.erase(it);
    return pm::set_last_error(err, err == PM_OK ? "" : "request failed");
}

int pm_server_get_stats(pm_server *s, pm_server_stats *st)
{
    if (!s || !st) return pm::set_last_error(PM_ERR_INVAL, "server or stats is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->stats;
    return pm::set_last_error(PM_OK, "");
}

int pm_server_destroy(pm_server *s)
{
    if (!s) return pm::set_last_error(PM_OK, "");
    s->stop.store(true);
    s->cv.notify_all();
    if (s->thr.joinable()) s->thr.join();
    destroy_slots(s);
    if (s->d_arena) cudaFree(s->d_arena);
    const int fatal = s->fatal.load();
    delete s;
    return pm::set_last_error(fatal, fatal == PM_OK ? "" : "server had failed");
}

int pm_server_replay(pm_server *s, uint32_t n, const uint8_t *const *h_texts, const uint64_t *lens,
                     const uint64_t *arrival_ns, int32_t *const *d_ids, int64_t *const *d_counts,
                     uint64_t *latency_ns, uint64_t *wall_ns)
{
    if (!s || (n && (!h_texts || !lens || !arrival_ns || !d_ids || !d_counts || !latency_ns)))
        return pm::set_last_error(PM_ERR_INVAL, "NULL argument");
    std::vector<uint64_t> ids(n), due(n);
    const uint64_t start = now_ns() + 1000000;  // 1 ms to get going
    for (uint32_t i = 0; i < n; ++i) {
        due[i] = start + arrival_ns[i];
        while (now_ns() < due[i]) {
        }
        pm_result out{d_ids[i], d_counts[i]};
        int rc;
        while ((rc = pm_submit(s, h_texts[i], lens[i], out, &ids[i])) == PM_ERR_BUSY)
            std::this_thread::yield();
        if (rc != PM_OK) return rc;
    }
    uint64_t last = start;
    const uint64_t deadline = now_ns() + 120ull * 1000000000ull;
    for (uint32_t i = 0; i < n; ++i) {
        std::unique_lock<std::mutex> lk(s->mu);
        const bool ok = s->done_cv.wait_until(
            lk, std::chrono::steady_clock::time_point(std::chrono::nanoseconds(deadline)), [&] {
                auto it = s->table.find(ids[i]);
                return it == s->table.end() || it->second.done;
            });
        auto it = s->table.find(ids[i]);
        if (!ok || it == s->table.end())
            return pm::set_last_error(PM_ERR_TIMEOUT, "replay: request did not complete");
        if (it->second.error != PM_OK) return pm::set_last_error(it->second.error, "replay: request failed");
        latency_ns[i] = it->second.t_done - due[i];
        last = std::max(last, it->second.t_done);
        s->table.erase(it);
    }
    if (wall_ns) *wall_ns = last - start;
    return pm::set_last_error(PM_OK, "");
}

int pm_replay_plain(const pm_trie *h, uint32_t n, const uint8_t *const *h_texts,
                    const uint64_t *lens, const uint64_t *arrival_ns, uint8_t *const *d_texts,
                    int32_t *const *d_ids, int64_t *const *d_counts, uint64_t *latency_ns,
                    uint64_t *wall_ns, pm_stream stream)
{
    if (!h || (n && (!h_texts || !lens || !arrival_ns || !d_texts || !d_ids || !d_counts || !latency_ns)))
        return pm::set_last_error(PM_ERR_INVAL, "NULL argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    constexpr uint32_t kEv = 256;
    cudaEvent_t ev[kEv];
    for (uint32_t e = 0; e < kEv; ++e)
        if (cudaEventCreateWithFlags(&ev[e], cudaEventDisableTiming) != cudaSuccess) {
            for (uint32_t f = 0; f < e; ++f) cudaEventDestroy(ev[f]);
            return pm::set_last_error(PM_ERR_CUDA, "event creation failed");
        }
    std::vector<uint64_t> due(n), done_t(n, 0);
    uint32_t next_done = 0;  // requests complete in launch order on one stream
    uint32_t launched = 0;
    auto reap = [&](bool block) {
        while (next_done < launched) {
            cudaEvent_t e = ev[next_done % kEv];
            cudaError_t q = block ? cudaEventSynchronize(e) : cudaEventQuery(e);
            if (q == cudaErrorNotReady) return;
            done_t[next_done] = now_ns();
            ++next_done;
        }
    };
    const uint64_t start = now_ns() + 1000000;
    int rc = PM_OK;
    for (uint32_t i = 0; i < n && rc == PM_OK; ++i) {
        due[i] = start + arrival_ns[i];
        while (now_ns() < due[i]) reap(false);
        while (i >= next_done + kEv) reap(true);  // event i % kEv is free again
        if (lens[i] &&
            cudaMemcpyAsync(d_texts[i], h_texts[i], lens[i], cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = PM_ERR_CUDA;
            break;
        }
        rc = pm_scan(h, d_texts[i], lens[i], pm_result{d_ids[i], d_counts[i]}, stream);
        if (rc == PM_OK && cudaEventRecord(ev[i % kEv], st) != cudaSuccess) rc = PM_ERR_CUDA;
        if (rc == PM_OK) ++launched;
    }
    if (rc == PM_OK) {
        while (next_done < n) reap(true);
        uint64_t last = start;
        for (uint32_t i = 0; i < n; ++i) {
            latency_ns[i] = done_t[i] - due[i];
            last = std::max(last, done_t[i]);
        }
        if (wall_ns) *wall_ns = last - start;
    }
    for (uint32_t e = 0; e < kEv; ++e) cudaEventDestroy(ev[e]);
    return pm::set_last_error(rc, rc == PM_OK ? "" : "plain replay failed");
}

}  // extern "C"
