// Serving loop: transcode requests of mixed size and direction as they
// arrive, with continuous batching (declared in include/gbutf.h).
//
// The paper transcodes one buffer per call; a server sees a stream of calls.
// Here a dispatcher thread keeps up to `slots` batches in flight, each on its
// own stream and context (its own look-back scratch and batch plan), so the
// batches overlap on the GPU. Whenever a slot is free it admits the queued
// requests in arrival order, as long as their bytes fit into a device memory
// pool (input copy + worst-case output), copies their inputs into the pool
// with one gather kernel, and launches one persistent transcoding kernel over
// all of them (the batch call of api.cu). A finished batch frees its pool
// blocks and completes its requests. Every result equals that of the
// single-buffer call on the same input: the batch kernel gives each input its
// own scan, first error and result.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/gbutf.h"

namespace {

bool ok(cudaError_t e) { return e == cudaSuccess; }

using Clock = std::chrono::steady_clock;

// ---- device memory pool: first fit over one arena, coalescing frees --------
class Pool {
public:
    bool init(uint64_t bytes)
    {
        if (!ok(cudaMalloc(&base_, bytes))) return false;
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    ~Pool()
    {
        if (base_) cudaFree(base_);
    }
    // offset of a block of `bytes` (multiple of 256), or ~0 if none fits
    uint64_t alloc(uint64_t bytes)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            high_ = std::max(high_, used_);
            return off;
        }
        return ~0ull;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    uint8_t *base() const { return base_; }
    uint64_t size() const { return size_; }
    uint64_t high_water() const { return high_; }

private:
    uint8_t *base_ = nullptr;
    uint64_t size_ = 0, used_ = 0, high_ = 0;
    std::map<uint64_t, uint64_t> free_;   // offset -> bytes
};

constexpr uint64_t kAlign = 256;

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

bool is_utf16_op(int32_t op)
{
    return op == GBU_OP_UTF16LE_TO_UTF8 || op == GBU_OP_UTF8_LENGTH_FROM_UTF16LE ||
           op == GBU_OP_UTF16BE_TO_UTF8 || op == GBU_OP_UTF8_LENGTH_FROM_UTF16BE;
}

// Worst-case output bytes of a request (the capacity it is given).
uint64_t out_bytes(const gbu_request &r)
{
    if (r.op == GBU_OP_UTF8_TO_UTF16LE || r.op == GBU_OP_UTF8_TO_UTF16BE)
        return 2 * r.n;   // one unit per byte
    if (r.op == GBU_OP_UTF16LE_TO_UTF8 || r.op == GBU_OP_UTF16BE_TO_UTF8)
        return 3 * r.n;   // three bytes per unit
    return 0;
}

uint64_t in_bytes(const gbu_request &r) { return r.n * (is_utf16_op(r.op) ? 2 : 1); }

// Pool block of a request: its input copy, placed at the source's offset
// modulo 16 (so the gather copies 16-byte blocks and the kernel sees the same
// alignment), then its output.
uint64_t block_bytes(const gbu_request &r)
{
    return round_up(16 + in_bytes(r), 16) + round_up(out_bytes(r), kAlign) + kAlign;
}

struct Seg {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t n;
    uint64_t piece0;   // index of the segment's first piece (exclusive prefix)
};

constexpr uint64_t kPiece = 32 << 10;   // gather work unit (bytes)

// Copy every segment (src and dst congruent modulo 16), cut into kPiece-byte
// pieces spread over all CTAs so that large segments do not leave a tail:
// 16-byte loads and stores for the body, bytes at the unaligned edges.
__global__ void gather_kernel(const Seg *segs, uint32_t count, uint64_t pieces)
{
    for (uint64_t p = blockIdx.x; p < pieces; p += gridDim.x) {
        uint32_t lo = 0, hi = count;   // the segment holding piece p
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (segs[mid].piece0 <= p) lo = mid; else hi = mid;
        }
        const Seg g = segs[lo];
        const uint64_t b0 = (p - g.piece0) * kPiece;
        const uint64_t b1 = b0 + kPiece < g.n ? b0 + kPiece : g.n;
        const uint8_t *src = g.src + b0;
        uint8_t *dst = g.dst + b0;
        const uint64_t n = b1 - b0;
        const uint32_t head = (uint32_t)((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15);
        const uint64_t h = head < n ? head : n;
        for (uint64_t i = threadIdx.x; i < h; i += blockDim.x) dst[i] = src[i];
        const uint64_t nblk = (n - h) / 16;
        const uint4 *sv = reinterpret_cast<const uint4 *>(src + h);
        uint4 *dv = reinterpret_cast<uint4 *>(dst + h);
        for (uint64_t i = threadIdx.x; i < nblk; i += blockDim.x) dv[i] = __ldcs(sv + i);
        for (uint64_t i = h + 16 * nblk + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
}

struct Pending {
    gbu_request req;
    double t_submit = 0, t_admit = 0;
    uint64_t off = 0, bytes = 0;     // pool block
};

struct Slot {
    gbu_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    gbu_result *h_res = nullptr, *d_res = nullptr;   // pinned, mapped
    Seg *h_seg = nullptr, *d_seg = nullptr;
    std::vector<Pending> reqs;
    std::vector<gbu_batch_item> items;
    double t_launch = 0;
    uint32_t batch_id = 0;
    bool busy = false, failed = false;
};

}  // namespace

struct gbu_server {
    int device = 0;
    uint32_t max_items = 0;
    Pool pool;
    std::vector<Slot> slots;
    Clock::time_point t0;
    std::mutex mu;                         // guards queue, done, counters below
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::vector<gbu_completion> done;
    uint64_t submitted = 0, completed = 0, batches = 0;
    std::atomic<bool> stop{false};
    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    bool launch(Slot &s);
    void retire(Slot &s);
};

bool gbu_server::launch(Slot &s)
{
    const uint32_t n = (uint32_t)s.reqs.size();
    s.items.resize(n);
    uint64_t pieces = 0;
    for (uint32_t i = 0; i < n; i++) {
        const Pending &p = s.reqs[i];
        const uint8_t *src = static_cast<const uint8_t *>(p.req.in);
        uint8_t *blk = pool.base() + p.off;
        uint8_t *in = blk + (reinterpret_cast<uintptr_t>(src) & 15);
        uint8_t *out = blk + round_up(16 + in_bytes(p.req), 16);
        s.h_seg[i] = Seg{src, in, in_bytes(p.req), pieces};
        pieces += (in_bytes(p.req) + kPiece - 1) / kPiece;
        gbu_batch_item &it = s.items[i];
        it.in = p.req.n ? in : nullptr;
        it.n = p.req.n;
        it.op = p.req.op;
        it.reserved = 0;
        const bool write = p.req.op == GBU_OP_UTF8_TO_UTF16LE || p.req.op == GBU_OP_UTF16LE_TO_UTF8 ||
                           p.req.op == GBU_OP_UTF8_TO_UTF16BE || p.req.op == GBU_OP_UTF16BE_TO_UTF8;
        it.out = write ? out : nullptr;
        it.cap = write ? (is_utf16_op(p.req.op) ? 3 * p.req.n : p.req.n) : 0;
    }
    if (gbu_batch_plan(s.ctx, s.items.data(), n, s.d_res, s.stream) != GBU_OK) return false;
    if (!ok(cudaMemcpyAsync(s.d_seg, s.h_seg, n * sizeof(Seg), cudaMemcpyHostToDevice, s.stream)))
        return false;
    if (pieces) {
        gather_kernel<<<(unsigned)std::min<uint64_t>(pieces, 1216), 256, 0, s.stream>>>(s.d_seg, n,
                                                                                      pieces);
        if (!ok(cudaGetLastError())) return false;
    }
    if (gbu_batch_launch(s.ctx, s.stream) != GBU_OK) return false;
    for (uint32_t i = 0; i < n; i++) {
        const Pending &p = s.reqs[i];
        if (!p.req.out_copy || !s.items[i].out) continue;
        const uint64_t b = std::min(out_bytes(p.req), p.req.out_copy_cap_bytes);
        if (b && !ok(cudaMemcpyAsync(p.req.out_copy, s.items[i].out, b, cudaMemcpyDeviceToDevice,
                                     s.stream)))
            return false;
    }
    return ok(cudaEventRecord(s.done, s.stream));
}

void gbu_server::retire(Slot &s)
{
    const double t = now();
    std::vector<gbu_completion> out(s.reqs.size());
    for (size_t i = 0; i < s.reqs.size(); i++) {
        gbu_completion &c = out[i];
        c.tag = s.reqs[i].req.tag;
        if (s.failed) {
            c.result.status = GBU_DEVICE_ERROR;
            c.result.reserved = 0;
            c.result.in_offset = 0;
            c.result.out_len = 0;
        } else {
            c.result = s.h_res[i];
        }
        c.t_submit = s.reqs[i].t_submit;
        c.t_admit = s.reqs[i].t_admit;
        c.t_launch = s.t_launch;
        c.t_done = t;
        c.batch = s.batch_id;
        c.batch_items = (uint32_t)s.reqs.size();
    }
    std::lock_guard<std::mutex> lock(mu);
    for (const Pending &p : s.reqs) pool.release(p.off, p.bytes);
    for (auto &c : out) done.push_back(c);
    completed += out.size();
    s.reqs.clear();
    s.busy = false;
    s.failed = false;
    cv.notify_all();
}

void gbu_server::run()
{
    cudaSetDevice(device);
    while (!stop.load(std::memory_order_relaxed)) {
        bool progress = false;
        for (Slot &s : slots) {
            if (s.busy) {
                const cudaError_t e = cudaEventQuery(s.done);
                if (e == cudaErrorNotReady) continue;
                if (!ok(e)) s.failed = true;
                retire(s);
                progress = true;
            }
        }
        for (Slot &s : slots) {
            if (s.busy) continue;
            {
                std::lock_guard<std::mutex> lock(mu);
                // admit in arrival order while the pool has room
                while (!queue.empty() && s.reqs.size() < max_items) {
                    Pending p = queue.front();
                    p.bytes = block_bytes(p.req);
                    p.off = pool.alloc(p.bytes);
                    if (p.off == ~0ull) break;
                    p.t_admit = now();
                    queue.pop_front();
                    s.reqs.push_back(p);
                }
                if (s.reqs.empty()) break;
                s.batch_id = (uint32_t)batches++;
            }
            s.busy = true;
            if (!launch(s)) {
                s.failed = true;
                cudaStreamSynchronize(s.stream);
                retire(s);
            } else {
                s.t_launch = now();
            }
            progress = true;
        }
        if (!progress) std::this_thread::yield();
    }
}

extern "C" {

gbu_server *gbu_server_create(int device, uint64_t pool_bytes, uint32_t slots,
                              uint32_t max_batch_items)
{
    if (slots == 0 || slots > 16 || max_batch_items == 0 || pool_bytes < (1u << 20)) return nullptr;
    if (!ok(cudaSetDevice(device))) return nullptr;
    gbu_server *srv = new (std::nothrow) gbu_server();
    if (!srv) return nullptr;
    srv->device = device;
    srv->max_items = max_batch_items;
    bool good = srv->pool.init(pool_bytes);
    srv->slots.resize(slots);
    for (Slot &s : srv->slots) {
        if (!good) break;
        s.ctx = gbu_create(device);
        void *h = nullptr, *d = nullptr;
        good = s.ctx && gbu_reserve(s.ctx, pool_bytes) == GBU_OK &&
               ok(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) &&
               ok(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) &&
               ok(cudaHostAlloc(&h, max_batch_items * sizeof(gbu_result), cudaHostAllocMapped)) &&
               ok(cudaHostGetDevicePointer(&d, h, 0));
        if (!good) break;
        s.h_res = static_cast<gbu_result *>(h);
        s.d_res = static_cast<gbu_result *>(d);
        good = ok(cudaHostAlloc(reinterpret_cast<void **>(&s.h_seg), max_batch_items * sizeof(Seg),
                                cudaHostAllocDefault)) &&
               ok(cudaMalloc(&s.d_seg, max_batch_items * sizeof(Seg)));
        s.reqs.reserve(max_batch_items);
    }
    if (!good) {
        gbu_server_destroy(srv);
        return nullptr;
    }
    srv->t0 = Clock::now();
    srv->worker = std::thread([srv] { srv->run(); });
    return srv;
}

void gbu_server_destroy(gbu_server *srv)
{
    if (!srv) return;
    srv->stop.store(true);
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (Slot &s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.ctx) gbu_destroy(s.ctx);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_res) cudaFreeHost(s.h_res);
        if (s.h_seg) cudaFreeHost(s.h_seg);
        if (s.d_seg) cudaFree(s.d_seg);
    }
    delete srv;
}

int32_t gbu_server_submit(gbu_server *srv, const gbu_request *req)
{
    if (!srv || !req) return GBU_INVALID_ARG;
    const gbu_request &r = *req;
    if (r.op < GBU_OP_UTF8_TO_UTF16LE || r.op > GBU_OP_UTF8_LENGTH_FROM_UTF16BE) return GBU_INVALID_ARG;
    if (r.n && !r.in) return GBU_INVALID_ARG;
    if (is_utf16_op(r.op) && (reinterpret_cast<uintptr_t>(r.in) & 1u)) return GBU_INVALID_ARG;
    if (block_bytes(r) > srv->pool.size()) return GBU_INVALID_ARG;   // could never be admitted
    Pending p;
    p.req = r;
    std::lock_guard<std::mutex> lock(srv->mu);
    p.t_submit = srv->now();
    srv->queue.push_back(p);
    srv->submitted++;
    return GBU_OK;
}

uint32_t gbu_server_poll(gbu_server *srv, gbu_completion *out, uint32_t max)
{
    if (!srv || !out) return 0;
    std::lock_guard<std::mutex> lock(srv->mu);
    const uint32_t n = (uint32_t)std::min<size_t>(max, srv->done.size());
    std::copy(srv->done.begin(), srv->done.begin() + n, out);
    srv->done.erase(srv->done.begin(), srv->done.begin() + n);
    return n;
}

int32_t gbu_server_wait_idle(gbu_server *srv, double timeout_s)
{
    if (!srv) return GBU_INVALID_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    const bool idle = srv->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), [srv] {
        return srv->completed == srv->submitted;
    });
    return idle ? GBU_OK : GBU_DEVICE_TIMEOUT;
}

int32_t gbu_server_replay(gbu_server *srv, const gbu_request *reqs, const double *t_arrival,
                          uint32_t count, gbu_completion *out, double timeout_s)
{
    if (!srv || (count && (!reqs || !t_arrival || !out))) return GBU_INVALID_ARG;
    for (uint32_t i = 0; i < count; i++) {
        gbu_request r = reqs[i];
        if (r.op < GBU_OP_UTF8_TO_UTF16LE || r.op > GBU_OP_UTF8_LENGTH_FROM_UTF16BE ||
            (r.n && !r.in) || block_bytes(r) > srv->pool.size() ||
            (is_utf16_op(r.op) && (reinterpret_cast<uintptr_t>(r.in) & 1u)))
            return GBU_INVALID_ARG;
    }
    std::vector<gbu_completion> got(count);
    std::vector<char> have(count, 0);
    uint32_t n_done = 0;
    std::vector<gbu_completion> buf(1024);
    auto drain = [&]() {
        const uint32_t k = gbu_server_poll(srv, buf.data(), (uint32_t)buf.size());
        for (uint32_t j = 0; j < k; j++) {
            const uint64_t tag = buf[j].tag;
            if (tag < count && !have[tag]) {
                got[tag] = buf[j];
                have[tag] = 1;
                n_done++;
            }
        }
        return k;
    };
    const double start = srv->now();
    for (uint32_t i = 0; i < count; i++) {
        while (srv->now() - start < t_arrival[i]) {
            if (!drain()) std::this_thread::yield();
        }
        gbu_request r = reqs[i];
        r.tag = i;   // completions are matched to requests by index
        if (gbu_server_submit(srv, &r) != GBU_OK) return GBU_INVALID_ARG;
    }
    const double deadline = srv->now() + timeout_s;
    while (n_done < count) {
        if (!drain()) {
            if (srv->now() > deadline) return GBU_DEVICE_TIMEOUT;
            std::this_thread::yield();
        }
    }
    for (uint32_t i = 0; i < count; i++) {
        out[i] = got[i];
        out[i].tag = reqs[i].tag;
        // times relative to the start of the replay
        out[i].t_submit -= start;
        out[i].t_admit -= start;
        out[i].t_launch -= start;
        out[i].t_done -= start;
    }
    return GBU_OK;
}

int32_t gbu_server_stats(gbu_server *srv, gbu_server_stats_t *st)
{
    if (!srv || !st) return GBU_INVALID_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    st->submitted = srv->submitted;
    st->completed = srv->completed;
    st->batches = srv->batches;
    st->pool_bytes = srv->pool.size();
    st->pool_high_water = srv->pool.high_water();
    return GBU_OK;
}

}  // extern "C"
