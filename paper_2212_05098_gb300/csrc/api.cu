// C ABI of the library (declared in include/gbutf.h): contexts, scratch
// management, the synchronous / asynchronous / host-buffer entry points, the
// batch calls and their autotuner. Every step of the transcoding runs in the
// kernels of transcode.cuh (one translation unit per kernel shape) and
// utf32.cu; this file only validates arguments, picks a kernel shape, sizes
// scratch, enqueues work and times launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gbutf.h"
#include "kernels.h"
#include "utf32.h"
#include "validate.h"

using namespace gbu;

static_assert(sizeof(gbu_result) == sizeof(ResultSlot), "result layout");
static_assert((int)GBU_DEVICE_TIMEOUT == (int)kDeviceTimeout &&
                  (int)GBU_LONE_LOW_SURROGATE == (int)kLoneLow,
              "status numbering");

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr uint64_t kMaxUnits = 1ull << 39;

}  // namespace

namespace gbu {
// Kernel launches of every entry point (gbu_kernel_launch_count).
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

const Variant &variant(int i)
{
    switch (i) {
    case 1: return variant_256x32();
    case 2: return variant_512x32();
    case 3: return variant_128x48();
    case 4: return variant_512x48();
    default: return variant_256x48();
    }
}

int variant_index(int threads, uint32_t chunk_bytes)
{
    for (int i = 0; i < kVariants; i++)
        if (variant(i).threads == threads && variant(i).chunk_bytes == chunk_bytes) return i;
    return -1;
}

__global__ void write_result_kernel(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                    uint64_t out_len)
{
    volatile ResultSlot *r = dst;
    r->status = status;
    r->reserved = 0;
    r->in_offset = in_offset;
    r->out_len = out_len;
    __threadfence_system();
}

cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream)
{
    write_result_kernel<<<1, 1, 0, stream>>>(dst, status, in_offset, out_len);
    return cudaGetLastError();
}
}  // namespace gbu

namespace {

gbu_result make(int32_t st, uint64_t off = 0, uint64_t len = 0)
{
    gbu_result r;
    r.status = st;
    r.reserved = 0;
    r.in_offset = off;
    r.out_len = len;
    return r;
}

}  // namespace

struct gbu_ctx {
    int device = 0;
    uint8_t *scratch = nullptr;       // header + status[] + err_prefix[]
    uint64_t max_chunks = 0;
    bool dirty = true;                // header needs re-initialisation
    gbu_result *h_result = nullptr;   // pinned, mapped
    gbu_result *d_result = nullptr;   // device alias of h_result
    uint8_t *io = nullptr;            // device staging for the host-buffer forms
    size_t io_bytes = 0;
    // planned batch
    gbu::Item *d_items = nullptr, *h_items = nullptr;            // device / pinned host
    uint32_t *d_chunk_item = nullptr, *h_chunk_item = nullptr;
    unsigned long long *d_item_err = nullptr;
    unsigned int *d_item_done = nullptr;
    uint64_t items_cap = 0, chunk_map_cap = 0;
    uint32_t batch_items = 0, batch_chunks = 0;
    bool batch_write = false, batch_be = false;
    // the persistent jobs of a batch: one per input encoding (UTF-8, UTF-16),
    // each numbering its own chunks from 0 at chunk_item[grp_start[g]]
    uint32_t grp_start[2] = {0, 0}, grp_chunks[2] = {0, 0};
    int grp_in[2] = {0, 0};
    bool grp_be[2] = {false, false}, grp_write[2] = {false, false};
    // the batch's one-chunk items, run one CTA each apart from the persistent job
    gbu::Item *d_small = nullptr, *h_small = nullptr;
    uint64_t small_cap = 0;
    uint32_t batch_small = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    gbu::Tune tune;                   // launch parameters of every call on the context
    std::vector<gbu_batch_item> batch_src;   // the planned batch as the caller gave it
    gbu_result *batch_results = nullptr;
    int batch_variant = 0;            // kernel shape the batch's chunks were counted for
    uint64_t wait_ns = 0;             // limit of the kernels' bounded waits (0: the default)
    uint32_t skip_chunks = 0;         // test hook: the next launch starts at this chunk
    // host-buffer pipeline: copy streams, per-slice events and mapped results
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[64] = {}, ev_done[64] = {};
    gbu_result *h_slice_res = nullptr, *d_slice_res = nullptr;
    // UTF-32 calls: per-tile counts, offsets and first errors
    void *scratch32 = nullptr;
    size_t scratch32_bytes = 0;
};

namespace {

bool ok(cudaError_t e) { return e == cudaSuccess; }

// Properties of a gbu_op.
bool op_utf16_in(int32_t op)
{
    return op == GBU_OP_UTF16LE_TO_UTF8 || op == GBU_OP_UTF8_LENGTH_FROM_UTF16LE ||
           op == GBU_OP_UTF16BE_TO_UTF8 || op == GBU_OP_UTF8_LENGTH_FROM_UTF16BE;
}
bool op_writes(int32_t op)
{
    return op == GBU_OP_UTF8_TO_UTF16LE || op == GBU_OP_UTF16LE_TO_UTF8 ||
           op == GBU_OP_UTF8_TO_UTF16BE || op == GBU_OP_UTF16BE_TO_UTF8;
}
bool op_big_endian(int32_t op)
{
    return op == GBU_OP_UTF8_TO_UTF16BE || op == GBU_OP_UTF16BE_TO_UTF8 ||
           op == GBU_OP_UTF8_LENGTH_FROM_UTF16BE;
}

// Kernel shape of a single-buffer call of `bytes` input bytes when the
// context leaves the shape to the input's size (largest size of each class).
// From the latency sweep of every shape on GB300 (device time per call, both
// directions, mix profile): up to 1 MiB the 8 KiB chunks of 256 x 32 are
// fastest (the 12 KiB shape is 2-4 us slower per call: longer per-thread
// work and code path); from 16 MiB the default 256 x 48 is (4 MiB: within
// the timer's 2 us steps).
struct SizeClass {
    uint64_t max_bytes;
    int variant;
};
constexpr SizeClass kSizeClasses[] = {{1ull << 20, 1}, {~0ull, 0}};

int shape_for(const gbu_ctx *c, uint64_t bytes)
{
    if (c->tune.variant >= 0) return c->tune.variant;
    for (const SizeClass &k : kSizeClasses)
        if (bytes <= k.max_bytes) return k.variant;
    return 0;
}

// Smallest chunk of any shape (scratch sized for it fits every shape).
uint32_t min_chunk_bytes()
{
    uint32_t m = variant(0).chunk_bytes;
    for (int i = 1; i < kVariants; i++) m = std::min(m, variant(i).chunk_bytes);
    return m;
}

// Point a one-item job at the context's scratch.
void attach_scratch(gbu_ctx *c, Job &J)
{
    uint8_t *h = c->scratch;
    J.chunks_done = reinterpret_cast<unsigned int *>(h + kHdrChunks);
    J.claim = reinterpret_cast<unsigned int *>(h + kHdrClaim);
    J.exit_count = reinterpret_cast<unsigned int *>(h + kHdrExit);
    J.flags = reinterpret_cast<unsigned int *>(h + kHdrFlags);
    J.item_done = reinterpret_cast<unsigned int *>(h + kHdrDone);
    J.item_err = reinterpret_cast<unsigned long long *>(h + kHdrErr);
    J.epoch = reinterpret_cast<unsigned int *>(h + kHdrEpoch);
    J.status = reinterpret_cast<unsigned long long *>(h + kHeaderBytes);
    J.status_capacity = (uint32_t)c->max_chunks;
    J.err_prefix = J.status + c->max_chunks;
}

// Make sure scratch covers `chunks` chunks; (re)initialise the header.
int32_t ensure_scratch(gbu_ctx *c, uint64_t chunks, cudaStream_t stream)
{
    if (chunks > c->max_chunks) {
        uint64_t want = c->max_chunks ? c->max_chunks : 256;
        while (want < chunks) want *= 2;
        if (c->scratch) {
            if (!ok(cudaStreamSynchronize(stream)) || !ok(cudaDeviceSynchronize()))
                return GBU_DEVICE_ERROR;
            cudaFree(c->scratch);
            c->scratch = nullptr;
        }
        if (!ok(cudaMalloc(&c->scratch, kHeaderBytes + 16 * want))) {
            c->max_chunks = 0;
            return GBU_DEVICE_ERROR;
        }
        c->max_chunks = want;
        if (!ok(cudaMemset(c->scratch, 0, kHeaderBytes + 16 * want))) return GBU_DEVICE_ERROR;
        c->dirty = true;
    }
    if (c->dirty) {
        // chunks_done = exit = flags = done = 0, first-error word = ~0, epoch =
        // claim = 0, the validation kernel's first-error word = ~0, and no
        // status word may look ready
        static const uint64_t hdr[5] = {0, 0, ~0ull, 0, ~0ull};
        if (!ok(cudaMemcpyAsync(c->scratch, hdr, sizeof hdr, cudaMemcpyHostToDevice, stream)) ||
            !ok(cudaMemsetAsync(c->scratch + kHeaderBytes, 0, 8 * c->max_chunks, stream)))
            return GBU_DEVICE_ERROR;
        c->dirty = false;
    }
    return GBU_OK;
}

enum class Op { U8toU16, U16toU8, U8toU16BE, U16BEtoU8 };
bool utf16_in(Op op) { return op == Op::U16toU8 || op == Op::U16BEtoU8; }
bool big_endian(Op op) { return op == Op::U8toU16BE || op == Op::U16BEtoU8; }

// Enqueue one call; result goes to `dst` (device-visible). `validate`: the
// validation-only form (implies !write).
int32_t enqueue(gbu_ctx *c, Op op, const void *in, uint64_t n, void *out, uint64_t cap,
                bool write, ResultSlot *dst, cudaStream_t stream, bool validate = false)
{
    if (!c || !dst || (n && !in) || (write && cap && !out)) return GBU_INVALID_ARG;
    if (n >= kMaxUnits) return GBU_INVALID_ARG;
    if (utf16_in(op) && (reinterpret_cast<uintptr_t>(in) & 1u)) return GBU_INVALID_ARG;
    if (!utf16_in(op) && write && (reinterpret_cast<uintptr_t>(out) & 1u)) return GBU_INVALID_ARG;
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    if (n == 0) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return ok(launch_write_result(dst, GBU_OK, 0, 0, stream)) ? GBU_OK : GBU_DEVICE_ERROR;
    }
    const bool utf16 = utf16_in(op);
    const Variant &V = variant(shape_for(c, utf16 ? 2 * n : n));
    Job J{};
    J.item0 = V.make_item(in, n, utf16, out, cap, write, dst, 0, big_endian(op));
    J.num_items = 1;
    J.total_chunks = J.item0.nchunks;
    J.validate = validate ? 1u : 0u;
    if (J.total_chunks <= (uint32_t)c->tune.small_chunks && !c->skip_chunks) {
        // a few chunks: one cluster launch, no scratch
        const cudaError_t e = V.launch_small(J.item0, write, validate, stream);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return ok(e) ? GBU_OK : GBU_DEVICE_ERROR;
    }
    int32_t st = ensure_scratch(c, validate && !c->skip_chunks ? 1 : J.total_chunks, stream);
    if (st != GBU_OK) {
        c->dirty = true;
        return st;
    }
    if (validate && !c->skip_chunks) {
        // a validation needs no offsets: the streaming kernel (two launches)
        unsigned long long *err = reinterpret_cast<unsigned long long *>(c->scratch + kHdrValidErr);
        const cudaError_t e = launch_validate(in, n, utf16, big_endian(op), err, dst, stream);
        g_launches.fetch_add(2, std::memory_order_relaxed);
        if (!ok(e)) {
            c->dirty = true;
            return GBU_DEVICE_ERROR;
        }
        return GBU_OK;
    }
    attach_scratch(c, J);
    J.wait_ns = c->wait_ns;
    if (c->skip_chunks) {
        // failure-detection hook: the launch hands out chunks from here on
        const uint32_t from = c->skip_chunks;
        c->skip_chunks = 0;
        if (!ok(cudaMemcpyAsync(J.claim, &from, sizeof from, cudaMemcpyHostToDevice, stream)) ||
            !ok(cudaStreamSynchronize(stream)))
            return GBU_DEVICE_ERROR;
    }
    int grid = V.grid(c->device, c->tune);
    if (grid <= 0) return GBU_DEVICE_ERROR;
    if ((uint32_t)grid > J.total_chunks) grid = (int)J.total_chunks;
    const cudaError_t e =
        V.launch_job(J, write, grid, stream, c->tune.look, big_endian(op), utf16 ? 2 : 1);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!ok(e)) {
        c->dirty = true;
        return GBU_DEVICE_ERROR;
    }
    return GBU_OK;
}

gbu_result run_sync(gbu_ctx *c, Op op, const void *in, uint64_t n, void *out, uint64_t cap,
                    bool write, void *stream, bool validate = false)
{
    if (!c) return make(GBU_INVALID_ARG);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return make(GBU_OK, 0, 0);
    int32_t st = enqueue(c, op, in, n, out, cap, write,
                         reinterpret_cast<ResultSlot *>(c->d_result), s, validate);
    if (st != GBU_OK) return make(st);
    if (!ok(cudaStreamSynchronize(s))) {
        c->dirty = true;
        return make(GBU_DEVICE_ERROR);
    }
    gbu_result r;
    std::memcpy(&r, const_cast<const gbu_result *>(c->h_result), sizeof r);
    if (r.status == GBU_DEVICE_TIMEOUT || r.status == GBU_DEVICE_ERROR) c->dirty = true;
    return r;
}

}  // namespace

extern "C" {

gbu_ctx *gbu_create(int device)
{
    gbu_ctx *c = new (std::nothrow) gbu_ctx();
    if (!c) return nullptr;
    c->device = device;
    void *h = nullptr;
    if (!ok(cudaSetDevice(device)) ||
        !ok(cudaHostAlloc(&h, sizeof(gbu_result), cudaHostAllocMapped))) {
        delete c;
        return nullptr;
    }
    c->h_result = static_cast<gbu_result *>(h);
    std::memset(c->h_result, 0, sizeof(gbu_result));
    void *d = nullptr;
    if (!ok(cudaHostGetDevicePointer(&d, h, 0))) {
        cudaFreeHost(h);
        delete c;
        return nullptr;
    }
    c->d_result = static_cast<gbu_result *>(d);
    return c;
}

void gbu_destroy(gbu_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->d_items) cudaFree(c->d_items);
    if (c->h_items) cudaFreeHost(c->h_items);
    if (c->d_small) cudaFree(c->d_small);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->d_chunk_item) cudaFree(c->d_chunk_item);
    if (c->h_chunk_item) cudaFreeHost(c->h_chunk_item);
    if (c->d_item_err) cudaFree(c->d_item_err);
    if (c->d_item_done) cudaFree(c->d_item_done);
    if (c->scratch) cudaFree(c->scratch);
    if (c->scratch32) cudaFree(c->scratch32);
    if (c->io) cudaFree(c->io);
    for (int k = 0; k < 64; k++) {
        if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
        if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
    }
    if (c->h2d) cudaStreamDestroy(c->h2d);
    if (c->d2h) cudaStreamDestroy(c->d2h);
    if (c->h_slice_res) cudaFreeHost(c->h_slice_res);
    if (c->h_result) cudaFreeHost(c->h_result);
    delete c;
}

int32_t gbu_reserve(gbu_ctx *c, uint64_t max_input_bytes)
{
    if (!c) return GBU_INVALID_ARG;
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    const uint64_t cb = min_chunk_bytes();
    const uint64_t chunks = (max_input_bytes + 16 + cb - 1) / cb + 1;
    int32_t st = ensure_scratch(c, chunks, nullptr);
    if (st == GBU_OK && !ok(cudaDeviceSynchronize())) st = GBU_DEVICE_ERROR;
    return st;
}

gbu_result gbu_utf8_to_utf16le(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint16_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_sync(c, Op::U8toU16, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf16le_to_utf8(gbu_ctx *c, const uint16_t *d_in, uint64_t n, uint8_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_sync(c, Op::U16toU8, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf16_length_from_utf8(gbu_ctx *c, const uint8_t *d_in, uint64_t n, void *stream)
{
    return run_sync(c, Op::U8toU16, d_in, n, nullptr, 0, false, stream);
}

gbu_result gbu_validate_utf8(gbu_ctx *c, const uint8_t *d_in, uint64_t n, void *stream)
{
    return run_sync(c, Op::U8toU16, d_in, n, nullptr, 0, false, stream, true);
}

gbu_result gbu_validate_utf16le(gbu_ctx *c, const uint16_t *d_in, uint64_t n, void *stream)
{
    return run_sync(c, Op::U16toU8, d_in, n, nullptr, 0, false, stream, true);
}

int32_t gbu_validate_utf8_async(gbu_ctx *c, const uint8_t *d_in, uint64_t n, gbu_result *d_result,
                                void *stream)
{
    return enqueue(c, Op::U8toU16, d_in, n, nullptr, 0, false,
                   reinterpret_cast<ResultSlot *>(d_result), static_cast<cudaStream_t>(stream), true);
}

int32_t gbu_validate_utf16le_async(gbu_ctx *c, const uint16_t *d_in, uint64_t n,
                                   gbu_result *d_result, void *stream)
{
    return enqueue(c, Op::U16toU8, d_in, n, nullptr, 0, false,
                   reinterpret_cast<ResultSlot *>(d_result), static_cast<cudaStream_t>(stream), true);
}

gbu_result gbu_utf8_to_utf16be(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint16_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_sync(c, Op::U8toU16BE, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf16be_to_utf8(gbu_ctx *c, const uint16_t *d_in, uint64_t n, uint8_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_sync(c, Op::U16BEtoU8, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf8_length_from_utf16be(gbu_ctx *c, const uint16_t *d_in, uint64_t n,
                                        void *stream)
{
    return run_sync(c, Op::U16BEtoU8, d_in, n, nullptr, 0, false, stream);
}

gbu_result gbu_validate_utf16be(gbu_ctx *c, const uint16_t *d_in, uint64_t n, void *stream)
{
    return run_sync(c, Op::U16BEtoU8, d_in, n, nullptr, 0, false, stream, true);
}

int32_t gbu_utf8_to_utf16be_async(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint16_t *d_out,
                                  uint64_t cap, gbu_result *result, void *stream)
{
    return enqueue(c, Op::U8toU16BE, d_in, n, d_out, cap, true,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

int32_t gbu_utf16be_to_utf8_async(gbu_ctx *c, const uint16_t *d_in, uint64_t n, uint8_t *d_out,
                                  uint64_t cap, gbu_result *result, void *stream)
{
    return enqueue(c, Op::U16BEtoU8, d_in, n, d_out, cap, true,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

gbu_result gbu_utf8_length_from_utf16le(gbu_ctx *c, const uint16_t *d_in, uint64_t n,
                                        void *stream)
{
    return run_sync(c, Op::U16toU8, d_in, n, nullptr, 0, false, stream);
}

int32_t gbu_utf8_to_utf16le_async(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint16_t *d_out,
                                  uint64_t cap, gbu_result *result, void *stream)
{
    return enqueue(c, Op::U8toU16, d_in, n, d_out, cap, true,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

int32_t gbu_utf16le_to_utf8_async(gbu_ctx *c, const uint16_t *d_in, uint64_t n, uint8_t *d_out,
                                  uint64_t cap, gbu_result *result, void *stream)
{
    return enqueue(c, Op::U16toU8, d_in, n, d_out, cap, true,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

int32_t gbu_utf16_length_from_utf8_async(gbu_ctx *c, const uint8_t *d_in, uint64_t n,
                                         gbu_result *result, void *stream)
{
    return enqueue(c, Op::U8toU16, d_in, n, nullptr, 0, false,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

int32_t gbu_utf8_length_from_utf16le_async(gbu_ctx *c, const uint16_t *d_in, uint64_t n,
                                           gbu_result *result, void *stream)
{
    return enqueue(c, Op::U16toU8, d_in, n, nullptr, 0, false,
                   reinterpret_cast<ResultSlot *>(result), static_cast<cudaStream_t>(stream));
}

// Host-buffer form. Inputs of a few slices or more are cut at character
// boundaries into slices that are copied in, transcoded and copied out in a
// pipeline (copy-in on one stream, kernels on the caller's stream, copy-out
// on a third), so both copy directions and the kernels overlap. Each slice is
// an independent call; the results are joined on the host in order: the
// first slice with an encoding error ends the input (offset and valid prefix
// shifted by the slices before it), and a total above the capacity is
// OUTPUT_TOO_SMALL with the required length, as for the one-call form.
// ---- UTF-32LE ------------------------------------------------------------------

static bool ensure_scratch32(gbu_ctx *c, size_t bytes, cudaStream_t s)
{
    if (bytes <= c->scratch32_bytes) return true;
    if (!ok(cudaStreamSynchronize(s)) || !ok(cudaDeviceSynchronize())) return false;
    if (c->scratch32) cudaFree(c->scratch32);
    c->scratch32 = nullptr;
    c->scratch32_bytes = 0;
    if (!ok(cudaMalloc(&c->scratch32, bytes))) return false;
    c->scratch32_bytes = bytes;
    return true;
}

static gbu_result finish32(gbu_ctx *c, cudaStream_t s)
{
    if (!ok(cudaStreamSynchronize(s))) return make(GBU_DEVICE_ERROR);
    gbu_result r;
    std::memcpy(&r, const_cast<const gbu_result *>(c->h_result), sizeof r);
    return r;
}

static gbu_result run_utf32_in(gbu_ctx *c, const uint32_t *d_in, uint64_t n, uint8_t *d_out,
                               uint64_t cap, bool write, void *stream)
{
    if (!c || (n && !d_in) || (write && cap && !d_out)) return make(GBU_INVALID_ARG);
    if (reinterpret_cast<uintptr_t>(d_in) & 3u) return make(GBU_INVALID_ARG);
    if (n >= kMaxUnits) return make(GBU_INVALID_ARG);
    if (n == 0) return make(GBU_OK, 0, 0);
    if (!ok(cudaSetDevice(c->device))) return make(GBU_DEVICE_ERROR);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t ntiles = utf32_tiles(d_in, n);
    if (!ensure_scratch32(c, utf32_scratch_bytes(ntiles), s)) return make(GBU_DEVICE_ERROR);
    if (!ok(launch_utf32_to_utf8(d_in, n, d_out, write ? cap : ~0ull, write, c->scratch32,
                                 reinterpret_cast<ResultSlot *>(c->d_result), s)))
        return make(GBU_DEVICE_ERROR);
    return finish32(c, s);
}

static gbu_result run_utf8_to_32(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint32_t *d_out,
                                 uint64_t cap, bool write, void *stream)
{
    if (!c || (n && !d_in) || (write && cap && !d_out)) return make(GBU_INVALID_ARG);
    if (write && (reinterpret_cast<uintptr_t>(d_out) & 3u)) return make(GBU_INVALID_ARG);
    if (n == 0) return make(GBU_OK, 0, 0);
    // the UTF-8 rules of Sec. 6.4, by the UTF-8 kernel (validation only)
    const gbu_result v = run_sync(c, Op::U8toU16, d_in, n, nullptr, 0, false, stream, true);
    if (v.status >= GBU_INVALID_ARG) return v;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t p = v.status == GBU_OK ? n : v.in_offset;   // the valid prefix
    const uint64_t ntiles = utf8_tiles(d_in, p);
    if (!ensure_scratch32(c, utf32_scratch_bytes(ntiles), s)) return make(GBU_DEVICE_ERROR);
    if (!ok(launch_utf8_to_utf32(d_in, n, p, v.status, v.in_offset, d_out, write ? cap : ~0ull,
                                 write, c->scratch32, reinterpret_cast<ResultSlot *>(c->d_result),
                                 s)))
        return make(GBU_DEVICE_ERROR);
    return finish32(c, s);
}

extern "C" {

gbu_result gbu_utf32le_to_utf8(gbu_ctx *c, const uint32_t *d_in, uint64_t n, uint8_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_utf32_in(c, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf8_length_from_utf32le(gbu_ctx *c, const uint32_t *d_in, uint64_t n, void *stream)
{
    return run_utf32_in(c, d_in, n, nullptr, 0, false, stream);
}

gbu_result gbu_validate_utf32le(gbu_ctx *c, const uint32_t *d_in, uint64_t n, void *stream)
{
    gbu_result r = run_utf32_in(c, d_in, n, nullptr, 0, false, stream);
    if (r.status < GBU_INVALID_ARG) r.out_len = 0;
    return r;
}

gbu_result gbu_utf8_to_utf32le(gbu_ctx *c, const uint8_t *d_in, uint64_t n, uint32_t *d_out,
                               uint64_t cap, void *stream)
{
    return run_utf8_to_32(c, d_in, n, d_out, cap, true, stream);
}

gbu_result gbu_utf32_length_from_utf8(gbu_ctx *c, const uint8_t *d_in, uint64_t n, void *stream)
{
    return run_utf8_to_32(c, d_in, n, nullptr, 0, false, stream);
}

}  // extern "C"

static constexpr int kMaxSlices = 64;
static constexpr uint64_t kMinSliceBytes = 32ull << 20;

static bool host_pipeline_ready(gbu_ctx *c)
{
    if (!c->h2d && !ok(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking))) return false;
    if (!c->d2h && !ok(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking))) return false;
    for (int k = 0; k < kMaxSlices; k++) {
        if (!c->ev_in[k] && !ok(cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming)))
            return false;
        if (!c->ev_done[k] && !ok(cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming)))
            return false;
    }
    if (!c->h_slice_res) {
        void *h = nullptr, *d = nullptr;
        if (!ok(cudaHostAlloc(&h, kMaxSlices * sizeof(gbu_result), cudaHostAllocMapped)) ||
            !ok(cudaHostGetDevicePointer(&d, h, 0)))
            return false;
        c->h_slice_res = static_cast<gbu_result *>(h);
        c->d_slice_res = static_cast<gbu_result *>(d);
    }
    return true;
}

static gbu_result run_host(gbu_ctx *c, Op op, const void *h_in, uint64_t n, void *h_out,
                           uint64_t cap, void *stream)
{
    if (!c || (n && !h_in) || (cap && !h_out)) return make(GBU_INVALID_ARG);
    if (n == 0) return make(GBU_OK, 0, 0);
    if (n >= kMaxUnits) return make(GBU_INVALID_ARG);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!ok(cudaSetDevice(c->device))) return make(GBU_DEVICE_ERROR);
    const bool u16 = utf16_in(op);
    const uint64_t uin = u16 ? 2 : 1;                 // input unit bytes
    const uint64_t ub = u16 ? 1 : 2;                  // output unit bytes
    const uint64_t per_unit = u16 ? 3 : 1;            // worst-case output units per input unit
    const uint64_t in_bytes = n * uin;
    // slice cut points (input units), each at a character boundary
    uint64_t cuts[kMaxSlices + 1];
    int ns = (int)std::min<uint64_t>(kMaxSlices, std::max<uint64_t>(1, in_bytes / kMinSliceBytes));
    const uint8_t *hb = static_cast<const uint8_t *>(h_in);
    cuts[0] = 0;
    for (int k = 1; k < ns; k++) {
        uint64_t cu = std::max(cuts[k - 1], n * k / ns);
        if (u16) {
            const uint16_t *hw = static_cast<const uint16_t *>(h_in);
            if (cu < n && (hw[cu] & 0xFC00u) == 0xDC00u) cu++;        // not between a pair
        } else {
            for (int t = 0; t < 3 && cu < n && (hb[cu] & 0xC0u) == 0x80u; t++) cu++;
        }
        cuts[k] = std::min(cu, n);
    }
    cuts[ns] = n;
    // device staging: the input, then each slice's worst-case output
    const uint64_t in_al = (in_bytes + 255) & ~uint64_t(255);
    uint64_t out_base[kMaxSlices + 1];
    out_base[0] = in_al;
    for (int k = 0; k < ns; k++)
        out_base[k + 1] = out_base[k] + (((cuts[k + 1] - cuts[k]) * per_unit * ub + 255) & ~uint64_t(255));
    const uint64_t need = out_base[ns] + 16;
    if (need > c->io_bytes) {
        if (!ok(cudaStreamSynchronize(s)) || !ok(cudaDeviceSynchronize())) return make(GBU_DEVICE_ERROR);
        if (c->io) cudaFree(c->io);
        c->io = nullptr;
        c->io_bytes = 0;
        if (!ok(cudaMalloc(&c->io, need))) return make(GBU_DEVICE_ERROR);
        c->io_bytes = need;
    }
    if (ns == 1) {   // one slice: copy in, transcode, copy out
        uint8_t *d_in = c->io, *d_out = c->io + in_al;
        if (!ok(cudaMemcpyAsync(d_in, h_in, in_bytes, cudaMemcpyHostToDevice, s)))
            return make(GBU_DEVICE_ERROR);
        gbu_result r = run_sync(c, op, d_in, n, d_out, cap, true, stream);
        if (r.status >= GBU_INVALID_ARG) return r;
        const uint64_t keep = r.out_len < cap ? r.out_len : cap;
        if (keep) {
            if (!ok(cudaMemcpyAsync(h_out, d_out, keep * ub, cudaMemcpyDeviceToHost, s)) ||
                !ok(cudaStreamSynchronize(s)))
                return make(GBU_DEVICE_ERROR);
        }
        return r;
    }
    if (!host_pipeline_ready(c)) return make(GBU_DEVICE_ERROR);
    // scratch for the largest slice, before anything is enqueued
    uint64_t max_units = 0;
    for (int k = 0; k < ns; k++) max_units = std::max(max_units, cuts[k + 1] - cuts[k]);
    const uint64_t cb = min_chunk_bytes();
    if (ensure_scratch(c, (16 + max_units * uin + cb - 1) / cb + 1, s) != GBU_OK)
        return make(GBU_DEVICE_ERROR);
    if (!ok(cudaStreamSynchronize(s))) return make(GBU_DEVICE_ERROR);
    // Every return below first waits for all three streams: no copy may
    // still read the caller's input or write its output after the call.
    auto drain = [&]() {
        cudaStreamSynchronize(c->h2d);
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(c->d2h);
    };
    // copy-in and kernels for every slice
    for (int k = 0; k < ns; k++) {
        const uint64_t u0 = cuts[k], nu = cuts[k + 1] - cuts[k];
        if (!ok(cudaMemcpyAsync(c->io + u0 * uin, hb + u0 * uin, nu * uin, cudaMemcpyHostToDevice,
                                c->h2d)) ||
            !ok(cudaEventRecord(c->ev_in[k], c->h2d)) || !ok(cudaStreamWaitEvent(s, c->ev_in[k], 0))) {
            drain();
            return make(GBU_DEVICE_ERROR);
        }
        const int32_t st = enqueue(c, op, c->io + u0 * uin, nu, c->io + out_base[k], nu * per_unit,
                                   true, reinterpret_cast<ResultSlot *>(c->d_slice_res + k), s);
        if (st != GBU_OK || !ok(cudaEventRecord(c->ev_done[k], s))) {
            drain();
            return make(st != GBU_OK ? st : GBU_DEVICE_ERROR);
        }
    }
    // join the results in order; copy each slice's output out as it finishes
    uint64_t out_off = 0;
    gbu_result total = make(GBU_OK, n, 0);
    for (int k = 0; k < ns; k++) {
        if (!ok(cudaEventSynchronize(c->ev_done[k]))) {
            drain();
            return make(GBU_DEVICE_ERROR);
        }
        gbu_result r;
        std::memcpy(&r, const_cast<const gbu_result *>(c->h_slice_res + k), sizeof r);
        if (r.status >= GBU_INVALID_ARG) {
            drain();
            if (r.status == GBU_DEVICE_TIMEOUT || r.status == GBU_DEVICE_ERROR) c->dirty = true;
            return r;
        }
        const uint64_t keep = out_off < cap ? std::min<uint64_t>(r.out_len, cap - out_off) : 0;
        if (keep && !ok(cudaMemcpyAsync(static_cast<uint8_t *>(h_out) + out_off * ub,
                                        c->io + out_base[k], keep * ub, cudaMemcpyDeviceToHost,
                                        c->d2h))) {
            drain();
            return make(GBU_DEVICE_ERROR);
        }
        if (r.status != GBU_OK) {   // an encoding error ends the input
            total = make(r.status, cuts[k] + r.in_offset, out_off + r.out_len);
            break;
        }
        out_off += r.out_len;
        total.out_len = out_off;
    }
    if (!ok(cudaStreamSynchronize(c->h2d)) || !ok(cudaStreamSynchronize(s)) ||
        !ok(cudaStreamSynchronize(c->d2h)))
        return make(GBU_DEVICE_ERROR);
    if (total.status == GBU_OK && total.out_len > cap) total.status = GBU_OUTPUT_TOO_SMALL;
    return total;
}

gbu_result gbu_utf8_to_utf16le_host(gbu_ctx *c, const uint8_t *h_in, uint64_t n, uint16_t *h_out,
                                    uint64_t cap, void *stream)
{
    return run_host(c, Op::U8toU16, h_in, n, h_out, cap, stream);
}

gbu_result gbu_utf16le_to_utf8_host(gbu_ctx *c, const uint16_t *h_in, uint64_t n, uint8_t *h_out,
                                    uint64_t cap, void *stream)
{
    return run_host(c, Op::U16toU8, h_in, n, h_out, cap, stream);
}

// ---- batches -----------------------------------------------------------------

static bool grow_batch(gbu_ctx *c, uint64_t items, uint64_t chunks)
{
    if (items > c->items_cap) {
        uint64_t want = c->items_cap ? c->items_cap : 64;
        while (want < items) want *= 2;
        if (c->d_items) cudaFree(c->d_items);
        if (c->h_items) cudaFreeHost(c->h_items);
        if (c->d_small) cudaFree(c->d_small);
        if (c->h_small) cudaFreeHost(c->h_small);
        if (c->d_item_err) cudaFree(c->d_item_err);
        if (c->d_item_done) cudaFree(c->d_item_done);
        c->d_items = nullptr; c->h_items = nullptr; c->d_item_err = nullptr; c->d_item_done = nullptr;
        c->d_small = nullptr; c->h_small = nullptr;
        c->items_cap = 0;
        if (!ok(cudaMalloc(&c->d_items, want * sizeof(Item))) ||
            !ok(cudaHostAlloc(&c->h_items, want * sizeof(Item), cudaHostAllocDefault)) ||
            !ok(cudaMalloc(&c->d_small, want * sizeof(Item))) ||
            !ok(cudaHostAlloc(&c->h_small, want * sizeof(Item), cudaHostAllocDefault)) ||
            !ok(cudaMalloc(&c->d_item_err, want * 8)) || !ok(cudaMalloc(&c->d_item_done, want * 4)))
            return false;
        c->items_cap = want;
    }
    if (chunks > c->chunk_map_cap) {
        uint64_t want = c->chunk_map_cap ? c->chunk_map_cap : 1024;
        while (want < chunks) want *= 2;
        if (c->d_chunk_item) cudaFree(c->d_chunk_item);
        if (c->h_chunk_item) cudaFreeHost(c->h_chunk_item);
        c->d_chunk_item = nullptr; c->h_chunk_item = nullptr;
        c->chunk_map_cap = 0;
        if (!ok(cudaMalloc(&c->d_chunk_item, want * 4)) ||
            !ok(cudaHostAlloc(&c->h_chunk_item, want * 4, cudaHostAllocDefault)))
            return false;
        c->chunk_map_cap = want;
    }
    return true;
}

}  // extern "C"

// A large batch (at least kSpreadBytes of input) runs its one-chunk items in
// a kernel of their own and the rest as one persistent job per input
// encoding, each on the kernel with that direction's code only (+3 % on
// 50,000 log-uniform strings); a smaller one (a served batch, say) runs as
// one persistent job, since every extra launch adds to its latency.
constexpr uint64_t kSpreadBytes = 512ull << 20;

// Count the chunks of the context's batch for its kernel shape (the pinned
// one, else the default), number them operation by operation, and copy the
// descriptors to the device. The caller has validated the items.
static int32_t plan_batch(gbu_ctx *c, cudaStream_t s)
{
    const gbu_batch_item *items = c->batch_src.data();
    const uint32_t count = (uint32_t)c->batch_src.size();
    const int vi = c->tune.variant >= 0 ? c->tune.variant : 0;
    const Variant &V = variant(vi);
    uint64_t chunks = 0;
    bool any_write = false, any_be = false;
    uint64_t in_bytes = 0;
    for (uint32_t i = 0; i < count; i++) {
        const gbu_batch_item &b = items[i];
        in_bytes += op_utf16_in(b.op) ? 2 * b.n : b.n;
    }
    const bool spread = in_bytes >= kSpreadBytes;
    for (uint32_t i = 0; i < count; i++) {
        const gbu_batch_item &b = items[i];
        any_write |= op_writes(b.op);
        any_be |= op_big_endian(b.op);
        const uint64_t k = chunks_of(V, b.in, b.n, op_utf16_in(b.op));
        if (k > 1 || !spread) chunks += k;   // one-chunk items run apart
    }
    c->batch_items = 0;
    if (chunks >= (1ull << 31)) return GBU_INVALID_ARG;   // the claim counter may run past the end
    if (!ok(cudaStreamSynchronize(s))) return GBU_DEVICE_ERROR;   // host staging is reused
    if (!grow_batch(c, count ? count : 1, chunks ? chunks : 1)) return GBU_DEVICE_ERROR;
    // Chunks are numbered operation by operation (items keep their index and
    // result slot): a CTA then mostly runs one code path at a time, which
    // keeps the instruction cache warm. In a large batch the UTF-8-input and
    // UTF-16-input items form two jobs, each numbered from 0.
    uint32_t base = 0;
    // Within an operation, items with more chunks first: the last chunks
    // handed out are then the shortest of the persistent job's items (+3 %
    // on 50,000 log-uniform strings against the callers' order). One-chunk
    // items go to the one-CTA-per-item kernel instead: in the persistent
    // job each would pay a chunk iteration's fixed costs (claim, descriptor
    // loads, TMA hand-off, barriers, deferred write-out) for a few bytes.
    std::vector<uint32_t> order(count);
    std::vector<uint64_t> nch(count);
    for (uint32_t i = 0; i < count; i++) {
        order[i] = i;
        nch[i] = chunks_of(V, items[i].in, items[i].n, op_utf16_in(items[i].op));
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return nch[a] > nch[b]; });
    uint32_t nsmall = 0, pos = 0;   // pos: next entry of the chunk -> item map
    const int ngrp = spread ? 2 : 1;
    for (int g = 0; g < ngrp; g++) {
        c->grp_start[g] = pos;
        base = 0;   // each job numbers its chunks from 0
        bool g8 = false, g16 = false, gbe = false, gw = false;
        for (int op = GBU_OP_UTF8_TO_UTF16LE; op <= GBU_OP_UTF8_LENGTH_FROM_UTF16BE; op++) {
            if (spread && (op_utf16_in(op) ? 1 : 0) != g) continue;
            for (const uint32_t i : order) {
                const gbu_batch_item &b = items[i];
                if (b.op != op) continue;
                const bool big = nch[i] > 1 || !spread;
                Item I = V.make_item(b.in, b.n, op_utf16_in(b.op), b.out, b.cap, op_writes(b.op),
                                     reinterpret_cast<ResultSlot *>(c->batch_results + i),
                                     big ? base : 0, op_big_endian(b.op));
                c->h_items[i] = I;
                if (!big) {
                    c->h_small[nsmall++] = I;
                    continue;
                }
                (op_utf16_in(b.op) ? g16 : g8) = true;
                gbe |= op_big_endian(b.op);
                gw |= op_writes(b.op);
                for (uint32_t k = 0; k < I.nchunks; k++) c->h_chunk_item[pos + k] = i;
                base += I.nchunks;
                pos += I.nchunks;
            }
        }
        c->grp_chunks[g] = base;
        c->grp_in[g] = g8 && !g16 ? 1 : (g16 && !g8 ? 2 : 0);
        c->grp_be[g] = gbe;
        c->grp_write[g] = gw;
    }
    for (int g = ngrp; g < 2; g++) c->grp_chunks[g] = 0;
    int32_t st = ensure_scratch(c, chunks ? chunks : 1, s);
    if (st != GBU_OK) return st;
    if (count) {
        if (!ok(cudaMemcpyAsync(c->d_items, c->h_items, count * sizeof(Item), cudaMemcpyHostToDevice, s)) ||
            (nsmall && !ok(cudaMemcpyAsync(c->d_small, c->h_small, nsmall * sizeof(Item),
                                           cudaMemcpyHostToDevice, s))) ||
            (chunks && !ok(cudaMemcpyAsync(c->d_chunk_item, c->h_chunk_item, chunks * 4,
                                           cudaMemcpyHostToDevice, s))) ||
            !ok(cudaMemsetAsync(c->d_item_err, 0xFF, (size_t)count * 8, s)) ||
            !ok(cudaMemsetAsync(c->d_item_done, 0, (size_t)count * 4, s)) ||
            !ok(cudaStreamSynchronize(s)))
            return GBU_DEVICE_ERROR;
    }
    c->batch_items = count;
    c->batch_chunks = (uint32_t)chunks;
    c->batch_small = nsmall;
    c->batch_write = any_write;
    c->batch_be = any_be;
    c->batch_variant = vi;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return GBU_OK;
}

// The planned batch counted for the context's current kernel shape.
static int32_t plan_current(gbu_ctx *c, cudaStream_t s)
{
    const int vi = c->tune.variant >= 0 ? c->tune.variant : 0;
    if (c->batch_src.empty() || c->batch_variant == vi) return GBU_OK;
    return plan_batch(c, s);
}

extern "C" {

int32_t gbu_batch_plan(gbu_ctx *c, const gbu_batch_item *items, uint32_t count,
                       gbu_result *results, void *stream)
{
    if (!c || (count && (!items || !results))) return GBU_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    for (uint32_t i = 0; i < count; i++) {
        const gbu_batch_item &b = items[i];
        if (b.op < GBU_OP_UTF8_TO_UTF16LE || b.op > GBU_OP_UTF8_LENGTH_FROM_UTF16BE)
            return GBU_INVALID_ARG;
        const bool utf16 = op_utf16_in(b.op);
        const bool write = op_writes(b.op);
        if (b.n >= kMaxUnits || (b.n && !b.in)) return GBU_INVALID_ARG;
        if (utf16 && (reinterpret_cast<uintptr_t>(b.in) & 1u)) return GBU_INVALID_ARG;
        if (write && b.cap && !b.out) return GBU_INVALID_ARG;
        if (write && !utf16 && (reinterpret_cast<uintptr_t>(b.out) & 1u)) return GBU_INVALID_ARG;
    }
    c->batch_src.assign(items, items + count);
    c->batch_results = results;
    return plan_batch(c, s);
}

// Enqueue the planned batch; `counted`: a real launch (not a graph capture).
static int32_t batch_enqueue(gbu_ctx *c, cudaStream_t s, bool counted = true)
{
    if (c->batch_items == 0) return GBU_OK;
    const Variant &V = variant(c->batch_variant);
    if (c->batch_small) {
        const cudaError_t e =
            V.launch_small_items(c->d_small, c->batch_small, c->batch_write, c->batch_be, s);
        if (counted) g_launches.fetch_add(1, std::memory_order_relaxed);
        if (!ok(e)) return GBU_DEVICE_ERROR;
    }
    for (int g = 0; g < 2; g++) {
        if (c->grp_chunks[g] == 0) continue;
        Job J{};
        J.items = c->d_items;
        J.chunk_item = c->d_chunk_item + c->grp_start[g];
        J.num_items = c->batch_items;
        J.total_chunks = c->grp_chunks[g];
        attach_scratch(c, J);
        J.item_err = c->d_item_err;
        J.item_done = c->d_item_done;
        J.wait_ns = c->wait_ns;
        int grid = V.grid(c->device, c->tune);
        if (grid <= 0) return GBU_DEVICE_ERROR;
        if ((uint32_t)grid > J.total_chunks) grid = (int)J.total_chunks;
        const cudaError_t e = V.launch_job(J, c->grp_write[g], grid, s, c->tune.look,
                                           c->grp_be[g], c->grp_in[g]);
        if (counted) g_launches.fetch_add(1, std::memory_order_relaxed);
        if (!ok(e)) return GBU_DEVICE_ERROR;
    }
    return GBU_OK;
}

int32_t gbu_batch_launch(gbu_ctx *c, void *stream)
{
    if (!c) return GBU_INVALID_ARG;
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan_current(c, s) != GBU_OK) return GBU_DEVICE_ERROR;
    if (c->dirty && ensure_scratch(c, c->batch_chunks ? c->batch_chunks : 1, s) != GBU_OK)
        return GBU_DEVICE_ERROR;
    return batch_enqueue(c, s);
}

int32_t gbu_batch_launch_graph(gbu_ctx *c, void *stream)
{
    if (!c) return GBU_INVALID_ARG;
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan_current(c, s) != GBU_OK) return GBU_DEVICE_ERROR;
    if (c->batch_items == 0) return GBU_OK;
    if (c->dirty && ensure_scratch(c, c->batch_chunks, s) != GBU_OK) return GBU_DEVICE_ERROR;
    if (!c->graph) {
        if (!c->capture_stream &&
            !ok(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)))
            return GBU_DEVICE_ERROR;
        // kernel attributes are set before the capture
        if (variant(c->batch_variant).grid(c->device, Tune{}) <= 0) return GBU_DEVICE_ERROR;
        cudaGraph_t g = nullptr;
        if (!ok(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal)))
            return GBU_DEVICE_ERROR;
        const int32_t st = batch_enqueue(c, c->capture_stream, false);
        const cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
        if (st != GBU_OK || !ok(e) || !g) {
            if (g) cudaGraphDestroy(g);
            return GBU_DEVICE_ERROR;
        }
        const cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (!ok(ie)) {
            c->graph = nullptr;
            return GBU_DEVICE_ERROR;
        }
    }
    if (!ok(cudaGraphLaunch(c->graph, s))) return GBU_DEVICE_ERROR;
    // the graph holds the one-chunk items' kernel and the persistent kernel (either may be absent)
    g_launches.fetch_add((c->batch_small ? 1 : 0) + (c->grp_chunks[0] ? 1 : 0) +
                             (c->grp_chunks[1] ? 1 : 0),
                         std::memory_order_relaxed);
    return GBU_OK;
}

int32_t gbu_set_wait_limit(gbu_ctx *c, uint64_t ns)
{
    if (!c || ns > 60ull * 1000000000ull) return GBU_INVALID_ARG;
    c->wait_ns = ns;
    if (c->graph) {   // the captured launch has the old limit
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return GBU_OK;
}

int32_t gbu_test_skip_chunks(gbu_ctx *c, uint32_t first_chunk)
{
    if (!c) return GBU_INVALID_ARG;
    c->skip_chunks = first_chunk;
    return GBU_OK;
}

int32_t gbu_get_tune(gbu_ctx *c, gbu_tune *t)
{
    if (!c || !t) return GBU_INVALID_ARG;
    t->look_width = c->tune.look;
    t->ctas_per_sm = c->tune.ctas_per_sm;
    t->small_chunks = c->tune.small_chunks;
    const bool pinned = c->tune.variant >= 0;
    t->chunk_bytes = pinned ? (int32_t)variant(c->tune.variant).chunk_bytes : 0;
    t->compute_threads = pinned ? variant(c->tune.variant).threads : 0;
    return GBU_OK;
}

int32_t gbu_set_tune(gbu_ctx *c, const gbu_tune *t)
{
    if (!c || !t) return GBU_INVALID_ARG;
    bool known = false;
    for (const int w : kLookWidths) known |= w == t->look_width;
    if (!known || t->ctas_per_sm < 0 || t->small_chunks < 0 || t->small_chunks > kSmallMaxChunks)
        return GBU_INVALID_ARG;
    int vi = -1;
    if (t->chunk_bytes != 0 || t->compute_threads != 0) {
        vi = variant_index(t->compute_threads, (uint32_t)t->chunk_bytes);
        if (vi < 0) return GBU_INVALID_ARG;
    }
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    // CTAs per SM: at most what the pinned shape (every shape, when none is
    // pinned) fits; shapes that fit fewer use as many as fit
    int per = 0;
    for (int i = 0; i < kVariants; i++) {
        if (vi >= 0 && i != vi) continue;
        const int p = variant(i).max_ctas_per_sm(c->device);
        if (p <= 0) return GBU_DEVICE_ERROR;
        per = std::max(per, p);
    }
    if (t->ctas_per_sm > per) return GBU_INVALID_ARG;
    c->tune.small_chunks = t->small_chunks;   // single-buffer calls only: no graph holds it
    if (c->tune.look != t->look_width || c->tune.ctas_per_sm != t->ctas_per_sm ||
        c->tune.variant != vi) {
        c->tune.look = t->look_width;
        c->tune.ctas_per_sm = t->ctas_per_sm;
        c->tune.variant = vi;   // a planned batch is counted again at its next launch
        if (c->graph) {   // the captured launch has the old parameters
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
    }
    return GBU_OK;
}

int32_t gbu_call_shape(gbu_ctx *c, uint64_t input_bytes, gbu_tune *t)
{
    if (!c || !t) return GBU_INVALID_ARG;
    const int vi = shape_for(c, input_bytes);
    t->look_width = c->tune.look;
    t->ctas_per_sm = c->tune.ctas_per_sm;
    t->small_chunks = c->tune.small_chunks;
    t->chunk_bytes = (int32_t)variant(vi).chunk_bytes;
    t->compute_threads = variant(vi).threads;
    return GBU_OK;
}

int32_t gbu_tune_shapes(gbu_tune *shapes, int32_t max_shapes)
{
    if (max_shapes < 0 || (max_shapes && !shapes)) return GBU_INVALID_ARG;
    for (int i = 0; i < kVariants && i < max_shapes; i++) {
        gbu_tune t{};
        t.look_width = GBU_DEFAULT_LOOK;
        t.ctas_per_sm = 0;
        t.small_chunks = kSmallMaxChunks;
        t.chunk_bytes = (int32_t)variant(i).chunk_bytes;
        t.compute_threads = variant(i).threads;
        shapes[i] = t;
    }
    return kVariants;
}

}  // extern "C"

namespace {

// Cache key of a planned batch on this device: the device, and the batch's
// shape in coarse buckets (item count and input bytes by powers of two, the
// UTF-16 and writing shares by tenths).
std::string tune_key(gbu_ctx *c)
{
    cudaDeviceProp prop{};
    if (!ok(cudaGetDeviceProperties(&prop, c->device))) return std::string();
    uint64_t bytes = 0;
    uint32_t u16 = 0, wr = 0;
    for (uint32_t i = 0; i < c->batch_items; i++) {
        const Item &I = c->h_items[i];
        const bool is16 = (I.op & kOpUtf16) != 0;
        bytes += I.n * (is16 ? 2 : 1);
        u16 += is16;
        wr += (I.op & kOpWrite) != 0;
    }
    char buf[384];
    std::string name(prop.name);
    std::replace(name.begin(), name.end(), ' ', '_');
    const int items_b = (int)std::floor(std::log2((double)c->batch_items + 1));
    const int bytes_b = (int)std::floor(std::log2((double)bytes + 1));
    std::snprintf(buf, sizeof buf, "%s/sm%d/items2^%d/bytes2^%d/u16_%d/write_%d", name.c_str(),
                  prop.multiProcessorCount, items_b, bytes_b,
                  (int)(10.0 * u16 / c->batch_items + 0.5), (int)(10.0 * wr / c->batch_items + 0.5));
    return std::string(buf);
}

bool tune_lookup(const char *path, const std::string &key, gbu::Tune *t)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512], k[400];
    int look = 0, ctas = 0, chunk = 0, threads = 0;
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        if (std::sscanf(line, "%399s %d %d %d %d", k, &look, &ctas, &chunk, &threads) == 5 &&
            key == k) {
            const int vi = variant_index(threads, (uint32_t)chunk);
            if (vi < 0) continue;
            t->look = look;   // the last entry for a key wins
            t->ctas_per_sm = ctas;
            t->variant = vi;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

}  // namespace

extern "C" {

int32_t gbu_batch_autotune(gbu_ctx *c, void *stream, const char *cache_path, gbu_tune *chosen)
{
    if (!c) return GBU_INVALID_ARG;
    if (!ok(cudaSetDevice(c->device))) return GBU_DEVICE_ERROR;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto report = [&]() {
        if (chosen) gbu_get_tune(c, chosen);
        return GBU_OK;
    };
    if (c->batch_src.empty()) return report();
    if (plan_current(c, s) != GBU_OK) return GBU_DEVICE_ERROR;
    const std::string key = tune_key(c);
    if (key.empty()) return GBU_DEVICE_ERROR;
    auto apply = [&](const gbu::Tune &b) {
        const Variant &V = variant(b.variant);
        gbu_tune t{b.look, b.ctas_per_sm, c->tune.small_chunks, (int32_t)V.chunk_bytes, V.threads};
        int32_t st = gbu_set_tune(c, &t);
        if (st == GBU_OK) st = plan_current(c, s);   // count the chunks for the shape now
        return st;
    };
    gbu::Tune cached;
    if (cache_path && tune_lookup(cache_path, key, &cached) && apply(cached) == GBU_OK)
        return report();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!ok(cudaEventCreate(&e0)) || !ok(cudaEventCreate(&e1))) return GBU_DEVICE_ERROR;
    const gbu::Tune saved = c->tune;
    gbu::Tune best = c->tune;
    float best_ms = 1e30f;
    int32_t st = GBU_OK;
    constexpr int kReps = 3;
    // every shape (the batch counted again for each), look-back width and
    // resident CTAs per SM
    for (int vi = 0; vi < kVariants && st == GBU_OK; vi++) {
        const int per = variant(vi).max_ctas_per_sm(c->device);
        c->tune.variant = vi;
        if (per <= 0 || (st = plan_current(c, s)) != GBU_OK ||
            (c->dirty && ensure_scratch(c, c->batch_chunks, s) != GBU_OK)) {
            if (st == GBU_OK) st = GBU_DEVICE_ERROR;
            break;
        }
        for (const int look : kLookWidths) {
            for (int ctas = 1; ctas <= per && st == GBU_OK; ctas++) {
                c->tune.look = look;
                c->tune.ctas_per_sm = ctas;
                st = batch_enqueue(c, s);   // warm-up
                std::vector<float> ms;
                for (int r = 0; r < kReps && st == GBU_OK; r++) {
                    float t = 0;
                    if (!ok(cudaEventRecord(e0, s)) || (st = batch_enqueue(c, s)) != GBU_OK ||
                        !ok(cudaEventRecord(e1, s)) || !ok(cudaEventSynchronize(e1)) ||
                        !ok(cudaEventElapsedTime(&t, e0, e1))) {
                        if (st == GBU_OK) st = GBU_DEVICE_ERROR;
                        break;
                    }
                    ms.push_back(t);
                }
                if (st != GBU_OK) break;
                std::sort(ms.begin(), ms.end());
                if (ms[kReps / 2] < best_ms) {
                    best_ms = ms[kReps / 2];
                    best = c->tune;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune = saved;
    if (st != GBU_OK) {
        plan_current(c, s);
        return st;
    }
    st = apply(best);
    if (st != GBU_OK) return st;
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "a")) {
            const Variant &V = variant(best.variant);
            std::fprintf(f, "%s %d %d %u %d %.4f\n", key.c_str(), best.look, best.ctas_per_sm,
                         V.chunk_bytes, V.threads, best_ms);
            std::fclose(f);
        }
    }
    return report();
}

const char *gbu_status_name(int32_t s)
{
    switch (s) {
    case GBU_OK: return "GBU_OK";
    case GBU_HEADER_BITS: return "GBU_HEADER_BITS";
    case GBU_TOO_SHORT: return "GBU_TOO_SHORT";
    case GBU_TOO_LONG: return "GBU_TOO_LONG";
    case GBU_OVERLONG: return "GBU_OVERLONG";
    case GBU_TOO_LARGE: return "GBU_TOO_LARGE";
    case GBU_SURROGATE: return "GBU_SURROGATE";
    case GBU_LONE_HIGH_SURROGATE: return "GBU_LONE_HIGH_SURROGATE";
    case GBU_LONE_LOW_SURROGATE: return "GBU_LONE_LOW_SURROGATE";
    case GBU_OUTPUT_TOO_SMALL: return "GBU_OUTPUT_TOO_SMALL";
    case GBU_INVALID_ARG: return "GBU_INVALID_ARG";
    case GBU_DEVICE_ERROR: return "GBU_DEVICE_ERROR";
    case GBU_DEVICE_TIMEOUT: return "GBU_DEVICE_TIMEOUT";
    default: return "GBU_UNKNOWN";
    }
}

uint64_t gbu_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
