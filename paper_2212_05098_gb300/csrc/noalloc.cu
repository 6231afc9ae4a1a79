// UTF-8 -> UTF-16LE for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs where another component
// owns all of the device's memory (a framework's caching allocator, a memory
// budget fixed at start-up), code that must never trigger the implicit device
// synchronisation an allocation can cause (latency-critical request paths), or
// plug-ins that are not allowed to own device memory at all. gbu_create /
// gbu_reserve allocate scratch, so those callers get this entry point instead.
//
// It runs the same kernels as gbu_utf8_to_utf16le (the one-launch cluster
// kernel for inputs of a few chunks, which needs no scratch, else the
// persistent kernel), but the persistent kernel's scratch
// (chunk counters, first-error word, look-back status words, per-chunk error
// prefixes and the result slot) lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process exits.
// That fixes the largest input: GBU_NOALLOC_MAX_BYTES.
//
// In host code the array's name only stands in for the symbol; it is not a
// device address. Its device address is looked up with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on that
// device; make that first call before any stream capture. The array has no
// initializer, so it is zero when the library's device code is loaded: the
// look-back status words start "not ready" and the kernel keeps their epoch
// from call to call; each call clears the counters it needs zero.
#include <cstring>
#include <mutex>

#include "../../include/gbutf.h"
#include "kernels.h"

using namespace gbu;

namespace {

// The call runs the default kernel shape (256 compute threads x 48 bytes).
static_assert(kChunkBytes == 256 * 48, "chunks of the default kernel shape");
constexpr uint64_t kNoAllocChunks = (GBU_NOALLOC_MAX_BYTES + 15 + kChunkBytes - 1) / kChunkBytes;
constexpr size_t kScratchBytes = kHeaderBytes + 16 * kNoAllocChunks;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceState {
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

gbu_result fail(int32_t st)
{
    gbu_result r;
    r.status = st;
    r.reserved = 0;
    r.in_offset = 0;
    r.out_len = 0;
    return r;
}

}  // namespace

extern "C" gbu_result gbu_utf8_to_utf16le_noalloc(const uint8_t *d_in, uint64_t n_bytes,
                                                  uint16_t *d_out, uint64_t cap_units,
                                                  void *stream)
{
    if ((n_bytes && !d_in) || (cap_units && !d_out)) return fail(GBU_INVALID_ARG);
    if (n_bytes > GBU_NOALLOC_MAX_BYTES) return fail(GBU_INVALID_ARG);
    if (reinterpret_cast<uintptr_t>(d_out) & 1u) return fail(GBU_INVALID_ARG);
    if (n_bytes == 0) {
        gbu_result r = fail(GBU_OK);
        return r;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(GBU_DEVICE_ERROR);
    // the array used is the current device's: the stream must belong to it
    // (checked before anything is enqueued)
    if (s) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return fail(GBU_INVALID_ARG);
        if (sdev != dev) return fail(GBU_INVALID_ARG);
    }

    Job J{};
    const Variant &V = variant_256x48();
    J.item0 = V.make_item(d_in, n_bytes, false, d_out, cap_units, true, nullptr, 0, false);
    J.num_items = 1;
    J.total_chunks = J.item0.nchunks;
    if (J.total_chunks > kNoAllocChunks) return fail(GBU_INVALID_ARG);
    const bool small = J.total_chunks <= (uint32_t)kSmallMaxChunks;
    const int max_grid = small ? 1 : V.grid(dev, Tune{});
    if (max_grid <= 0) return fail(GBU_DEVICE_ERROR);

    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        DeviceState &d = g_dev[dev];
        if (!d.base) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return fail(GBU_DEVICE_ERROR);
            d.base = static_cast<unsigned char *>(p);
        }
        base = d.base;
    }
    gbu_result r;
    if (small) {
        // a few chunks: one cluster launch that touches nothing but the
        // result slot
        J.item0.result = reinterpret_cast<ResultSlot *>(base + kHdrResult);
        if (V.launch_small(J.item0, true, false, s) != cudaSuccess) return fail(GBU_DEVICE_ERROR);
        note_launch();
        if (cudaMemcpyAsync(&r, base + kHdrResult, sizeof r, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(GBU_DEVICE_ERROR);
        return r;
    }
    // The array keeps whatever the previous call left: counters and flags must
    // start at zero and the first-error word at all ones.
    if (cudaMemsetAsync(base, 0, 16, s) != cudaSuccess ||
        cudaMemsetAsync(base + 16, 0xFF, 8, s) != cudaSuccess ||
        cudaMemsetAsync(base + kHdrClaim, 0, 4, s) != cudaSuccess)
        return fail(GBU_DEVICE_ERROR);

    J.chunks_done = reinterpret_cast<unsigned int *>(base + kHdrChunks);

    J.claim = reinterpret_cast<unsigned int *>(base + kHdrClaim);
    J.exit_count = reinterpret_cast<unsigned int *>(base + kHdrExit);
    J.flags = reinterpret_cast<unsigned int *>(base + kHdrFlags);
    J.item_done = reinterpret_cast<unsigned int *>(base + kHdrDone);
    J.item_err = reinterpret_cast<unsigned long long *>(base + kHdrErr);
    J.epoch = reinterpret_cast<unsigned int *>(base + kHdrEpoch);
    J.status = reinterpret_cast<unsigned long long *>(base + kHeaderBytes);
    J.status_capacity = (uint32_t)kNoAllocChunks;
    J.err_prefix = J.status + kNoAllocChunks;
    J.item0.result = reinterpret_cast<ResultSlot *>(base + kHdrResult);
    const int grid = (uint32_t)max_grid > J.total_chunks ? (int)J.total_chunks : max_grid;
    if (V.launch_job(J, true, grid, s, GBU_DEFAULT_LOOK, false, 1) != cudaSuccess)
        return fail(GBU_DEVICE_ERROR);
    note_launch();
    if (cudaMemcpyAsync(&r, base + kHdrResult, sizeof r, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(GBU_DEVICE_ERROR);
    return r;
}
