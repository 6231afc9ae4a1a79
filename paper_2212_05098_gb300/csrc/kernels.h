// Host-side view of the transcoding kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

// Resident CTAs per SM the kernel is compiled for (register budget).
#ifndef GBU_MIN_BLOCKS
#define GBU_MIN_BLOCKS 2
#endif

namespace gbu {

constexpr int kMinBlocks = GBU_MIN_BLOCKS;

// Scratch header shared by every job launch on one scratch area.
constexpr size_t kHdrChunks = 0, kHdrExit = 4, kHdrFlags = 8, kHdrDone = 12, kHdrErr = 16,
                 kHdrEpoch = 24, kHdrClaim = 28, kHdrValidErr = 32;
constexpr size_t kHdrResult = 64;   // result slot (used where no caller slot exists)
constexpr size_t kHeaderBytes = 256;

// Inputs of at most kSmallMaxChunks chunks may take the one-launch cluster
// path (one CTA per chunk, nothing kept in global memory between launches).
constexpr int kSmallMaxChunks = 8;

// Tuning parameters of a launch: look-back width (status words per lane per
// round, one of kLookWidths), resident CTAs per SM (0: as many as fit), the
// largest single input (in chunks) sent down the one-launch path, and the
// kernel shape (an index into the compiled shapes; -1: chosen per call from
// the input's size).
constexpr int kLookWidths[] = {1, 2, 4, 8, 16};
#ifndef GBU_DEFAULT_LOOK
#define GBU_DEFAULT_LOOK 1
#endif
struct Tune {
    int look = GBU_DEFAULT_LOOK;
    int ctas_per_sm = 0;
    int small_chunks = kSmallMaxChunks;
    int variant = -1;
};

// One compiled kernel shape (a translation unit of its own): its compute
// threads per CTA, input bytes per thread and chunk, the resident CTAs per SM
// it is compiled for, and its host entry points:
//   make_item        describe one input (chunk count included) for a job
//                    starting at chunk_base;
//   smem_bytes       dynamic shared memory of one CTA of the persistent kernel;
//   max_ctas_per_sm  CTAs per SM that fit (sets the kernels' attributes once
//                    per device; 0 on failure);
//   grid             persistent grid for a tuning (every CTA resident);
//   launch_job       the persistent kernel over a job (`be`: the job holds
//                    UTF-16BE items, which selects a kernel with byte swaps;
//                    `in`: 1 / 2 when every item's input is UTF-8 / UTF-16,
//                    which may select a kernel with that direction's code
//                    only, 0 otherwise);
//   launch_small     the one-launch cluster kernel over one item of at most
//                    kSmallMaxChunks chunks;
//   launch_small_items  one CTA per item over `count` one-chunk items (device
//                    array; `any_be`: some item is UTF-16BE).
struct Variant {
    int threads;
    int bpt;
    int min_blocks;
    uint32_t chunk_bytes;
    Item (*make_item)(const void *in, uint64_t n, bool utf16, void *out, uint64_t cap, bool write,
                      ResultSlot *result, uint32_t chunk_base, bool big_endian);
    size_t (*smem_bytes)(bool write);
    int (*max_ctas_per_sm)(int device);
    int (*grid)(int device, const Tune &t);
    cudaError_t (*launch_job)(const Job &J, bool write, int grid, cudaStream_t stream, int look,
                              bool be, int in);
    cudaError_t (*launch_small)(const Item &I, bool write, bool validate, cudaStream_t stream);
    cudaError_t (*launch_small_items)(const Item *items, uint32_t count, bool write, bool any_be,
                                      cudaStream_t stream);
};

// The compiled shapes (compute threads x bytes per thread).
const Variant &variant_256x48();
const Variant &variant_256x32();
const Variant &variant_512x32();
const Variant &variant_128x48();
const Variant &variant_512x48();
constexpr int kVariants = 5;
// Shape i (0: 256 x 48, the default; any i outside [0, kVariants): the default).
const Variant &variant(int i);
// Index of the shape with these compute threads and chunk bytes, or -1.
int variant_index(int threads, uint32_t chunk_bytes);

// Chunks of one input for a shape (counted from the 16-byte boundary at or
// before the input; an empty input has one).
inline uint64_t chunks_of(const Variant &v, const void *in, uint64_t n, bool utf16)
{
    if (n == 0) return 1;
    const uint64_t p = reinterpret_cast<uintptr_t>(in) & 15u;
    const uint64_t head = utf16 ? p >> 1 : p;
    const uint64_t units = utf16 ? v.chunk_bytes / 2 : v.chunk_bytes;
    return (head + n + units - 1) / units;
}

cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream);

// Count one kernel launch (gbu_kernel_launch_count).
void note_launch();

}  // namespace gbu
