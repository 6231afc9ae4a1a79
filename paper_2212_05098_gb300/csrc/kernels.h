// Host-side view of the transcoding kernel (internal).
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
                 kHdrEpoch = 24, kHdrClaim = 28;
constexpr size_t kHdrResult = 64;   // result slot (used where no caller slot exists)
constexpr size_t kHeaderBytes = 256;

// Describe one input (chunk count included) for a job starting at chunk_base.
Item make_item(const void *in, uint64_t n, bool utf16, void *out, uint64_t cap, bool write,
               ResultSlot *result, uint32_t chunk_base, bool big_endian = false);

// Tuning parameters of a launch: look-back width (status words per lane per
// round, one of kLookWidths) and resident CTAs per SM (0: as many as fit).
constexpr int kLookWidths[] = {1, 2, 4, 8, 16};
#ifndef GBU_DEFAULT_LOOK
#define GBU_DEFAULT_LOOK 1
#endif
struct Tune {
    int look = GBU_DEFAULT_LOOK;
    int ctas_per_sm = 0;
};

// Dynamic shared memory of one CTA; CTAs per SM that fit; grid size for a
// tuning (every CTA resident); grid size with as many CTAs as fit.
size_t job_smem_bytes(bool write);
int job_max_ctas_per_sm(int device);
int job_grid(int device, const Tune &t);
int job_max_grid(int device);

// `be`: the job holds UTF-16BE items (selects a kernel with the byte swaps).
cudaError_t launch_job(const Job &J, bool write, int grid, cudaStream_t stream,
                       int look = GBU_DEFAULT_LOOK, bool be = false);
cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream);

// Count one kernel launch (gbu_kernel_launch_count).
void note_launch();

}  // namespace gbu
