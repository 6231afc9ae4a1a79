// Host-side launch functions for the transcoding kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbu {

// Input units per chunk (one CTA iteration) for each direction.
constexpr uint32_t kChunk8 = 8192;    // UTF-8 bytes per chunk
constexpr uint32_t kChunk16 = 4096;   // UTF-16 words per chunk

// Fill in L.head / L.num_chunks for an input pointer and size; returns the
// 16-byte aligned base the kernels read from.
const uint8_t *plan_utf8(const uint8_t *in, uint64_t n, Launch &L);
const uint16_t *plan_utf16(const uint16_t *in, uint64_t n, Launch &L);

cudaError_t launch_utf8_to_utf16(const uint8_t *in_aligned, uint16_t *out, bool write,
                                 const Launch &L, cudaStream_t stream);
cudaError_t launch_utf16_to_utf8(const uint16_t *in_aligned, uint8_t *out, bool write,
                                 const Launch &L, cudaStream_t stream);
cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream);

}  // namespace gbu
