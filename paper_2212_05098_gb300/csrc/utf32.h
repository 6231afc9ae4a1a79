// Host-side view of the UTF-32LE kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbu {
// UTF-32LE (utf32.cu): tiles of kTile32 units / kTile8 UTF-8 bytes, one CTA
// of kThreads each; scratch of utf32_scratch_bytes(tiles) bytes, 16-aligned.
constexpr uint32_t kTile32 = 8 * kThreads;
constexpr uint32_t kTile8 = 32 * kThreads;
// Tiles of a call: counted from the 16-byte boundary at or before the input.
uint64_t utf32_tiles(const uint32_t *in, uint64_t n);
uint64_t utf8_tiles(const uint8_t *in, uint64_t p);
size_t utf32_scratch_bytes(uint64_t ntiles);
// UTF-32LE -> UTF-8 (write = false: length / validation only); the result
// lands in *res at stream completion.
cudaError_t launch_utf32_to_utf8(const uint32_t *in, uint64_t n, uint8_t *out, uint64_t cap,
                                 bool write, void *scratch, ResultSlot *res, cudaStream_t s);
// UTF-8 -> UTF-32LE over the valid prefix of p bytes, given the UTF-8
// validation's status and first-error offset.
cudaError_t launch_utf8_to_utf32(const uint8_t *in, uint64_t n, uint64_t p, int32_t status,
                                 uint64_t in_offset, uint32_t *out, uint64_t cap, bool write,
                                 void *scratch, ResultSlot *res, cudaStream_t s);

}  // namespace gbu
