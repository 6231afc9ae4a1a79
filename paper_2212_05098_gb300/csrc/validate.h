// Host-side view of the validation-only kernel (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbu {
// Validate n input units (UTF-8 bytes, or UTF-16 words, big-endian if
// `big_endian`) at `in` on `stream` and store the result (status, first
// error offset, out_len 0) to `dst`. `err` is a device word holding ~0 before
// the call; it holds ~0 again when the launch is done.
cudaError_t launch_validate(const void *in, uint64_t n, bool utf16, bool big_endian,
                            unsigned long long *err, ResultSlot *dst, cudaStream_t stream);
}  // namespace gbu
