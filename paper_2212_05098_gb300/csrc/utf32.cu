// UTF-32LE transcoding (paper Sec. 2: a UTF-32 unit is the code point
// itself; Fig. 1(a) for the UTF-8 byte layouts).
//
// Three short launches per call instead of the persistent single-pass
// kernel of the UTF-16 paths:
//   count  one CTA per tile: the tile's output length up to its first
//          invalid input unit, and that unit;
//   scan   one CTA: exclusive prefix of the tile lengths (each tile's output
//          offset), the first invalid unit of the input, the call's result;
//   write  one CTA per tile: encode, stage at the scanned offsets in shared
//          memory, write the tile out with aligned 16-byte stores.
// UTF-8 -> UTF-32 validates with the UTF-8 kernel first (exactly the UTF-8
// rules of Sec. 6.4); count, scan and write then decode the valid prefix,
// one code point per character start.
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "utf32.h"

namespace gbu {

namespace {

constexpr uint32_t kBadNone = 0xFFFFFFFFu;   // tile without an invalid unit

// Sum over the CTA's kThreads threads (every thread gets the total).
__device__ __forceinline__ uint32_t cta_sum(uint32_t v, uint32_t *s_warp)
{
    uint32_t total;
    block_exclusive_scan(v, s_warp, &total);
    return total;
}

// ---- UTF-32LE input --------------------------------------------------------

// Output bytes of one valid unit (Fig. 1(a)).
__device__ __forceinline__ uint32_t u32_len(uint32_t u)
{
    return 1u + (u >= 0x80u) + (u >= 0x800u) + (u >= 0x10000u);
}

// Invalid unit kind: 0 (valid), TOO_LARGE above U+10FFFF, SURROGATE in D800-DFFF.
__device__ __forceinline__ uint32_t u32_kind(uint32_t u)
{
    if (u > 0x10FFFFu) return kTooLarge;
    if (u >= 0xD800u && u <= 0xDFFFu) return kSurrogate;
    return 0;
}

// Each thread owns units [8 * tid, 8 * tid + 8) of its tile.
__global__ void __launch_bounds__(kThreads) u32_count_kernel(const uint32_t *in, uint64_t n,
                                                             uint32_t *tile_cnt, uint32_t *tile_bad)
{
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_bad;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile32;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) s_bad = kBadNone;
    uint32_t u[8], my_bad = kBadNone, my_kind = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint64_t g = t0 + 8 * tid + j;
        u[j] = g < n ? in[g] : 0u;
        const uint32_t k = g < n ? u32_kind(u[j]) : 0u;
        if (k && my_bad == kBadNone) {
            my_bad = 8 * tid + j;
            my_kind = k;
        }
    }
    __syncthreads();
    if (my_bad != kBadNone) atomicMin(&s_bad, my_bad);
    __syncthreads();
    const uint32_t bad = s_bad;
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint64_t g = t0 + 8 * tid + j;
        if (g < n && 8 * tid + j < bad) cnt += u32_len(u[j]);
    }
    const uint32_t total = cta_sum(cnt, s_warp);
    if (tid == 0) tile_cnt[blockIdx.x] = total;
    if (my_bad == bad && bad != kBadNone) tile_bad[blockIdx.x] = (my_kind << 24) | bad;
    if (tid == 0 && bad == kBadNone) tile_bad[blockIdx.x] = kBadNone;
}

__global__ void __launch_bounds__(kThreads) u32_write_kernel(const uint32_t *in, uint8_t *out,
                                                             uint64_t cap, const uint64_t *tile_base,
                                                             const uint64_t *limit)
{
    __shared__ __align__(16) uint8_t s_stage[4 * kTile32 + 64];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile32;
    const uint64_t lim = *limit;                 // valid units of the input
    const uint64_t base = tile_base[blockIdx.x];
    if (t0 >= lim || base >= cap) return;        // the same for the whole CTA
    const uint32_t tid = threadIdx.x;
    uint32_t v[8], len[8], cnt = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint64_t g = t0 + 8 * tid + j;
        const uint32_t u = g < lim ? in[g] : 0u;
        len[j] = g < lim ? u32_len(u) : 0u;
        // the code point's 6-bit groups, most significant first, one per
        // byte, the last len[j] of them with their tags (F0/E0/C0 lead, 80)
        const uint32_t grp = (u >> 18) | ((u >> 4) & 0x3F00u) | ((u << 10) & 0x3F0000u) |
                             ((u << 24) & 0x3F000000u);
        uint32_t x = u;
        if (len[j] == 2) x = (grp >> 16) | 0x80C0u;
        if (len[j] == 3) x = (grp >> 8) | 0x8080E0u;
        if (len[j] == 4) x = grp | 0x808080F0u;
        v[j] = x;
        cnt += len[j];
    }
    uint32_t total;
    uint32_t off = block_exclusive_scan(cnt, s_warp, &total);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        for (uint32_t b = 0; b < len[j]; b++) s_stage[off + b] = (uint8_t)(v[j] >> (8 * b));
        off += len[j];
    }
    __syncthreads();
    const uint64_t room = cap - base;
    const uint32_t nbytes = total < room ? total : (uint32_t)room;
    block_store_bytes(s_stage, out + base, nbytes);
}

// ---- UTF-8 input (valid prefix of p bytes) -----------------------------------

// Each thread owns bytes [32 * tid, 32 * tid + 32) of its tile; a character
// belongs to the thread holding its first byte.
__global__ void __launch_bounds__(kThreads) u8_starts_kernel(const uint8_t *in, uint64_t p,
                                                             uint32_t *tile_cnt, uint32_t *tile_bad)
{
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile8;
    uint32_t cnt = 0;
    for (int j = 0; j < 32; j++) {
        const uint64_t g = t0 + 32 * threadIdx.x + j;
        if (g < p && (in[g] & 0xC0u) != 0x80u) cnt++;
    }
    const uint32_t total = cta_sum(cnt, s_warp);
    if (threadIdx.x == 0) {
        tile_cnt[blockIdx.x] = total;
        tile_bad[blockIdx.x] = kBadNone;
    }
}

__global__ void __launch_bounds__(kThreads) u8_write32_kernel(const uint8_t *in, uint64_t p,
                                                              uint32_t *out, uint64_t cap,
                                                              const uint64_t *tile_base)
{
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile8;
    const uint64_t base = tile_base[blockIdx.x];
    if (base >= cap) return;                     // the same for the whole CTA
    const uint64_t g0 = t0 + 32 * threadIdx.x;
    uint32_t cnt = 0;
    for (int j = 0; j < 32; j++) {
        const uint64_t g = g0 + j;
        if (g < p && (in[g] & 0xC0u) != 0x80u) cnt++;
    }
    uint32_t total;
    uint64_t idx = base + block_exclusive_scan(cnt, s_warp, &total);
    for (int j = 0; j < 32; j++) {
        const uint64_t g = g0 + j;
        if (g >= p) break;
        const uint32_t b = in[g];
        if ((b & 0xC0u) == 0x80u) continue;
        // a character start of the valid prefix: its continuations lie
        // inside the prefix too (Fig. 1(a) payload bits)
        uint32_t cp;
        if (b < 0x80u) {
            cp = b;
        } else if (b < 0xE0u) {
            cp = ((b & 0x1Fu) << 6) | (in[g + 1] & 0x3Fu);
        } else if (b < 0xF0u) {
            cp = ((b & 0x0Fu) << 12) | ((in[g + 1] & 0x3Fu) << 6) | (in[g + 2] & 0x3Fu);
        } else {
            cp = ((b & 0x07u) << 18) | ((in[g + 1] & 0x3Fu) << 12) | ((in[g + 2] & 0x3Fu) << 6) |
                 (in[g + 3] & 0x3Fu);
        }
        if (idx < cap) out[idx] = cp;
        idx++;
    }
}

// ---- scan over the tiles ---------------------------------------------------

constexpr int kScanThreads = 1024;

// One CTA. Tile t's output offset into tile_base[t]; the number of valid
// input units into *limit; the call's result into *res. With a tile error
// (from u32_count_kernel) the result is that error; otherwise pre_status /
// pre_offset (a UTF-8 validation's result) or OK, and OUTPUT_TOO_SMALL when
// the output exceeds cap.
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(
    const uint32_t *tile_cnt, const uint32_t *tile_bad, uint64_t *tile_base, uint64_t *limit,
    uint64_t ntiles, uint64_t n, uint64_t tile_units, uint64_t cap, int32_t pre_status,
    uint64_t pre_offset, ResultSlot *res)
{
    __shared__ unsigned long long s_first;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
    const uint64_t lo = tid * per < ntiles ? tid * per : ntiles;
    const uint64_t hi = lo + per < ntiles ? lo + per : ntiles;
    if (tid == 0) s_first = ~0ull;
    uint64_t sum = 0, first = ~0ull;
    for (uint64_t t = lo; t < hi; t++) {
        sum += tile_cnt[t];
        if (first == ~0ull && tile_bad[t] != kBadNone) first = t;
    }
    // exclusive scan of the per-thread sums
    uint64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t x = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += x;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (first != ~0ull) atomicMin(&s_first, (unsigned long long)first);
    uint64_t below = 0, all = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
        const uint64_t x = s_warp[w];
        if (w < (int)warp) below += x;
        all += x;
    }
    __syncthreads();
    uint64_t run = below + inc - sum;
    const uint64_t err_tile = s_first;
    for (uint64_t t = lo; t < hi; t++) {
        tile_base[t] = run;
        if (t == err_tile) {
            const uint32_t bad = tile_bad[t];
            const uint64_t at = t * tile_units + (bad & 0xFFFFFFu);
            res->status = (int32_t)(bad >> 24);
            res->reserved = 0;
            res->in_offset = at;
            res->out_len = run + tile_cnt[t];
            *limit = at;
        }
        run += tile_cnt[t];
    }
    if (tid == 0 && err_tile == ~0ull) {
        res->status = pre_status != kOk ? pre_status : (all > cap ? kOutputTooSmall : kOk);
        res->reserved = 0;
        res->in_offset = pre_status != kOk ? pre_offset : n;
        res->out_len = all;
        *limit = n;
    }
}

}  // namespace

size_t utf32_scratch_bytes(uint64_t ntiles)
{
    return 16 + ntiles * (8 + 4 + 4);
}

// Scratch layout: limit (u64), pad, tile_base[ntiles] (u64), tile_cnt[ntiles],
// tile_bad[ntiles] (u32).
static void carve(void *scratch, uint64_t ntiles, uint64_t *&limit, uint64_t *&base,
                  uint32_t *&cnt, uint32_t *&bad)
{
    uint8_t *p = static_cast<uint8_t *>(scratch);
    limit = reinterpret_cast<uint64_t *>(p);
    base = reinterpret_cast<uint64_t *>(p + 16);
    cnt = reinterpret_cast<uint32_t *>(p + 16 + 8 * ntiles);
    bad = cnt + ntiles;
}

cudaError_t launch_utf32_to_utf8(const uint32_t *in, uint64_t n, uint8_t *out, uint64_t cap,
                                 bool write, void *scratch, ResultSlot *res, cudaStream_t s)
{
    const uint64_t ntiles = (n + kTile32 - 1) / kTile32;
    uint64_t *limit, *base;
    uint32_t *cnt, *bad;
    carve(scratch, ntiles, limit, base, cnt, bad);
    u32_count_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, cnt, bad);
    tile_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, bad, base, limit, ntiles, n, kTile32, cap,
                                                kOk, 0, res);
    if (write) u32_write_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, cap, base, limit);
    return cudaGetLastError();
}

cudaError_t launch_utf8_to_utf32(const uint8_t *in, uint64_t n, uint64_t p, int32_t status,
                                 uint64_t in_offset, uint32_t *out, uint64_t cap, bool write,
                                 void *scratch, ResultSlot *res, cudaStream_t s)
{
    const uint64_t ntiles = (p + kTile8 - 1) / kTile8;
    uint64_t *limit, *base;
    uint32_t *cnt, *bad;
    carve(scratch, ntiles, limit, base, cnt, bad);
    if (ntiles) u8_starts_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in, p, cnt, bad);
    tile_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, bad, base, limit, ntiles, n, kTile8, cap,
                                                status, in_offset, res);
    if (write && ntiles)
        u8_write32_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in, p, out, cap, base);
    return cudaGetLastError();
}

}  // namespace gbu
