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
// Count and write read their tiles with aligned 16-byte loads (tiles start at
// the 16-byte boundary at or before the input).
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

// Tiles are counted from the 16-byte boundary at or before the input
// ("virtual" positions): the input occupies virtual units [head, head + n),
// every thread reads its units with aligned 16-byte loads, and a read never
// leaves the 16-byte blocks that hold input bytes.

// Unit j of a thread's 8 (virtual g0 + j) lies inside [lo, hi): bit j.
__device__ __forceinline__ uint32_t range_bits8(uint64_t g0, uint64_t lo, uint64_t hi)
{
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 8; j++)
        if (g0 + j >= lo && g0 + j < hi) m |= 1u << j;
    return m;
}

// The thread's 8 units at virtual g0 (zeros beyond endv, a multiple of 4).
__device__ __forceinline__ void load_units8(const uint32_t *in_al, uint64_t g0, uint64_t endv,
                                            uint32_t (&u)[8])
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    const uint4 a = g0 < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + g0)) : z;
    const uint4 b = g0 + 4 < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + g0 + 4)) : z;
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}

// Each thread owns virtual units [8 * tid, 8 * tid + 8) of its tile.
__global__ void __launch_bounds__(kThreads) u32_count_kernel(const uint32_t *in_al, uint64_t head,
                                                             uint64_t n, uint32_t *tile_cnt,
                                                             uint32_t *tile_bad)
{
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_bad;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile32;
    const uint64_t endv = (head + n + 3) & ~3ull;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) s_bad = kBadNone;
    const uint64_t g0 = t0 + 8 * tid;
    uint32_t u[8];
    load_units8(in_al, g0, endv, u);
    const uint32_t in_range = range_bits8(g0, head, head + n);
    uint32_t my_bad = kBadNone, my_kind = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t k = ((in_range >> j) & 1u) ? u32_kind(u[j]) : 0u;
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
    for (int j = 0; j < 8; j++)
        if (((in_range >> j) & 1u) && 8 * tid + j < bad) cnt += u32_len(u[j]);
    const uint32_t total = cta_sum(cnt, s_warp);
    if (tid == 0) tile_cnt[blockIdx.x] = total;
    if (my_bad == bad && bad != kBadNone) tile_bad[blockIdx.x] = (my_kind << 24) | bad;
    if (tid == 0 && bad == kBadNone) tile_bad[blockIdx.x] = kBadNone;
}

__global__ void __launch_bounds__(kThreads) u32_write_kernel(const uint32_t *in_al, uint64_t head,
                                                             uint64_t n, uint8_t *out, uint64_t cap,
                                                             const uint64_t *tile_base,
                                                             const uint64_t *limit)
{
    __shared__ __align__(16) uint8_t s_stage[4 * kTile32 + 64];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile32;
    const uint64_t lim = head + *limit;          // virtual end of the valid units
    const uint64_t base = tile_base[blockIdx.x];
    if (t0 >= lim || base >= cap) return;        // the same for the whole CTA
    const uint32_t tid = threadIdx.x;
    const uint64_t g0 = t0 + 8 * tid;
    uint32_t u[8];
    load_units8(in_al, g0, (head + n + 3) & ~3ull, u);
    const uint32_t in_range = range_bits8(g0, head, lim);
    uint32_t v[8], len[8], cnt = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        len[j] = ((in_range >> j) & 1u) ? u32_len(u[j]) : 0u;
        // the code point's 6-bit groups, most significant first, one per
        // byte, the last len[j] of them with their tags (F0/E0/C0 lead, 80)
        const uint32_t x0 = u[j];
        const uint32_t grp = (x0 >> 18) | ((x0 >> 4) & 0x3F00u) | ((x0 << 10) & 0x3F0000u) |
                             ((x0 << 24) & 0x3F000000u);
        uint32_t x = x0;
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

// Each thread owns virtual bytes [32 * tid, 32 * tid + 32) of its tile; a
// character belongs to the thread holding its first byte. The thread's words:
// w[0..7] its bytes, w[8] the 4 bytes after them (a character's last bytes).
__device__ __forceinline__ void load_bytes32(const uint8_t *in_al, uint64_t v, uint64_t endv,
                                             uint32_t (&w)[9])
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    const uint4 a = v < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + v)) : z;
    const uint4 b = v + 16 < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + v + 16)) : z;
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = v + 32 < endv ? __ldg(reinterpret_cast<const uint32_t *>(in_al + v + 32)) : 0u;
}

// Bit 7 of every byte of the thread's 32 that starts a character (not
// 10xxxxxx) inside the valid prefix [lo, hi), one word per 4 bytes.
__device__ __forceinline__ void start_bits(const uint32_t (&w)[9], uint64_t v, uint64_t lo,
                                           uint64_t hi, uint32_t (&st)[8])
{
    const bool whole = v >= lo && v + 32 <= hi;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t x = w[j];
        uint32_t m = ~(x & ~(x << 1)) & 0x80808080u;
        if (!whole) {
            uint32_t keep = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (v + 4 * j + k >= lo && v + 4 * j + k < hi) keep |= 0x80u << (8 * k);
            m &= keep;
        }
        st[j] = m;
    }
}

__global__ void __launch_bounds__(kThreads) u8_starts_kernel(const uint8_t *in_al, uint64_t head,
                                                             uint64_t p, uint32_t *tile_cnt,
                                                             uint32_t *tile_bad)
{
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t v = (uint64_t)blockIdx.x * kTile8 + 32 * threadIdx.x;
    uint32_t w[9], st[8], cnt = 0;
    load_bytes32(in_al, v, (head + p + 15) & ~15ull, w);
    start_bits(w, v, head, head + p, st);
#pragma unroll
    for (int j = 0; j < 8; j++) cnt += __popc(st[j]);
    const uint32_t total = cta_sum(cnt, s_warp);
    if (threadIdx.x == 0) {
        tile_cnt[blockIdx.x] = total;
        tile_bad[blockIdx.x] = kBadNone;
    }
}

__global__ void __launch_bounds__(kThreads) u8_write32_kernel(const uint8_t *in_al, uint64_t head,
                                                              uint64_t p, uint32_t *out,
                                                              uint64_t cap,
                                                              const uint64_t *tile_base)
{
    __shared__ __align__(16) uint32_t s_out[kTile8 + 16];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    const uint64_t base = tile_base[blockIdx.x];
    if (base >= cap) return;                     // the same for the whole CTA
    const uint64_t v = (uint64_t)blockIdx.x * kTile8 + 32 * threadIdx.x;
    uint32_t w[9], st[8], cnt = 0;
    load_bytes32(in_al, v, (head + p + 15) & ~15ull, w);
    start_bits(w, v, head, head + p, st);
#pragma unroll
    for (int j = 0; j < 8; j++) cnt += __popc(st[j]);
    uint32_t total;
    uint32_t o = block_exclusive_scan(cnt, s_warp, &total);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (!((st[i >> 2] >> (8 * (i & 3) + 7)) & 1u)) continue;
        // a character start of the valid prefix: its continuations lie inside
        // the prefix too (Fig. 1(a) payload bits)
        const uint32_t x = __funnelshift_r(w[i >> 2], w[(i >> 2) + 1], 8 * (i & 3));
        const uint32_t b0 = x & 0xFFu, b1 = (x >> 8) & 0x3Fu, b2 = (x >> 16) & 0x3Fu,
                       b3 = (x >> 24) & 0x3Fu;
        uint32_t cp;
        if (b0 < 0x80u)
            cp = b0;
        else if (b0 < 0xE0u)
            cp = ((b0 & 0x1Fu) << 6) | b1;
        else if (b0 < 0xF0u)
            cp = ((b0 & 0x0Fu) << 12) | (b1 << 6) | b2;
        else
            cp = ((b0 & 0x07u) << 18) | (b1 << 12) | (b2 << 6) | b3;
        s_out[o++] = cp;
    }
    __syncthreads();
    const uint64_t room = cap - base;
    const uint32_t units = total < room ? total : (uint32_t)room;
    block_store_bytes(reinterpret_cast<const uint8_t *>(s_out),
                      reinterpret_cast<uint8_t *>(out + base), 4u * units);
}

// ---- scan over the tiles ---------------------------------------------------

constexpr int kScanThreads = 1024;

// One CTA. Tile t's output offset into tile_base[t]; the number of valid
// input units into *limit; the call's result into *res (tiles count virtual
// units: the input starts `head` units into tile 0). With a tile error
// (from u32_count_kernel) the result is that error; otherwise pre_status /
// pre_offset (a UTF-8 validation's result) or OK, and OUTPUT_TOO_SMALL when
// the output exceeds cap.
__global__ void __launch_bounds__(kScanThreads, 1) tile_scan_kernel(
    const uint32_t *tile_cnt, const uint32_t *tile_bad, uint64_t *tile_base, uint64_t *limit,
    uint64_t ntiles, uint64_t n, uint64_t head, uint64_t tile_units, uint64_t cap,
    int32_t pre_status, uint64_t pre_offset, ResultSlot *res)
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
            const uint64_t at = t * tile_units + (bad & 0xFFFFFFu) - head;   // input units
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

uint64_t utf32_tiles(const uint32_t *in, uint64_t n)
{
    const uint64_t head = (reinterpret_cast<uintptr_t>(in) & 15u) >> 2;
    return (head + n + kTile32 - 1) / kTile32;
}

uint64_t utf8_tiles(const uint8_t *in, uint64_t p)
{
    const uint64_t head = reinterpret_cast<uintptr_t>(in) & 15u;
    return p ? (head + p + kTile8 - 1) / kTile8 : 0;
}

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
    const uint64_t head = (reinterpret_cast<uintptr_t>(in) & 15u) >> 2;
    const uint32_t *in_al = in - head;
    const uint64_t ntiles = utf32_tiles(in, n);
    uint64_t *limit, *base;
    uint32_t *cnt, *bad;
    carve(scratch, ntiles, limit, base, cnt, bad);
    u32_count_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in_al, head, n, cnt, bad);
    tile_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, bad, base, limit, ntiles, n, head, kTile32,
                                                cap, kOk, 0, res);
    if (write)
        u32_write_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in_al, head, n, out, cap, base, limit);
    return cudaGetLastError();
}

cudaError_t launch_utf8_to_utf32(const uint8_t *in, uint64_t n, uint64_t p, int32_t status,
                                 uint64_t in_offset, uint32_t *out, uint64_t cap, bool write,
                                 void *scratch, ResultSlot *res, cudaStream_t s)
{
    const uint64_t head = reinterpret_cast<uintptr_t>(in) & 15u;
    const uint8_t *in_al = in - head;
    const uint64_t ntiles = utf8_tiles(in, p);
    uint64_t *limit, *base;
    uint32_t *cnt, *bad;
    carve(scratch, ntiles, limit, base, cnt, bad);
    if (ntiles) u8_starts_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in_al, head, p, cnt, bad);
    tile_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, bad, base, limit, ntiles, n, 0, kTile8, cap,
                                                status, in_offset, res);
    if (write && ntiles)
        u8_write32_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in_al, head, p, out, cap, base);
    return cudaGetLastError();
}

}  // namespace gbu
