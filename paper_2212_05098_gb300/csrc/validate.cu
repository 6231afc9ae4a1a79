// Validation-only calls (paper Sec. 6.4: the UTF-8 rules; Sec. 7.4: the
// pairing of UTF-16 surrogates) as a plain streaming kernel. A validation
// writes no output, so it needs no output offsets: no scan, no look-back, no
// shared memory and no barrier.
//
// Each thread checks kVB = 32 input bytes per step with two aligned 16-byte
// loads, issued one step ahead (the next step's loads are in flight while the
// thread checks the current block). The lanes of a warp hold consecutive
// 32-byte blocks, so the 4 bytes before and after a thread's block (the
// context its checks need) come from the neighbouring lanes by shuffles, and
// from global memory at the two ends of the warp. Bytes are counted from the 16-byte boundary at or before the
// input ("virtual" positions); bytes outside the input read as zero, which
// neither creates nor hides an error inside it, and no read leaves the
// 16-byte blocks that hold input bytes.
//
// A thread runs the checks of the transcoding kernel's first phase: the exact
// structure check (the continuations the leads expect are exactly the
// continuation bytes) and value checks that never miss an error but may flag
// valid text. A flagged thread applies the exact per-position rule (the check
// the sequential decoder applies if a character starts there) and posts the
// key (position << 8 | kind) of its first error with a 64-bit atomicMin; the
// smallest key over all threads is the input's first error (the paper's ell),
// because every earlier position is a validated character start or a
// continuation inside one. A one-thread kernel then turns the key into the
// call's result and resets it for the next call.
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "validate.h"

namespace gbu {

namespace {

constexpr int kVB = 32;          // input bytes per thread and step
constexpr int kVW = kVB / 4;     // their 32-bit words
constexpr int kVThreads = 256;   // threads per CTA
constexpr int kV8Blocks = 4;     // resident CTAs per SM the UTF-8 kernel is compiled for
constexpr int kV16Blocks = 6;    // and the UTF-16 kernels
constexpr uint32_t kHi7 = 0x80808080u;

__device__ __forceinline__ uint32_t ldg32(const uint8_t *p)
{
    return __ldg(reinterpret_cast<const uint32_t *>(p));
}

// A thread's loads for the block at virtual byte v: its 32 bytes, and at the
// two ends of the warp the word beyond the warp's blocks (lane 0: the 4 bytes
// before v, lane 31: the 4 bytes after its block). Nothing at or beyond the
// readable end endv (a multiple of 16) is read; those bytes are zero.
struct Raw {
    uint4 a, b;
    uint32_t edge;
};

__device__ __forceinline__ void fetch_block(const uint8_t *in_al, uint64_t v, uint64_t endv,
                                            uint32_t lane, Raw &r)
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    r.a = v < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + v)) : z;
    r.b = v + 16 < endv ? __ldg(reinterpret_cast<const uint4 *>(in_al + v + 16)) : z;
    r.edge = 0u;
    if (lane == 0)
        r.edge = v >= 4 && v - 4 < endv ? ldg32(in_al + v - 4) : 0u;
    else if (lane == 31)
        r.edge = v + kVB < endv ? ldg32(in_al + v + kVB) : 0u;
}

// The thread's words from its loads: w[1..kVW] its own, w[0] the 4 bytes
// before, w[kVW + 1] the 4 bytes after. Every lane of the warp calls it
// (shuffles).
__device__ __forceinline__ void block_words(const Raw &r, uint32_t lane, uint32_t (&w)[kVW + 2])
{
    w[1] = r.a.x; w[2] = r.a.y; w[3] = r.a.z; w[4] = r.a.w;
    w[5] = r.b.x; w[6] = r.b.y; w[7] = r.b.z; w[8] = r.b.w;
    uint32_t prev = __shfl_up_sync(0xffffffffu, w[kVW], 1);
    uint32_t next = __shfl_down_sync(0xffffffffu, w[1], 1);
    if (lane == 0) prev = r.edge;
    if (lane == 31) next = r.edge;
    w[0] = prev;
    w[kVW + 1] = next;
}

// Zero the bytes outside [lo, hi) (virtual bytes) when the block touches an
// end of the input.
__device__ __forceinline__ void mask_block8(uint32_t (&w)[kVW + 2], uint64_t v, uint64_t lo,
                                            uint64_t hi)
{
    if (v >= lo + 4 && v + kVB + 4 <= hi) return;
#pragma unroll
    for (int j = 0; j < kVW + 2; j++)
        w[j] = mask_word_bytes(w[j], (int64_t)v - 4 + 4 * j, (int64_t)lo, (int64_t)hi);
}

// ---- UTF-8 -----------------------------------------------------------------

struct Cls8 {
    uint32_t c2, c3, c4, ct;   // bit 7 of each byte: >= C0, >= E0, >= F0, 80-BF
};

__device__ __forceinline__ Cls8 classify8(uint32_t x, bool k3, bool k4)
{
    const uint32_t x1 = x << 1;
    Cls8 c;
    c.c2 = x & x1 & kHi7;
    c.c3 = k3 ? c.c2 & (x << 2) : 0u;
    c.c4 = k4 ? c.c3 & (x << 3) : 0u;
    c.ct = x & ~x1 & kHi7;
    return c;
}

// Non-zero when the thread's bytes may hold an error (never zero when they
// do). k3 / k4: the warp holds >= E0 / >= F0 leads (else those terms are 0).
template <bool k3, bool k4>
__device__ __forceinline__ uint32_t check8(const uint32_t (&w)[kVW + 2])
{
    Cls8 cp = classify8(w[0], k3, k4);
    uint32_t bad = 0;
#pragma unroll
    for (int j = 1; j <= kVW + 1; j++) {
        const uint32_t x = w[j];
        const Cls8 c = classify8(x, k3, k4);
        if (j <= kVW) {
            // continuation positions expected by the leads 1, 2, 3 bytes back
            uint32_t exp = __funnelshift_l(cp.c2, c.c2, 8);
            if (k3) exp |= __funnelshift_l(cp.c3, c.c3, 16);
            if (k4) exp |= __funnelshift_l(cp.c4, c.c4, 24);
            bad |= exp ^ c.ct;
            // C0 / C1
            const uint32_t x7 = x & 0x7F7F7F7Fu;
            bad |= c.c2 & ~(x7 + 0x3E3E3E3Eu);
            if (k3 || k4) {
                const uint32_t y = __funnelshift_r(x, w[j + 1], 8);   // the next byte of each
                if (k3) {
                    // E0 + 80..9F, ED + A0..BF: E0 where bit 5 of the next
                    // byte is clear, ED where it is set
                    const uint32_t m = (((y << 2) >> 7) & 0x01010101u) * 0x0Du;
                    bad |= zero_bytes(x ^ 0xE0E0E0E0u ^ m);
                }
                if (k4) {
                    // F0 + 80..8F, F4 + 90..BF, and F5..FF
                    const uint32_t m = (((y << 2) | (y << 3)) >> 5) & 0x04040404u;
                    bad |= zero_bytes(x ^ 0xF0F0F0F0u ^ m);
                    bad |= (x7 + 0x0B0B0B0Bu) & x & kHi7;
                }
            }
        } else {
            // continuations the thread's last leads expect in the next bytes
            uint32_t exp = cp.c2 >> 24;
            if (k3) exp |= cp.c3 >> 16;
            if (k4) exp |= cp.c4 >> 8;
            bad |= exp & ~c.ct;
        }
        cp = c;
    }
    return bad;
}

struct Words {
    uint32_t w[kVW + 2];
};

// The exact rule at every owned position inside [lo, hi), in order: the key
// of the first error, or ~0.
__device__ __noinline__ unsigned long long exact8(const Words W, uint64_t v, uint64_t lo,
                                                  uint64_t hi)
{
    for (int i = 0; i < kVB; i++) {
        if (v + i < lo || v + i >= hi) continue;
        const int j = (i >> 2) + 1;
        const int sh = (i & 3) * 8;
        const uint32_t xf = __funnelshift_r(W.w[j], W.w[j + 1], sh);   // bytes i .. i+3
        const uint32_t xb = __funnelshift_r(W.w[j - 1], W.w[j], sh);   // bytes i-4 .. i-1
        const uint32_t b0 = xf & 0xFFu;
        int kind = 0;
        if ((b0 & 0xC0u) == 0x80u) {
            // a continuation byte no lead at i-1, i-2, i-3 expects
            const uint32_t p1 = xb >> 24, p2 = (xb >> 16) & 0xFFu, p3 = (xb >> 8) & 0xFFu;
            if (!(p1 >= 0xC0u || p2 >= 0xE0u || p3 >= 0xF0u)) kind = kTooLong;
        } else if (b0 >= 0x80u) {
            if (b0 < 0xC2u) {
                kind = kOverlong;
            } else if (b0 >= 0xF5u) {
                kind = kHeaderBits;
            } else {
                const uint32_t len = b0 < 0xE0u ? 2u : (b0 < 0xF0u ? 3u : 4u);
                const uint32_t cont = (xf ^ 0x80808080u) & 0xC0C0C0C0u;   // zero: continuation
                const uint32_t need = len == 2 ? 0x0000FF00u : (len == 3 ? 0x00FFFF00u : 0xFFFFFF00u);
                if (cont & need) {
                    kind = kTooShort;
                } else {
                    const uint32_t b1 = (xf >> 8) & 0x3Fu, b2 = (xf >> 16) & 0x3Fu;
                    const uint32_t b3 = (xf >> 24) & 0x3Fu;
                    uint32_t cp;
                    if (len == 2) cp = ((b0 & 0x1Fu) << 6) | b1;
                    else if (len == 3) cp = ((b0 & 0x0Fu) << 12) | (b1 << 6) | b2;
                    else cp = ((b0 & 0x07u) << 18) | (b1 << 12) | (b2 << 6) | b3;
                    if (len == 3 && cp < 0x800u) kind = kOverlong;
                    else if (len == 3 && (cp & 0xF800u) == 0xD800u) kind = kSurrogate;
                    else if (len == 4 && cp < 0x10000u) kind = kOverlong;
                    else if (len == 4 && cp > 0x10FFFFu) kind = kTooLarge;
                }
            }
        }
        if (kind) return ((unsigned long long)(v + i - lo) << 8) | (unsigned)kind;
    }
    return ~0ull;
}

__global__ void __launch_bounds__(kVThreads, kV8Blocks)
    validate8_kernel(const uint8_t *in_al, uint64_t head, uint64_t n, unsigned long long *err)
{
    const uint64_t lo = head, hi = head + n;
    const uint64_t endv = (hi + 15) & ~15ull;
    const uint64_t stride = (uint64_t)gridDim.x * kVThreads * kVB;
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t wb = ((uint64_t)blockIdx.x * kVThreads + (threadIdx.x & ~31u)) * kVB;
    Raw cur;
    fetch_block(in_al, wb + (uint64_t)lane * kVB, endv, lane, cur);
    // a warp's lanes step together (the loop bound is warp-uniform)
    for (; wb < endv; wb += stride) {
        const uint64_t v = wb + (uint64_t)lane * kVB;
        Words W;
        block_words(cur, lane, W.w);
        fetch_block(in_al, v + stride, endv, lane, cur);   // the next step's block
        mask_block8(W.w, v, lo, hi);
        // >= E0 and >= F0 leads anywhere in the warp (the look-behind word
        // included): without them their terms are dropped
        uint32_t a3 = 0, a4 = 0;
#pragma unroll
        for (int j = 0; j <= kVW; j++) {
            const uint32_t x3 = W.w[j] & (W.w[j] << 1) & (W.w[j] << 2);
            a3 |= x3;
            a4 |= x3 & (W.w[j] << 3);
        }
        const bool k4 = __any_sync(0xffffffffu, (a4 & kHi7) != 0);
        const bool k3 = __any_sync(0xffffffffu, (a3 & kHi7) != 0);
        uint32_t bad;
        if (k4)
            bad = check8<true, true>(W.w);
        else if (k3)
            bad = check8<true, false>(W.w);
        else
            bad = check8<false, false>(W.w);
        if (bad) {
            const unsigned long long key = exact8(W, v, lo, hi);
            if (key != ~0ull) atomicMin(err, key);
        }
    }
}

// ---- UTF-16 ----------------------------------------------------------------

// Bit 15 of each 16-bit lane: the unit is a surrogate (D800-DFFF); of those,
// bit 10 of the unit (bit 15 of x << 5) tells a low one (DC00-DFFF) from a
// high one (D800-DBFF).
__device__ __forceinline__ uint32_t sur_lanes(uint32_t x)
{
    const uint32_t v = (x & 0xF800F800u) ^ 0xD800D800u;
    return (v - 0x00010001u) & ~v & 0x80008000u;
}

// Unit i of the thread (i in [-2, 18)); w[0] holds units -2, -1.
__device__ __forceinline__ uint32_t unit16(const uint32_t *w, int i)
{
    return (w[(i + 2) >> 1] >> (16 * ((i + 2) & 1))) & 0xFFFFu;
}

__device__ __noinline__ unsigned long long exact16(const Words W, uint64_t u0, uint64_t lo,
                                                   uint64_t hi)
{
    for (int i = 0; i < kVB / 2; i++) {
        if (u0 + i < lo || u0 + i >= hi) continue;
        const uint32_t u = unit16(W.w, i), pv = unit16(W.w, i - 1), nx = unit16(W.w, i + 1);
        int kind = 0;
        if ((u & 0xFC00u) == 0xD800u && (nx & 0xFC00u) != 0xDC00u) kind = kLoneHigh;
        if ((u & 0xFC00u) == 0xDC00u && (pv & 0xFC00u) != 0xD800u) kind = kLoneLow;
        if (kind) return ((unsigned long long)(u0 + i - lo) << 8) | (unsigned)kind;
    }
    return ~0ull;
}

// Units are counted from the 16-byte boundary at or before the input: the
// input is units [lo, hi).
template <bool kBE>
__global__ void __launch_bounds__(kVThreads, kV16Blocks)
    validate16_kernel(const uint8_t *in_al, uint64_t lo, uint64_t n, unsigned long long *err)
{
    const uint64_t hi = lo + n;
    const uint64_t endv = (2 * hi + 15) & ~15ull;   // bytes
    const uint64_t stride = (uint64_t)gridDim.x * kVThreads * kVB;
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t wb = ((uint64_t)blockIdx.x * kVThreads + (threadIdx.x & ~31u)) * kVB;
    Raw cur;
    fetch_block(in_al, wb + (uint64_t)lane * kVB, endv, lane, cur);
    for (; wb < endv; wb += stride) {
        const uint64_t v = wb + (uint64_t)lane * kVB;
        const uint64_t u0 = v / 2;   // the thread's first unit
        Words W;
        block_words(cur, lane, W.w);
        fetch_block(in_al, v + stride, endv, lane, cur);   // the next step's block
        if (u0 < lo + 2 || u0 + kVB / 2 + 2 > hi) {   // units outside the input read as zero
#pragma unroll
            for (int j = 0; j < kVW + 2; j++) {
                const uint64_t a = u0 - 2 + 2 * j;
                const uint32_t k0 = a >= lo && a < hi ? 0xFFFFu : 0u;
                const uint32_t k1 = a + 1 >= lo && a + 1 < hi ? 0xFFFF0000u : 0u;
                W.w[j] &= k0 | k1;
            }
        }
        if (kBE) {
#pragma unroll
            for (int j = 0; j < kVW + 2; j++) W.w[j] = prmt(W.w[j], 0, 0x2301);
        }
        // a unit is a low surrogate exactly when the unit before it is a high
        // one (and the thread's last unit may be high only if a low follows);
        // with no surrogate among the thread's own units none of them is an
        // error, and the pairing check is skipped
        uint32_t sur[kVW + 2], any = 0;
#pragma unroll
        for (int j = 1; j <= kVW; j++) {
            sur[j] = sur_lanes(W.w[j]);
            any |= sur[j];
        }
        uint32_t bad = 0;
        if (any) {
            sur[0] = sur_lanes(W.w[0]);
            sur[kVW + 1] = sur_lanes(W.w[kVW + 1]);
            uint32_t h_prev = sur[0] & ~(W.w[0] << 5);
#pragma unroll
            for (int j = 1; j <= kVW; j++) {
                const uint32_t x5 = W.w[j] << 5;
                const uint32_t h = sur[j] & ~x5;
                bad |= __funnelshift_l(h_prev, h, 16) ^ (sur[j] & x5);
                h_prev = h;
            }
            bad |= (h_prev ^ ((sur[kVW + 1] & (W.w[kVW + 1] << 5)) << 16)) & 0x80000000u;
        }
        if (bad) {
            const unsigned long long key = exact16(W, u0, lo, hi);
            if (key != ~0ull) atomicMin(err, key);
        }
    }
}

// The call's result from the first-error key (validation: out_len 0); the key
// is reset for the next call.
__global__ void validate_result_kernel(unsigned long long *err, uint64_t n, ResultSlot *dst)
{
    const unsigned long long key = *err;
    *err = ~0ull;
    volatile ResultSlot *r = dst;
    r->status = key == ~0ull ? (int32_t)kOk : (int32_t)(key & 0xFFu);
    r->reserved = 0;
    r->in_offset = key == ~0ull ? n : (uint64_t)(key >> 8);
    r->out_len = 0;
    __threadfence_system();
}

// Resident CTAs over the GPU for the UTF-8 kernel ([0]) and the UTF-16
// kernels ([1]), per device (each kernel fills the SMs at its own occupancy).
// Calls from several host threads may fill an entry at once; they store the
// same value.
std::atomic<int> g_grid[64][2] = {};

int validate_grid(int device, bool utf16)
{
    if (device < 0 || device >= 64) return 0;
    std::atomic<int> &g = g_grid[device][utf16 ? 1 : 0];
    const int known = g.load(std::memory_order_relaxed);
    if (known) return known;
    int sms = 0, per = 0, per_be = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    if (!utf16) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, validate8_kernel, kVThreads, 0) !=
            cudaSuccess)
            return 0;
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, validate16_kernel<false>, kVThreads,
                                                          0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_be, validate16_kernel<true>,
                                                          kVThreads, 0) != cudaSuccess)
            return 0;
        if (per_be < per) per = per_be;
    }
    const int grid = sms * (per > 0 ? per : 1);
    g.store(grid, std::memory_order_relaxed);
    return grid;
}

}  // namespace

cudaError_t launch_validate(const void *in, uint64_t n, bool utf16, bool big_endian,
                            unsigned long long *err, ResultSlot *dst, cudaStream_t stream)
{
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return cudaErrorInvalidDevice;
    int grid = validate_grid(device, utf16);
    if (grid <= 0) return cudaErrorInvalidValue;
    const uintptr_t p = reinterpret_cast<uintptr_t>(in);
    const uint8_t *in_al = reinterpret_cast<const uint8_t *>(p & ~(uintptr_t)15u);
    const uint64_t head = p & 15u;   // bytes
    const uint64_t bytes = head + (utf16 ? 2 * n : n);
    // no more CTAs than blocks of work
    const uint64_t per_cta = (uint64_t)kVThreads * kVB;
    const uint64_t need = (bytes + per_cta - 1) / per_cta;
    if ((uint64_t)grid > need) grid = (int)need;
    if (!utf16)
        validate8_kernel<<<grid, kVThreads, 0, stream>>>(in_al, head, n, err);
    else if (big_endian)
        validate16_kernel<true><<<grid, kVThreads, 0, stream>>>(in_al, head / 2, n, err);
    else
        validate16_kernel<false><<<grid, kVThreads, 0, stream>>>(in_al, head / 2, n, err);
    validate_result_kernel<<<1, 1, 0, stream>>>(err, n, dst);
    return cudaGetLastError();
}

}  // namespace gbu
