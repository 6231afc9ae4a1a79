// Device-side machinery shared by the transcoding kernels: scratch layout,
// block-wide scan, decoupled look-back over chunk status words, staged
// coalesced stores, and the last-CTA result finalisation.
//
// The paper's transcoders advance sequentially by the n_in / n_out of each
// 64-byte vector (Sec. 6.2, Eqs. for n_in and n_out; Sec. 7.3), and it sketches
// the parallel alternative of computing each segment's transcoded size first
// (Sec. 8, multithreading remark). On the GPU every chunk of the input is
// transcoded by one CTA; the chunk's output offset is the exclusive prefix sum
// of the output lengths of all earlier chunks, obtained in the same pass by a
// decoupled look-back over per-chunk status words.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbu {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Status codes (numerically equal to gbu_status in include/gbutf.h).
enum : int32_t {
    kOk = 0, kHeaderBits = 1, kTooShort = 2, kTooLong = 3, kOverlong = 4,
    kTooLarge = 5, kSurrogate = 6, kLoneHigh = 7, kLoneLow = 8,
    kOutputTooSmall = 16, kInvalidArg = 17, kDeviceError = 18, kDeviceTimeout = 19
};

// Look-back status word: [63:62] flag, [61:40] epoch, [39:0] value.
// A word whose epoch differs from the launch's epoch counts as "not ready",
// so the status array never needs clearing between launches.
constexpr uint64_t kFlagAggregate = 1;
constexpr uint64_t kFlagInclusive = 2;
constexpr int kEpochShift = 40;
constexpr uint32_t kEpochMask = (1u << 22) - 1;
constexpr uint64_t kValueMask = (1ull << 40) - 1;
// Bounded waits: a look-back poll gives up after this many rounds (each
// round sleeps ~0.1-1 us), sets the timeout flag and lets the CTA finish.
constexpr uint32_t kSpinLimit = 1u << 21;

struct ResultSlot {      // layout of gbu_result
    int32_t status;
    uint32_t reserved;
    uint64_t in_offset;
    uint64_t out_len;
};

struct Scratch {
    unsigned int *claim;            // next chunk to hand out
    unsigned int *done;             // CTAs finished
    unsigned int *flags;            // bit 0: a bounded wait timed out; bit 1: bad chunk id
    unsigned long long *err;        // (position << 8) | kind of the first error, ~0 if none
    unsigned long long *status;     // [num_chunks] look-back words
    unsigned long long *err_prefix; // [num_chunks] output units before the chunk's first error
};

// Arguments common to every launch.
struct Launch {
    Scratch s;
    ResultSlot *result;   // device-visible result destination
    uint64_t n;           // input units
    uint64_t cap;         // output capacity in units (ignored for length-only)
    uint32_t head;        // input units between the 16-byte aligned base and the input
    uint32_t num_chunks;
    uint32_t epoch;
};

__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t pack_status(uint64_t flag, uint32_t epoch, uint64_t value)
{
    return (flag << 62) | ((uint64_t)(epoch & kEpochMask) << kEpochShift) | (value & kValueMask);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide exclusive scan of one uint32 per thread (kThreads threads).
// Returns the thread's exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                         uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kThreads / 32 ? warp_tot[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp base
        if (lane == kThreads / 32 - 1) warp_tot[kThreads / 32] = wi;
    }
    __syncthreads();
    *total = warp_tot[kThreads / 32];
    return warp_tot[warp] + inc - v;
}

// Decoupled look-back, run by one full warp of the CTA that owns `chunk`
// (chunk > 0). Reads up to 32 predecessors at a time; sums aggregates back
// to the nearest inclusive prefix. Returns the chunk's exclusive prefix (all
// lanes). On a wait longer than kSpinLimit rounds it sets the timeout flag
// and returns what it has.
__device__ __forceinline__ uint64_t lookback(const Launch &L, uint32_t chunk)
{
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int64_t base = (int64_t)chunk - 1;
    uint32_t rounds = 0;
    while (true) {
        const int64_t idx = base - lane;
        uint64_t val = 0, flag = kFlagInclusive;   // before chunk 0: inclusive 0
        while (true) {
            if (idx >= 0) {
                const uint64_t w = ld_relaxed(&L.s.status[idx]);
                flag = w >> 62;
                if (((w >> kEpochShift) & kEpochMask) != L.epoch) flag = 0;
                val = w & kValueMask;
            }
            if (__all_sync(kFull, flag != 0)) break;
            ++rounds;
            // give up after kSpinLimit rounds, or at once when another CTA
            // of this launch already gave up
            const bool other = (rounds & 63u) == 0 &&
                               *reinterpret_cast<volatile unsigned int *>(L.s.flags) != 0;
            if (rounds > kSpinLimit || __any_sync(kFull, other)) {
                if (lane == 0) atomicOr(L.s.flags, 1u);
                return excl;
            }
            __nanosleep(rounds < 8 ? 32 : 256);
        }
        const uint32_t inc = __ballot_sync(kFull, flag == kFlagInclusive);
        if (inc) {
            const int l = __ffs(inc) - 1;    // nearest predecessor with a full prefix
            excl += warp_sum_u64(lane <= l ? val : 0);
            return excl;
        }
        excl += warp_sum_u64(val);
        base -= 32;
    }
}

// Copy nbytes from shared memory (4-byte aligned, readable 16 bytes past the
// end) to global dst with 16-byte aligned vector stores for the body and byte
// stores at the two unaligned edges. Called by all kThreads threads.
__device__ __forceinline__ void block_store_bytes(const uint8_t *s_src, uint8_t *dst,
                                                  uint32_t nbytes)
{
    const uint32_t tid = threadIdx.x;
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    uint32_t head = (uint32_t)((16u - (d & 15u)) & 15u);
    if (head > nbytes) head = nbytes;
    if (tid < head) dst[tid] = s_src[tid];
    const uint32_t nblk = (nbytes - head) >> 4;
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(s_src);
    for (uint32_t b = tid; b < nblk; b += kThreads) {
        const uint32_t so = head + 16u * b;
        const uint32_t *p = sw + (so >> 2);
        const uint32_t sh = (so & 3u) * 8u;
        const uint32_t w0 = p[0], w1 = p[1], w2 = p[2], w3 = p[3], w4 = p[4];
        uint4 v;
        v.x = __funnelshift_r(w0, w1, sh);
        v.y = __funnelshift_r(w1, w2, sh);
        v.z = __funnelshift_r(w2, w3, sh);
        v.w = __funnelshift_r(w3, w4, sh);
        *reinterpret_cast<uint4 *>(dst + so) = v;
    }
    const uint32_t tail0 = head + 16u * nblk;
    if (tid < nbytes - tail0) dst[tail0 + tid] = s_src[tail0 + tid];
}

// Zero the bytes of a 32-bit little-endian word whose virtual positions
// (vpos .. vpos+3) fall outside [lo, hi).
__device__ __forceinline__ uint32_t mask_word_bytes(uint32_t w, int64_t vpos, int64_t lo, int64_t hi)
{
    uint32_t keep = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (vpos + k >= lo && vpos + k < hi) keep |= 0xFFu << (8 * k);
    return w & keep;
}

// End of a launch, called by thread 0 of every CTA after its last status /
// error-word writes: count the CTA done; the last one assembles the
// gbu_result from the scan total and the first-error word, stores it, and
// resets the counters for the next launch on this scratch. Only the scan and
// error words need ordering before the done count (the output itself is not
// read by the finisher), so one thread fences, not the whole CTA.
template <bool kWrite>
__device__ __forceinline__ void finish_launch(const Launch &L, uint32_t chunk_elems)
{
    __threadfence();
    if (atomicAdd(L.s.done, 1u) != gridDim.x - 1) return;
    __threadfence();
    const uint64_t total = ld_relaxed(&L.s.status[L.num_chunks - 1]) & kValueMask;
    const uint64_t err = ld_relaxed(L.s.err);
    const unsigned int flags = atomicAdd(L.s.flags, 0u);
    int32_t st;
    uint64_t off, len;
    if (flags & 2u) {
        st = kDeviceError; off = 0; len = 0;
    } else if (flags & 1u) {
        st = kDeviceTimeout; off = 0; len = 0;
    } else if (err != ~0ull) {
        st = (int32_t)(err & 0xFF);
        off = err >> 8;
        const uint64_t c = (off + L.head) / chunk_elems;
        len = ld_relaxed(&L.s.err_prefix[c]);
    } else {
        st = (kWrite && total > L.cap) ? kOutputTooSmall : kOk;
        off = L.n;
        len = total;
    }
    volatile ResultSlot *r = L.result;
    r->status = st;
    r->reserved = 0;
    r->in_offset = off;
    r->out_len = len;
    *L.s.claim = 0;
    *L.s.done = 0;
    *L.s.flags = 0;
    st_relaxed(L.s.err, ~0ull);
    __threadfence_system();
}

// First-error key inside a CTA: position (39 bits) | kind (8 bits) | output
// units of the chunk before the error (15 bits). Positions are unique, so the
// minimum key is the first error and carries its prefix length along.
__device__ __forceinline__ uint64_t err_key(uint64_t pos, uint32_t kind, uint32_t units)
{
    return (pos << 23) | ((uint64_t)kind << 15) | (units & 0x7FFFu);
}

// Thread 0, after the look-back: publish the chunk's first error (if any)
// into the per-chunk prefix slot and the grid-wide first-error word.
__device__ __forceinline__ void publish_error(const Launch &L, uint32_t chunk, uint64_t key,
                                              uint64_t excl)
{
    if (key == ~0ull) return;
    const uint64_t pos = key >> 23;
    const uint32_t kind = (uint32_t)(key >> 15) & 0xFFu;
    L.s.err_prefix[chunk] = excl + (key & 0x7FFFu);
    atomicMin(L.s.err, (pos << 8) | kind);
}

// PTX prmt.b32 (generic mode): byte k of the result is byte sel[4k+2:4k] of
// the 8-byte value {b, a}; when sel bit 4k+3 is set, that byte's sign bit is
// replicated over the 8 bits instead. (The __byte_perm intrinsic ignores the
// sign bit of the selector, hence the inline PTX.)
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Byte-wise helpers on little-endian 32-bit words holding 4 input bytes.
// zero_bytes(v): bit 7 of every byte of v that is zero. Exact when no byte of
// v can be 0x01 directly above a zero byte (callers pass values whose bytes
// are even or multiples of 0x10); otherwise a superset, used only for flags.
__device__ __forceinline__ uint32_t zero_bytes(uint32_t v)
{
    return (v - 0x01010101u) & ~v & 0x80808080u;
}

}  // namespace gbu
