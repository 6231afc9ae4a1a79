// Device-side machinery shared by the transcoding kernel: job and item
// descriptors, block-wide scan, decoupled look-back over chunk status words,
// TMA bulk loads with mbarriers, staged coalesced stores, and per-item result
// finalisation.
//
// The paper's transcoders advance sequentially by the n_in / n_out of each
// 64-byte vector (Sec. 6.2, Eqs. for n_in and n_out; Sec. 7.3), and it sketches
// the parallel alternative of computing each segment's transcoded size first
// (Sec. 8, multithreading remark). On the GPU every chunk of an input is
// transcoded by one CTA iteration; the chunk's output offset is the exclusive
// prefix sum of the output lengths of the item's earlier chunks, obtained in
// the same pass by a decoupled look-back over per-chunk status words.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbu {

#ifndef GBU_THREADS
#define GBU_THREADS 256
#endif
constexpr int kThreads = GBU_THREADS;         // compute threads of a CTA
// Look-back warps per CTA (chunk j of a CTA is looked back by warp j % kLbWarps).
#ifndef GBU_LB_WARPS
#define GBU_LB_WARPS 1
#endif
constexpr int kLbWarps = GBU_LB_WARPS;
constexpr int kBlock = kThreads + 32 * kLbWarps + 32;   // + look-back warps and a producer warp
constexpr unsigned kFull = 0xffffffffu;

// Barrier among the kThreads compute threads only (named barrier 1), so the
// look-back warp never takes part.
__device__ __forceinline__ void cw_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}
__device__ __forceinline__ bool cw_sync_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kThreads)
        : "memory");
    return r != 0;
}

// Every chunk (the unit of work of one CTA iteration, and of the look-back)
// holds kBPT input bytes per compute thread in both directions: with 256
// compute threads and 64 bytes each, 16 KiB = 16384 UTF-8 bytes or 8192
// UTF-16 words. Thread t always owns input bytes [kBPT t, kBPT t + kBPT) of
// its chunk.
#ifndef GBU_BPT
#define GBU_BPT 48
#endif
constexpr int kBPT = GBU_BPT;
static_assert(kBPT % 16 == 0 && kBPT >= 32 && kBPT <= 64, "bytes per thread");
constexpr uint32_t kChunkBytes = kBPT * kThreads;
constexpr uint32_t kChunk8 = kChunkBytes;        // UTF-8 bytes per chunk
constexpr uint32_t kChunk16 = kChunkBytes / 2;   // UTF-16 words per chunk
// Input ring: each stage holds one chunk plus kHalo bytes on each side.
#ifndef GBU_STAGES
#define GBU_STAGES 3
#endif
constexpr int kStages = GBU_STAGES;
constexpr uint32_t kHalo = 16;
constexpr uint32_t kStageBytes = kChunkBytes + 2 * kHalo;
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
// Bounded waits: every wait gives up after a limit of global time (the job's
// wait_ns; kWaitNs when it is 0), sets the timeout flag and lets the CTA
// finish.
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s
// An mbarrier wait suspends the thread in hardware until the phase completes
// or this many nanoseconds pass, then checks the clock and waits again.
#ifndef GBU_SUSPEND_NS
#define GBU_SUSPEND_NS 20000
#endif
constexpr uint32_t kSuspendNs = GBU_SUSPEND_NS;
// Look-back rounds that find a predecessor not ready: the first few re-read
// at once (an L2 round trip paces them), later ones back off (ns).
#ifndef GBU_LB_SLEEP_SHORT
#define GBU_LB_SLEEP_SHORT 100
#endif
#ifndef GBU_LB_SLEEP_LONG
#define GBU_LB_SLEEP_LONG 500
#endif

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct ResultSlot {      // layout of gbu_result
    int32_t status;
    uint32_t reserved;
    uint64_t in_offset;
    uint64_t out_len;
};

// One input of a job.
// bit 0: input is UTF-16 (else UTF-8); bit 1: write output; bit 2: the UTF-16
// side (input or output) is big-endian
enum : uint32_t { kOpUtf16 = 1u, kOpWrite = 2u, kOpBE = 4u };
struct __align__(16) Item {   // 64 bytes, copied into shared memory in 16-byte pieces
    const uint8_t *in_al;   // 16-byte aligned base at or before the input
    uint8_t *out;           // output (UTF-16 words or UTF-8 bytes)
    uint64_t n;             // input units
    uint64_t cap;           // output capacity in units (0 when nothing is written)
    ResultSlot *result;     // device-visible result destination
    uint32_t head;          // input units between in_al and the input
    uint32_t op;            // kOpUtf16 | kOpWrite
    uint32_t chunk_base;    // global index of the item's first chunk
    uint32_t nchunks;       // chunks of this item (at least 1)
    uint32_t pad[2];
};
static_assert(sizeof(Item) == 64, "Item layout");

// A job: one persistent launch over the chunks of one or more items.
struct Job {
    const Item *items;              // device array; nullptr: the single item `item0`
    const uint32_t *chunk_item;     // per global chunk: its item (nullptr: item 0)
    Item item0;
    uint32_t num_items;
    uint32_t total_chunks;
    uint32_t status_capacity;       // status words in the scratch (cleared on epoch wrap)
    unsigned int *epoch;            // launch epoch: read at start, advanced by the last CTA
    unsigned int *chunks_done;      // chunks processed so far (summed by the CTAs on exit)
    unsigned int *claim;            // next chunk to hand out (when chunks are claimed)
    unsigned int *exit_count;       // CTAs that left the chunk loop
    unsigned int *flags;            // bit 0: a bounded wait timed out; bit 1: bad chunk id
    unsigned long long *status;     // [total_chunks] look-back words
    unsigned long long *err_prefix; // [total_chunks] output units before the chunk's first error
    unsigned long long *item_err;   // [num_items] (position << 8) | kind of the first error, ~0 if none
    unsigned int *item_done;        // [num_items] chunks written
    uint32_t validate;              // 1: validation only (no look-back; out_len reported as 0)
    uint64_t wait_ns;               // limit of every bounded wait (0: kWaitNs)
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

// Add with acquire-release semantics at GPU scope: publishes this thread's
// earlier writes with the increment and, for the thread that sees the final
// count, makes every earlier incrementer's writes visible.
__device__ __forceinline__ uint32_t atomic_add_acq_rel(unsigned int *p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
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

// Barrier among the compute threads that also counts the threads whose `v`
// is true (every thread gets the count).
__device__ __forceinline__ uint32_t cw_sync_count(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "bar.red.popc.u32 %0, 1, %2, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kThreads)
        : "memory");
    return r;
}

// Exclusive scan of one uint32 per compute thread whose barrier also counts
// the threads that raise `flag` (returned in *nflag). warp_tot must not be
// written again before every thread has passed another compute-thread
// barrier (callers alternate two arrays).
__device__ __forceinline__ uint32_t block_exclusive_scan_flag(uint32_t v, bool flag,
                                                              uint32_t *warp_tot, uint32_t *total,
                                                              uint32_t *nflag)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    *nflag = cw_sync_count(flag);
    constexpr int kWarps = kThreads / 32;
    uint32_t t = lane < kWarps ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += u;
    }
    *total = __shfl_sync(kFull, t, kWarps - 1);
    const uint32_t below = __shfl_sync(kFull, t, warp > 0 ? warp - 1 : 0);
    return (warp > 0 ? below : 0u) + inc - v;
}

// Exclusive scan of one uint32 per compute thread (kThreads threads), with
// one barrier: every warp scans its lanes and posts its total; after the
// barrier every thread adds up the totals of the warps before its own.
// Returns the thread's exclusive prefix; *total receives the block sum. The
// caller must not reuse warp_tot before another compute-thread barrier.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                         uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    cw_sync();
    // the warp totals, scanned across lanes 0 .. kWarps-1
    constexpr int kWarps = kThreads / 32;
    uint32_t t = lane < kWarps ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += u;
    }
    *total = __shfl_sync(kFull, t, kWarps - 1);
    const uint32_t below = __shfl_sync(kFull, t, warp > 0 ? warp - 1 : 0);
    return (warp > 0 ? below : 0u) + inc - v;
}

// One look-back window, already loaded: w[m] is the status word of the
// predecessor 32 m + lane places before the first one not yet summed. Sets
// *ready when every predecessor up to the nearest inclusive prefix (or the
// whole window) has published, *found when the window holds an inclusive
// prefix; returns this lane's share of the sum of values up to and including
// the nearest inclusive prefix (warp-sum it when ready).
template <int kLook>
__device__ __forceinline__ uint64_t lookback_window(const uint64_t (&w)[kLook], uint32_t epoch,
                                                    bool *ready, bool *found)
{
    const int lane = threadIdx.x & 31;
    bool rd = true, fd = false;
    uint64_t part = 0;
#pragma unroll
    for (int m = 0; m < kLook; m++) {
        if (fd) break;                               // warp-uniform
        const uint64_t x = w[m];
        const bool current = ((x >> kEpochShift) & kEpochMask) == epoch;
        const uint64_t flag = current ? x >> 62 : 0;
        const uint32_t inc = __ballot_sync(kFull, flag == kFlagInclusive);
        const uint32_t nr = __ballot_sync(kFull, flag == 0);
        // ready when no word before the nearest inclusive one is missing
        const uint32_t upto = inc ? ((inc & (0u - inc)) - 1u) : 0xFFFFFFFFu;
        if (nr & upto) rd = false;
        const uint64_t v = x & kValueMask;
        if (inc) {
            const int l = __ffs(inc) - 1;            // nearest predecessor with a full prefix
            if (lane <= l) part += v;
            fd = true;
        } else {
            part += v;
        }
    }
    *ready = rd;
    *found = fd;
    return part;
}

// The aligned middle part of block_store_bytes for a source offset of Q
// words (and `sh` bits) into each 16-byte block: a separate loop per Q, so
// the words are picked without selects.
template <int Q>
__device__ __forceinline__ void store_blocks(const uint4 *sv, uint8_t *d0, uint32_t nblk,
                                             uint32_t sh, uint32_t first, uint32_t stride)
{
    for (uint32_t b = first; b < nblk; b += stride) {
        const uint4 A = sv[b], B = sv[b + 1];                       // bytes 16b .. 16b+31
        const uint32_t x[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
        uint4 v;
        v.x = __funnelshift_r(x[Q], x[Q + 1], sh);
        v.y = __funnelshift_r(x[Q + 1], x[Q + 2], sh);
        v.z = __funnelshift_r(x[Q + 2], x[Q + 3], sh);
        v.w = __funnelshift_r(x[Q + 3], x[Q + 4], sh);
        *reinterpret_cast<uint4 *>(d0 + 16u * b) = v;
    }
}

// Copy nbytes from shared memory (16-byte aligned, readable 32 bytes past the
// end) to global dst with 16-byte aligned vector stores for the body and byte
// stores at the two unaligned edges. Each thread reads two aligned 16-byte
// blocks of the source and shifts them by the (block-uniform) misalignment,
// so the shared-memory reads are free of bank conflicts. Called by all
// kThreads compute threads.
__device__ __forceinline__ void block_store_bytes(const uint8_t *s_src, uint8_t *dst,
                                                  uint32_t nbytes)
{
    const uint32_t tid = threadIdx.x;
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    uint32_t head = (uint32_t)((16u - (d & 15u)) & 15u);
    if (head > nbytes) head = nbytes;
    if (tid < head) dst[tid] = s_src[tid];
    const uint32_t nblk = (nbytes - head) >> 4;
    const uint32_t sh = (head & 3u) * 8u;                      // same for every block
    const uint4 *sv = reinterpret_cast<const uint4 *>(s_src);
    uint8_t *d0 = dst + head;
    switch ((head >> 2) & 3u) {
    case 0: store_blocks<0>(sv, d0, nblk, sh, tid, kThreads); break;
    case 1: store_blocks<1>(sv, d0, nblk, sh, tid, kThreads); break;
    case 2: store_blocks<2>(sv, d0, nblk, sh, tid, kThreads); break;
    default: store_blocks<3>(sv, d0, nblk, sh, tid, kThreads); break;
    }
    const uint32_t tail0 = head + 16u * nblk;
    if (tid < nbytes - tail0) dst[tail0 + tid] = s_src[tail0 + tid];
}

// Zero the bytes of a 32-bit little-endian word whose virtual positions
// (vpos .. vpos+3, in bytes) fall outside [lo, hi).
__device__ __forceinline__ uint32_t mask_word_bytes(uint32_t w, int64_t vpos, int64_t lo, int64_t hi)
{
    uint32_t keep = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (vpos + k >= lo && vpos + k < hi) keep |= 0xFFu << (8 * k);
    return w & keep;
}

// First-error key inside a CTA: position (39 bits) | kind (8 bits) | output
// units of the chunk before the error (15 bits). Positions are unique, so the
// minimum key is the first error and carries its prefix length along.
__device__ __forceinline__ uint64_t err_key(uint64_t pos, uint32_t kind, uint32_t units)
{
    return (pos << 23) | ((uint64_t)kind << 15) | (units & 0x7FFFu);
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

// zero_bytes(v): bit 7 of every byte of v that is zero. Exact when no byte of
// v can be 0x01 directly above a zero byte (callers pass values whose bytes
// are even or multiples of 0x10); otherwise a superset, used only for flags.
__device__ __forceinline__ uint32_t zero_bytes(uint32_t v)
{
    return (v - 0x01010101u) & ~v & 0x80808080u;
}

// ---- mbarrier + TMA bulk copy (PTX) -------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte
// aligned), and the wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test for the completion of a phase of an mbarrier.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: if the phase is not complete, the thread
// is suspended until it completes or about hint_ns nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for a phase of an mbarrier; false when the wait gave up
// (after limit_ns of global time).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    do {
        if (mbar_try_wait_hint(bar, parity, kSuspendNs)) return true;
    } while (globaltimer_ns() - t0 < limit_ns);
    return false;
}

// Order earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) accesses by this thread.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D TMA bulk copy global -> shared, completing `bytes` on `bar`. Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- per-item result ------------------------------------------------------

// One thread, after the item's last chunk was written: assemble the
// gbu_result from the scan total and the first-error word, store it, and reset
// the item's counters for the next launch.
__device__ __forceinline__ void write_result(const Item &I, int32_t st, uint64_t off, uint64_t len,
                                             bool validate = false)
{
    if (validate) len = 0;
    // No fence: results are read once the launch has completed.
    volatile ResultSlot *r = I.result;
    r->status = st;
    r->reserved = 0;
    r->in_offset = off;
    r->out_len = len;
}

// Result of an item whose chunks are all counted (the caller's acquire made
// every chunk's status, error key and error prefix visible); resets the
// item's counters for the next launch.
__device__ __forceinline__ void finalize_item(const Job &J, uint32_t it, const Item &I)
{
    const uint64_t total =
        ld_relaxed(&J.status[I.chunk_base + I.nchunks - 1]) & kValueMask;
    const uint64_t err = ld_relaxed(&J.item_err[it]);
    const unsigned int flags = *reinterpret_cast<volatile unsigned int *>(J.flags);
    const uint32_t chunk_units = (I.op & kOpUtf16) ? kChunk16 : kChunk8;
    int32_t st;
    uint64_t off, len;
    if (flags & 2u) {
        st = kDeviceError; off = 0; len = 0;
    } else if (flags & 1u) {
        st = kDeviceTimeout; off = 0; len = 0;
    } else if (err != ~0ull) {
        st = (int32_t)(err & 0xFF);
        off = err >> 8;
        const uint64_t c = I.chunk_base + (off + I.head) / chunk_units;
        len = ld_relaxed(&J.err_prefix[c]);
    } else {
        st = ((I.op & kOpWrite) && total > I.cap) ? kOutputTooSmall : kOk;
        off = I.n;
        len = total;
    }
    write_result(I, st, off, len, J.validate != 0);
    J.item_done[it] = 0;
    st_relaxed(&J.item_err[it], ~0ull);
}

// Result of a one-chunk item straight from its chunk's aggregate and error
// key (no shared counters involved).
__device__ __forceinline__ void finalize_single(const Job &J, const Item &I, uint32_t agg,
                                                uint64_t key)
{
    const unsigned int flags = *reinterpret_cast<volatile unsigned int *>(J.flags);
    const bool v = J.validate != 0;
    if (flags & 2u)
        write_result(I, kDeviceError, 0, 0);
    else if (flags & 1u)
        write_result(I, kDeviceTimeout, 0, 0);
    else if (key != ~0ull)
        write_result(I, (int32_t)((key >> 15) & 0xFFu), key >> 23, key & 0x7FFFu, v);
    else
        write_result(I, ((I.op & kOpWrite) && agg > I.cap) ? kOutputTooSmall : kOk, I.n, agg, v);
}

}  // namespace gbu
