// Persistent, validating UTF-8 <-> UTF-16LE transcoding kernel (paper Sec. 6
// and Sec. 7) over a job of one or more inputs.
//
// Work decomposition. Every input ("item") is cut into chunks of kChunkBytes
// input bytes (kBPT bytes per compute thread; 12 KiB in the default shape of
// 256 threads x 48 bytes); the chunks of all items of a job are numbered
// globally and claimed in order from a counter by a persistent grid
// (kMinBlocks CTAs per SM). A CTA has kThreads compute threads, a producer
// warp and a look-back warp:
//   * the producer (one lane) claims each chunk just ahead of its processing
//     (once the compute warps have counted the chunk before it, so that the
//     chunks of all CTAs are processed about in the order of their numbers)
//     and loads it, with 16 bytes of context on either side, into a ring of
//     kStages shared-memory stages by a 1-D TMA bulk copy completing on the
//     stage's "full" mbarrier; a stage is refilled as soon as every compute
//     warp has arrived on its "empty" mbarrier, after the producer has
//     recorded the chunk's first error and counted the chunk done;
//   * the compute threads classify a chunk (thread t owns input bytes
//     [kBPT t, kBPT t + kBPT)), count its output and scan the counts across
//     the CTA;
//     thread 0 publishes the chunk's aggregate for the decoupled look-back;
//   * the look-back warp looks back for the chunk's offset (kLbSlots chunks
//     at a time), publishes the inclusive prefix and hands the offset back;
//   * the compute threads assemble the chunk's output into a shared-memory
//     staging buffer and write it out with 16-byte stores kDepth iterations
//     later, when its offset is long known.
// Compute warps run no look-back, TMA issue or result accounting, and meet
// at two CTA barriers per chunk: the scan's, which also tells every thread
// whether any wait gave up, and the one that frees the staging buffer after
// the write-out.
//
// Inputs of a few chunks take a one-launch cluster kernel instead (one CTA
// per chunk, the same chunk body, aggregates exchanged through distributed
// shared memory; see "One-launch path" below).
//
// Ownership: a UTF-8 unit belongs to the thread holding its end position
// (see the UTF-8 section below); a UTF-16 surrogate pair is split between
// its two words. Errors are located by the exact local rules described with
// each chunk body; the minimum (position, kind) over a chunk and then over
// the item is the sequential decoder's first error (the paper's ell).
//
// This file is the body of one kernel shape: a translation unit defines
// GBU_THREADS (compute threads), GBU_BPT (input bytes per thread and chunk),
// GBU_MIN_BLOCKS (resident CTAs per SM it is compiled for), GBU_VNS (its
// namespace) and GBU_VARIANT_FN (the name of its descriptor) and includes it.
#include "kernels.h"

namespace gbu {
namespace GBU_VNS {

namespace {

constexpr uint32_t kB7 = 0x80808080u;
constexpr int kW = kBPT / 4;     // 32-bit words a compute thread owns per chunk
constexpr int kU16 = kBPT / 2;   // UTF-16 words a compute thread owns per chunk
static_assert(kW % 4 == 0, "16-byte loads");
// Output staging per chunk: at most 2 bytes per UTF-8 input byte, 3 per
// UTF-16 input word, plus slack for the 16-byte block reads of the
// write-out.
constexpr uint32_t kOutBytes = 2 * kChunk8 > 3 * kChunk16 ? 2 * kChunk8 : 3 * kChunk16;
constexpr uint32_t kOutBuf = kOutBytes + 48;
constexpr uint32_t kWarpOutBytes = kOutBytes;   // bound of a thread's staging (one buffer)

// Positions i in [0, kBPT) (bytes or UTF-16 words counted by `unit`) with
// lo <= vt + i < hi, as a bit mask.
__device__ __forceinline__ uint64_t pos_mask(int64_t vt, int64_t lo, int64_t hi, int n)
{
    int64_t a = lo - vt, b = hi - vt;
    if (a < 0) a = 0;
    if (b > n) b = n;
    if (b <= a) return 0;
    const uint64_t upto = b >= 64 ? ~0ull : ((1ull << b) - 1ull);
    return upto & ~((1ull << a) - 1ull);
}

// ===========================================================================
// UTF-8 -> UTF-16LE chunk (paper Sec. 6)
//
// Classification (Sec. 6.1) four bytes at a time: indicator bit 7 of each
// byte for "continuation" (80-BF), ">= C0", ">= E0" and ">= F0" (the
// complement of the paper's m_1234, and m_234, m_34, m_4).
//
// Units are produced at the end positions of the sequences, as in the paper
// (Sec. 6.1-6.2): every last byte of a character, and the third byte of a
// 4-byte character, ends one UTF-16 unit, assembled from the last, second last
// and third last bytes with their tag bits stripped,
//   W = W_-2 << 12 | W_-1 << 6 | W_end   (Eq. W_sum, 16-bit),
// where W_-1 is used when the end byte is not ASCII and W_-2 when the byte two
// back is a 3/4-byte lead; high surrogates become (W >> 4) + 0xD7C0 and low
// surrogates W | 0xDC00 (Eq. W_out). Four end positions are assembled at once
// on two registers of 16-bit lanes. A position p is an end when the byte after
// it does not continue a sequence, or when it is the third byte of a 4-byte
// sequence; "continues" means a continuation byte that a lead at p-1, p-2 or
// p-3 expects (the paper's m_c), so a stray continuation byte also ends the
// valid prefix before it and the units of the valid prefix stay exact in a
// chunk that holds an error. Each position ends at most one unit.
//
// Validation (Sec. 6.4), two levels:
//  * fast, every thread: the structure check is exact (expected continuation
//    positions must equal the continuation positions: rules 2-3); bad bytes
//    and out-of-range values (rules 1, 4-6: C0/C1, F5-FF, E0+80..9F,
//    ED+A0..BF, F0+80..8F, F4+90..BF) are caught by a check that never misses
//    an error but may flag a valid word (its E0/ED and F0/F4/F5+ parts run
//    only in warps holding such bytes);
//  * exact, only in flagged threads: for every position p the rule the
//    sequential decoder applies if a character starts at p (stray
//    continuation -> TOO_LONG; C0/C1 -> OVERLONG; F5-FF -> HEADER_BITS; lead
//    without its continuations -> TOO_SHORT; then OVERLONG / SURROGATE /
//    TOO_LARGE from the value). The smallest such p is exactly where the
//    sequential decoder stops: every earlier position is a validated character
//    start or a continuation inside one.
// ===========================================================================

struct Cls {
    uint32_t c2, c3, c4, ct;   // bit 7 of each byte: >= C0, >= E0, >= F0, 80-BF
};

__device__ __forceinline__ Cls classify(uint32_t x)
{
    const uint32_t x1 = x << 1;
    Cls c;
    c.c2 = x & x1 & kB7;
    c.c3 = c.c2 & (x << 2);
    c.c4 = c.c3 & (x << 3);
    c.ct = x & ~x1 & kB7;
    return c;
}

// byte k of the result = byte k-n/8 of the 64-bit (cur:prev) (values n bytes back)
__device__ __forceinline__ uint32_t back(uint32_t prev, uint32_t cur, int n)
{
    return __funnelshift_l(prev, cur, n);
}
// byte k of the result = byte k+n/8 of (next:cur) (values n bytes ahead)
__device__ __forceinline__ uint32_t ahead(uint32_t cur, uint32_t next, int n)
{
    return __funnelshift_r(cur, next, n);
}

// 4 bits of a position mask -> bit 7 of the 4 bytes of a word.
__device__ __forceinline__ uint32_t spread4(uint32_t m4)
{
    return ((m4 * 0x00204081u) & 0x01010101u) << 7;
}

// The thread's words from the stage: w[0] = bytes -4..-1, w[1..kW] its own
// bytes, w[kW+1] = bytes kBPT..kBPT+3. Outside an interior chunk, bytes
// outside the input read as zero; *vmask gets the owned positions inside the
// input, *outside / *masked whether none / not all of them are.
struct Edge {
    uint64_t vmask;
    bool outside, masked, straddle;
};

__device__ __forceinline__ void load_words(uint32_t (&w)[kW + 2], const uint8_t *stage)
{
    const uint8_t *sp = stage + kHalo + kBPT * threadIdx.x;
#pragma unroll
    for (int q = 0; q < kW / 4; q++) {
        const uint4 a = reinterpret_cast<const uint4 *>(sp)[q];
        w[1 + 4 * q] = a.x;
        w[2 + 4 * q] = a.y;
        w[3 + 4 * q] = a.z;
        w[4 + 4 * q] = a.w;
    }
    w[0] = *reinterpret_cast<const uint32_t *>(sp - 4);
    w[kW + 1] = *reinterpret_cast<const uint32_t *>(sp + kBPT);
}

__device__ __forceinline__ void load8(uint32_t (&w)[kW + 2], const uint8_t *stage, bool interior,
                                      int64_t vt, int64_t lo, int64_t hi, Edge &e)
{
    load_words(w, stage);
    e.vmask = ~0ull;
    e.outside = e.masked = e.straddle = false;
    if (interior) return;
    e.outside = vt + kBPT <= lo || vt >= hi;
    if (e.outside) {
#pragma unroll
        for (int j = 0; j < kW + 2; j++) w[j] = 0;
        e.vmask = 0;
        e.masked = true;
        return;
    }
    if (vt < lo || vt + kBPT > hi) {   // straddles an end of the input
        e.masked = e.straddle = true;
        e.vmask = pos_mask(vt, lo, hi, kBPT);
#pragma unroll
        for (int j = 0; j < kW; j++) w[1 + j] = mask_word_bytes(w[1 + j], vt + 4 * j, lo, hi);
    }
    if (vt - 4 < lo || vt + kBPT + 4 > hi) {
        w[0] = mask_word_bytes(w[0], vt - 4, lo, hi);
        w[kW + 1] = mask_word_bytes(w[kW + 1], vt + kBPT, lo, hi);
    }
}

// Exact local rule for every owned position of a flagged thread (rare path).
// Re-reads the thread's bytes (positions -4 .. kBPT+3) from the stage and
// recomputes the end positions. Returns the key of the first error, or ~0.
__device__ __noinline__ uint64_t first_error_exact8(const uint8_t *stage, int64_t vt, int64_t lo,
                                                    int64_t hi, uint32_t t_off)
{
    const uint8_t *sp = stage + kHalo + kBPT * threadIdx.x;
    uint32_t w[kW + 2];
    for (int j = 0; j < kW + 2; j++)
        w[j] = mask_word_bytes(*reinterpret_cast<const uint32_t *>(sp - 4 + 4 * j), vt - 4 + 4 * j,
                               lo, hi);
    uint32_t units = 0;
    for (int i = 0; i < kBPT; i++) {
        const int j = (i >> 2) + 1;
        const int sh = (i & 3) * 8;
        const uint32_t xf = __funnelshift_r(w[j], w[j + 1], sh);   // bytes i .. i+3
        const uint32_t xb = __funnelshift_r(w[j - 1], w[j], sh);   // bytes i-4 .. i-1
        const uint32_t b0 = xf & 0xFFu;
        const bool valid = vt + i >= lo && vt + i < hi;
        int kind = 0;
        if ((b0 & 0xC0u) == 0x80u) {
            const uint32_t p1 = xb >> 24, p2 = (xb >> 16) & 0xFFu, p3 = (xb >> 8) & 0xFFu;
            if (!(p1 >= 0xC0u || p2 >= 0xE0u || p3 >= 0xF0u)) kind = kTooLong;
        } else if (b0 >= 0x80u) {
            if (b0 < 0xC2u) {
                kind = kOverlong;
            } else if (b0 >= 0xF5u) {
                kind = kHeaderBits;
            } else {
                const uint32_t len = b0 < 0xE0u ? 2u : (b0 < 0xF0u ? 3u : 4u);
                const uint32_t c = (xf ^ 0x80808080u) & 0xC0C0C0C0u;   // zero byte: continuation
                const uint32_t need = len == 2 ? 0x0000FF00u : (len == 3 ? 0x00FFFF00u : 0xFFFFFF00u);
                if (c & need) {
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
        if (kind != 0 && valid) return err_key((uint64_t)(vt + i - lo), kind, t_off + units);
        // position i ends a unit when the next byte does not continue a
        // sequence (a continuation expected by a lead at i, i-1 or i-2), or
        // when i is the third byte of a 4-byte sequence
        const uint32_t n1 = (xf >> 8) & 0xFFu;                     // byte i+1
        const uint32_t bm1 = xb >> 24, bm2 = (xb >> 16) & 0xFFu;  // bytes i-1, i-2
        const bool n1_cont = (n1 & 0xC0u) == 0x80u;
        const bool expected = b0 >= 0xC0u || bm1 >= 0xE0u || bm2 >= 0xF0u;
        const bool ends = !(n1_cont && expected) || bm2 >= 0xF0u;
        if (valid && ends) units++;
    }
    return ~0ull;
}

// Phase 2 reuses phase 1's end positions (kept in registers) or recomputes
// them from the words.
#ifndef GBU_CARRY_ENDS
#define GBU_CARRY_ENDS 1
#endif
constexpr bool kCarryEnds = GBU_CARRY_ENDS != 0;

struct St8 {
    uint32_t end[kCarryEnds ? kW : 1];   // end-position indicators (bit 7 of each byte)
    uint32_t bad;      // the fast check fired
    bool skip;         // the whole warp lies outside the input (warp-uniform)
    bool warp3, warp4; // the warp holds >= E0 / >= F0 leads (warp-uniform)
};

// One pass over the thread's words: classification, the exact structure
// check, the C0/C1 check, the value checks of 3- and 4-byte leads, and the
// end positions (Sec. 6.1, 6.4); returns the thread's unit count. k3 / k4:
// the warp holds >= E0 / >= F0 leads (else their terms are zero and dropped).
template <bool k3, bool k4>
__device__ __forceinline__ uint32_t structure8(const uint32_t (&w)[kW + 2], uint32_t (&end)[kW],
                                               bool wmasked, uint64_t vmask, uint32_t &bad)
{
    Cls cp = classify(w[0]);
    if (!k3) cp.c3 = 0;
    if (!k4) cp.c4 = 0;
    uint32_t ec_prev = 0, c4_pp = 0, cnt = 0;
#pragma unroll
    for (int j = 1; j <= kW + 1; j++) {
        const uint32_t x = w[j];
        Cls c = classify(x);
        if (!k3) c.c3 = 0;
        if (!k4) c.c4 = 0;
        uint32_t exp;
        if (j <= kW) {
            exp = back(cp.c2, c.c2, 8);
            if (k3) exp |= back(cp.c3, c.c3, 16);
            if (k4) exp |= back(cp.c4, c.c4, 24);
            bad |= exp ^ c.ct;
            // C0 / C1: leads >= C0 whose low 7 bits are below 0x42 (no carry
            // crosses a byte: 0x7F + 0x3E < 0x100)
            const uint32_t x7 = x & 0x7F7F7F7Fu;
            bad |= c.c2 & ~(x7 + 0x3E3E3E3Eu);
            if (k3 || k4) {
                const uint32_t y = ahead(x, w[j + 1], 8);   // the next byte of each position
                if (k3) {
                    // E0 + 80..9F (overlong), ED + A0..BF (surrogate): a byte
                    // that is E0 when bit 5 of the next byte is clear, or ED
                    // when it is set
                    const uint32_t y5 = y << 2;
                    const uint32_t m = ((y5 >> 7) & 0x01010101u) * 0x0Du;
                    bad |= zero_bytes(x ^ 0xE0E0E0E0u ^ m);
                }
                if (k4) {
                    // F0 + 80..8F (overlong), F4 + 90..BF (too large): a byte
                    // that is F0 when bits 5 and 4 of the next byte are clear,
                    // or F4 when one is set; and F5..FF (the low 7 bits reach
                    // 0x80 when 0x0B is added)
                    const uint32_t y54 = (y << 2) | (y << 3);
                    const uint32_t m = (y54 >> 5) & 0x04040404u;
                    bad |= zero_bytes(x ^ 0xF0F0F0F0u ^ m);
                    bad |= (x7 + 0x0B0B0B0Bu) & x & kB7;
                }
            }
        } else {
            // continuations the last leads expect at positions kBPT.. kBPT+2
            exp = cp.c2 >> 24;
            if (k3) exp |= cp.c3 >> 16;
            if (k4) exp |= cp.c4 >> 8;
            bad |= exp & ~c.ct;
        }
        const uint32_t ec = exp & c.ct;
        if (j >= 2) {   // the end positions of word j-1
            uint32_t e = ~ahead(ec_prev, ec, 8);
            if (k4) e |= back(c4_pp, cp.c4, 16);
            e &= kB7;
            if (wmasked) e &= spread4((uint32_t)(vmask >> (4 * (j - 2))) & 0xFu);
            end[j - 2] = e;
            cnt += __popc(e);
        }
        c4_pp = cp.c4;
        ec_prev = ec;
        cp = c;
    }
    return cnt;
}

// Load, classify, check, count units. Returns the thread's count.
__device__ __forceinline__ uint32_t chunk8_phase1(St8 &st, const uint8_t *stage, bool interior,
                                                  int64_t vt, int64_t lo, int64_t hi)
{
    uint32_t w[kW + 2];
    Edge e;
    load8(w, stage, interior, vt, lo, hi, e);
    st.bad = 0;
    st.skip = false;
    if (!interior) {
        // a warp wholly outside the input (the tail of an item's last chunk)
        // skips the chunk body
        st.skip = __all_sync(kFull, e.outside);
        if (st.skip) {
            st.warp3 = st.warp4 = false;
#pragma unroll
            for (int j = 0; j < (kCarryEnds ? kW : 1); j++) st.end[j] = 0;
            return 0;
        }
    }
    // some thread of the warp masks its end positions (warp-uniform, so the
    // unmasked warps branch around that work instead of predicating it)
    const bool wmasked = !interior && __any_sync(kFull, e.masked);
    // leads >= E0 (3/4-byte) and >= F0 anywhere in the warp, the look-behind
    // word included: without them the pass below drops their terms
    uint32_t a3 = 0, a4 = 0;
#pragma unroll
    for (int j = 0; j <= kW; j++) {
        const uint32_t x3 = w[j] & (w[j] << 1) & (w[j] << 2);
        a3 |= x3;
        a4 |= x3 & (w[j] << 3);
    }
    st.warp3 = __any_sync(kFull, (a3 & kB7) != 0);
    st.warp4 = __any_sync(kFull, (a4 & kB7) != 0);
    uint32_t bad = 0, cnt, end[kW];
    if (st.warp4)
        cnt = structure8<true, true>(w, end, wmasked, e.vmask, bad);
    else if (st.warp3)
        cnt = structure8<true, false>(w, end, wmasked, e.vmask, bad);
    else
        cnt = structure8<false, false>(w, end, wmasked, e.vmask, bad);
    st.bad = bad;
    if (kCarryEnds) {
#pragma unroll
        for (int j = 0; j < kW; j++) st.end[kCarryEnds ? j : 0] = end[j];
    }
    return cnt;
}

// End positions of a thread whose words passed the fast check (phase 2
// recomputes them word by word instead of keeping them in registers across
// chunks): every continuation byte of its words is then expected, so a
// position ends a unit when the next byte is not a continuation or when it is
// the third byte of a 4-byte sequence; the byte after its last position
// counts as a continuation only where the thread's last leads expect it (a
// stray continuation there is the next thread's error, and the valid prefix
// ends before it). Called for words j = 1 .. kW in order.
template <bool k3, bool k4>
struct EndsValid {
    const uint32_t (&w)[kW + 2];
    const bool wmasked;
    const uint64_t vmask;
    uint32_t ct, c4_prev;
    static __device__ __forceinline__ uint32_t cont(uint32_t x) { return x & ~(x << 1) & kB7; }
    static __device__ __forceinline__ uint32_t ge_f0(uint32_t x)
    {
        return x & (x << 1) & (x << 2) & (x << 3) & kB7;
    }
    __device__ __forceinline__ EndsValid(const uint32_t (&w_)[kW + 2], bool wm, uint64_t vm)
        : w(w_), wmasked(wm), vmask(vm)
    {
        c4_prev = k4 ? ge_f0(w[0]) : 0u;
        ct = cont(w[1]);
    }
    __device__ __forceinline__ uint32_t operator()(int j)
    {
        const uint32_t x = w[j];
        uint32_t ct_next;
        if (j < kW) {
            ct_next = cont(w[j + 1]);
        } else {
            const uint32_t c2 = x & (x << 1) & kB7;
            uint32_t exp = c2 >> 24;
            if (k3) {
                const uint32_t c3 = c2 & (x << 2);
                exp |= c3 >> 16;
                if (k4) exp |= (c3 & (x << 3)) >> 8;
            }
            ct_next = exp & cont(w[kW + 1]);
        }
        const uint32_t c4 = k4 ? ge_f0(x) : 0u;
        uint32_t e = ~ahead(ct, ct_next, 8);
        if (k4) e |= back(c4_prev, c4, 16);
        e &= kB7;
        if (wmasked) e &= spread4((uint32_t)(vmask >> (4 * (j - 1))) & 0xFu);
        ct = ct_next;
        c4_prev = c4;
        return e;
    }
};

// End positions from an array (the exact ones of structure8).
struct EndsArray {
    const uint32_t (&end)[kW];
    __device__ __forceinline__ uint32_t operator()(int j) const { return end[j - 1]; }
};

// Units at the end positions (Eq. W_sum, W_out), four positions at a time on
// two registers of 16-bit lanes, stored at p in order. k3 / k4: the warp
// holds 3- or 4-byte leads (4-byte leads are also >= E0, so k4 implies k3).
template <bool k3, bool k4, bool kBE, typename EndFn>
__device__ __forceinline__ void assemble8(const uint32_t (&w)[kW + 2], EndFn end_of, uint16_t *p)
{
    uint32_t s_prev, c3_prev = 0, c4_prev = 0;
    {
        const uint32_t x = w[0];
        const uint32_t na = prmt(x, 0, 0xBA98);
        s_prev = x & ~(na & 0xC0C0C0C0u);
        // >= E0 / >= F0 at bit 7 of each byte (the other bits are not used:
        // the masks below replicate bit 7)
        if (k3) c3_prev = x & (x << 1) & (x << 2);
        if (k4) c4_prev = c3_prev & (x << 3);
    }
#pragma unroll
    for (int j = 1; j <= kW; j++) {
        const uint32_t x = w[j];
        const uint32_t na = prmt(x, 0, 0xBA98);            // 0xFF where byte >= 0x80
        const uint32_t s = x & ~(na & 0xC0C0C0C0u);         // tag bits stripped
        uint32_t c3 = 0, c4 = 0;
        if (k3) c3 = x & (x << 1) & (x << 2);
        if (k4) c4 = c3 & (x << 3);
        const uint32_t s1 = back(s_prev, s, 8) & na;        // W_-1 where the end byte is not ASCII
        uint32_t wa = prmt(s, 0, 0x4140) + (prmt(s1, 0, 0x4140) << 6);
        uint32_t wb = prmt(s, 0, 0x4342) + (prmt(s1, 0, 0x4342) << 6);
        if (k3) {
            // W_-2 (low 4 bits) where the byte two back is a 3/4-byte lead
            const uint32_t m3 = prmt(c3_prev, c3, 0xDCBA);
            const uint32_t s2 = back(s_prev, s, 16) & m3 & 0x0F0F0F0Fu;
            wa += prmt(s2, 0, 0x4140) << 12;
            wb += prmt(s2, 0, 0x4342) << 12;
        }
        if (k4) {
            // surrogates: high at the third byte of a 4-byte sequence,
            // low at its fourth byte (Eq. W_out)
            const uint32_t hma = prmt(c4_prev, c4, 0xBBAA);
            const uint32_t hmb = prmt(c4_prev, c4, 0xDDCC);
            const uint32_t lma = prmt(c4_prev, c4, 0xAA99);
            const uint32_t lmb = prmt(c4_prev, c4, 0xCCBB);
            const uint32_t ha = ((wa >> 4) & 0x0FFF0FFFu) + 0xD7C0D7C0u;
            const uint32_t hb = ((wb >> 4) & 0x0FFF0FFFu) + 0xD7C0D7C0u;
            wa = ((ha & hma) | (wa & ~hma)) | (lma & 0xDC00DC00u);
            wb = ((hb & hmb) | (wb & ~hmb)) | (lmb & 0xDC00DC00u);
        }
        if (kBE) {   // UTF-16BE output
            wa = prmt(wa, 0, 0x2301);
            wb = prmt(wb, 0, 0x2301);
        }
        const uint32_t e = end_of(j);
        if (e & 0x00000080u) *p++ = (uint16_t)wa;
        if (e & 0x00008000u) *p++ = (uint16_t)(wa >> 16);
        if (e & 0x00800000u) *p++ = (uint16_t)wb;
        if (e & 0x80000000u) *p++ = (uint16_t)(wb >> 16);
        s_prev = s;
        c3_prev = c3;
        c4_prev = c4;
    }
}

// A thread the fast check flagged (rare; kept out of line so that it costs
// the common path no registers): the exact first error, and the units of the
// valid prefix at their exact end positions (a stray continuation ends the
// valid prefix before it).
template <bool kWrite, bool kBE>
__device__ __noinline__ void exact8(const uint8_t *stage, bool interior, int64_t vt, int64_t lo,
                                    int64_t hi, uint32_t t_off, bool wmasked, uint16_t *p,
                                    unsigned long long *s_err)
{
    const uint64_t key = first_error_exact8(stage, vt, lo, hi, t_off);
    if (key != ~0ull) atomicMin(s_err, key);
    if (!kWrite) return;
    uint32_t w[kW + 2], end[kW], b = 0;
    Edge e;
    load8(w, stage, interior, vt, lo, hi, e);
    structure8<true, true>(w, end, wmasked, e.vmask, b);
    assemble8<true, true, kBE>(w, EndsArray{end}, p);
}

// Phase 2 of a thread: exact first error (flagged threads) and staging of the
// units at p. t_off: the thread's output offset in the chunk (for the error
// key).
template <bool kWrite, bool kBE>
__device__ __forceinline__ void chunk8_phase2(const St8 &st, const uint8_t *stage, bool interior,
                                              uint16_t *p, uint32_t t_off, int64_t vt, int64_t lo,
                                              int64_t hi, unsigned long long *s_err)
{
    if (st.skip) return;
    if (!kWrite) {
        // Threads straddling an end of the input see the bytes outside it
        // as zeros (ASCII), which neither create nor hide an error inside
        // it, so the fast check covers them as well.
        if (st.bad) exact8<false, kBE>(stage, interior, vt, lo, hi, t_off, false, p, s_err);
        return;
    }
    uint32_t w[kW + 2];
    Edge e;
    load8(w, stage, interior, vt, lo, hi, e);
    const bool wmasked = !interior && __any_sync(kFull, e.masked);
    if (st.bad) {
        exact8<true, kBE>(stage, interior, vt, lo, hi, t_off, wmasked, p, s_err);
        return;
    }
    // the 3/4-byte parts only in warps that hold such leads (warp-uniform)
    if (kCarryEnds) {
        const uint32_t(&end)[kW] = reinterpret_cast<const uint32_t(&)[kW]>(st.end);
        if (st.warp4)
            assemble8<true, true, kBE>(w, EndsArray{end}, p);
        else if (st.warp3)
            assemble8<true, false, kBE>(w, EndsArray{end}, p);
        else
            assemble8<false, false, kBE>(w, EndsArray{end}, p);
    } else if (st.warp4) {
        assemble8<true, true, kBE>(w, EndsValid<true, true>(w, wmasked, e.vmask), p);
    } else if (st.warp3) {
        assemble8<true, false, kBE>(w, EndsValid<true, false>(w, wmasked, e.vmask), p);
    } else {
        assemble8<false, false, kBE>(w, EndsValid<false, false>(w, wmasked, e.vmask), p);
    }
}

// ===========================================================================
// UTF-16LE -> UTF-8 chunk (paper Sec. 7)
//
// Output length per word (Sec. 7, plan of attack): 1 byte below U+0080, 2
// below U+0800, 3 for other BMP words, and 2 for each half of a surrogate
// pair: the pair's 4 bytes are split between its two words (the high one
// holds the code point's bits 20-12, the low one, with the high word's
// last 2 bits, bits 11-0), so that no word depends on the word after it and
// a pair that crosses a thread or chunk boundary needs no special case.
// Counted two words at a time on 16-bit lanes.
//
// Paths: like the paper's fast paths (Sec. 7.1), each warp picks one from its
// own words: all below U+0800 (1-2 byte encoder), no surrogates (1-3 byte
// encoder) - neither needs validation - or the general path with the
// sequencing check of Sec. 7.4: a high surrogate not followed by a low one
// is LONE_HIGH at the high, a low surrogate not preceded by a high one is
// LONE_LOW at the low.
//
// Encoding (Fig. 1(a), Sec. 7.2-7.3): the 6-bit groups of the code point get
// the tag bits C0/E0/F0 (lead) and 80 (continuation); for a pair, the code
// point is 0x10000 + ((hi & 3FF) << 10) + (lo & 3FF), so its bits 20-10 are
// (hi & 3FF) + 0x40.
// ===========================================================================

__device__ __forceinline__ uint32_t ge80_lanes(uint32_t w)    // word >= 0x0080, bit 15 per lane
{
    return (((w & 0x7F807F80u) + 0x7F807F80u) | w) & 0x80008000u;
}
__device__ __forceinline__ uint32_t ge800_lanes(uint32_t w)   // word >= 0x0800
{
    return (((w & 0x78007800u) + 0x78007800u) | w) & 0x80008000u;
}
__device__ __forceinline__ uint32_t surr_lanes(uint32_t w)    // D800-DFFF (exact: low 11 bits zero)
{
    const uint32_t v = (w & 0xF800F800u) ^ 0xD800D800u;
    return (v - 0x00010001u) & ~v & 0x80008000u;
}

__device__ __forceinline__ uint32_t lane16(const uint32_t *w, int i)   // word i, i in [-2, kU16 + 2)
{
    return (w[(i + 2) >> 1] >> (16 * ((i + 2) & 1))) & 0xFFFFu;
}

// 1-2 byte encoder (Sec. 7.1): 110LKJHG 10FEDCBA from 00000LKJHGFEDCBA.
__device__ __forceinline__ uint32_t enc2(uint32_t u)
{
    return (((u << 8) | (u >> 6)) & 0x3F3Fu) | 0x80C0u;
}

// 3-byte encoder: 1110RQPN 10MLKJHG 10FEDCBA.
__device__ __forceinline__ uint32_t enc3(uint32_t u)
{
    return (u >> 12) | ((u << 2) & 0x3F00u) | ((u << 16) & 0x3F0000u) | 0x8080E0u;
}

struct St16 {
    uint32_t vmask;    // owned words inside the input
    bool slow;         // the thread straddles an end of the input
    bool skip;         // the whole warp lies outside the input (warp-uniform)
    bool sur, only12;  // the warp holds surrogates / only words below U+0800 (warp-uniform)
};

__device__ __forceinline__ uint32_t unit_keep(int64_t u, int64_t lo, int64_t hi)
{
    return (u >= lo && u < hi) ? 0xFFFFu : 0u;
}

// The thread's words (two UTF-16 words each) from the stage, as for load8:
// w[0] = words -2, -1; w[1..kW] its own; w[kW+1] = words kU16, kU16+1.
// Words outside the input read as zero; UTF-16BE words are byte-swapped.
template <bool kBE>
__device__ __forceinline__ void load16(uint32_t (&w)[kW + 2], const uint8_t *stage, bool interior,
                                       int64_t vt, int64_t lo, int64_t hi, Edge &e)
{
    load_words(w, stage);
    e.vmask = kU16 >= 32 ? 0xFFFFFFFFull : ((1ull << kU16) - 1ull);
    e.outside = e.masked = e.straddle = false;
    if (!interior) {
        e.outside = vt + kU16 <= lo || vt >= hi;
        if (e.outside) {
#pragma unroll
            for (int j = 0; j < kW + 2; j++) w[j] = 0;
            e.vmask = 0;
            e.masked = true;
        } else {
            if (vt < lo || vt + kU16 > hi) {   // straddles an end of the input
                e.straddle = e.masked = true;
                e.vmask = pos_mask(vt, lo, hi, kU16);
#pragma unroll
                for (int j = 0; j < kW; j++)
                    w[1 + j] &= unit_keep(vt + 2 * j, lo, hi) | (unit_keep(vt + 2 * j + 1, lo, hi) << 16);
            }
            if (vt - 2 < lo || vt + kU16 + 2 > hi) {
                w[0] &= unit_keep(vt - 2, lo, hi) | (unit_keep(vt - 1, lo, hi) << 16);
                w[kW + 1] &= unit_keep(vt + kU16, lo, hi) | (unit_keep(vt + kU16 + 1, lo, hi) << 16);
            }
        }
    }
    if (kBE) {   // UTF-16BE: swap the bytes of every word once, then as UTF-16LE
#pragma unroll
        for (int j = 0; j < kW + 2; j++) w[j] = prmt(w[j], 0, 0x2301);
    }
}

template <bool kBE>
__device__ __forceinline__ uint32_t chunk16_phase1(St16 &st, const uint8_t *stage, bool interior,
                                                   int64_t vt, int64_t lo, int64_t hi)
{
    uint32_t w[kW + 2];
    Edge e;
    load16<kBE>(w, stage, interior, vt, lo, hi, e);
    st.vmask = (uint32_t)e.vmask;
    st.skip = false;
    st.slow = e.straddle;
    if (!interior) {
        // threads wholly outside the input count nothing; a warp wholly
        // outside skips the chunk body
        st.skip = __all_sync(kFull, e.outside);
        if (st.skip) {
            st.slow = st.sur = st.only12 = false;
            return 0;
        }
    }
    // some thread of the warp counts only part of its words (warp-uniform)
    const bool wmasked = !interior && __any_sync(kFull, e.masked);
    // does the warp hold words of U+0800 and above? (warp-uniform; words
    // outside the input are zero)
    uint32_t top5 = 0;
#pragma unroll
    for (int j = 0; j < kW; j++) top5 |= w[1 + j] & 0xF800F800u;
    st.only12 = !__any_sync(kFull, top5 != 0);
    // per word: 1 + [>=80] + [>=800] - [surrogate]: 1-3 bytes, 2 for either
    // half of a pair
    uint32_t cnt = 0, anysur = 0;
    if (!wmasked && st.only12) {
        cnt = kU16;
#pragma unroll
        for (int j = 0; j < kW; j++) cnt += __popc(ge80_lanes(w[1 + j]));
    } else if (!wmasked) {
        cnt = kU16;
#pragma unroll
        for (int j = 0; j < kW; j++) {
            const uint32_t x = w[1 + j];
            const uint32_t ga = ge80_lanes(x), gb = ge800_lanes(x), s = surr_lanes(x);
            cnt += __popc(ga) + __popc(gb) - __popc(s);
            anysur |= s;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kW; j++) {
            const uint32_t x = w[1 + j];
            const uint32_t ga = ge80_lanes(x), gb = ge800_lanes(x), s = surr_lanes(x);
            const uint32_t vm = (((st.vmask >> (2 * j)) & 1u) << 15) | (((st.vmask >> (2 * j + 1)) & 1u) << 31);
            cnt += __popc(vm) + __popc(ga & vm) + __popc(gb & vm) - __popc(s & vm);
            anysur |= s;
        }
    }
    st.sur = __any_sync(kFull, anysur != 0);
    return cnt;
}

// UTF-8 bytes of the thread's words, two at a time on 16-bit lanes
// (Fig. 1(a)): lead F (the word itself, C0 | u >> 6, or E0 | u >> 12),
// second byte S (80 | u & 3F, or 80 | (u >> 6) & 3F in the 3-byte form) and
// third byte T (80 | u & 3F); each word stores its 1-3 bytes at p.
// A surrogate pair's 4 bytes (Sec. 7.3) are split between its halves, 2
// each: with U = (high & 3FF) + 40 (the code point >> 10), the high
// surrogate stores F0 | U >> 8 and 80 | (U >> 2) & 3F, the low one
// 80 | (high & 3) << 4 | (low >> 6) & F and 80 | low & 3F.
// kSur: the words may hold surrogates (validly paired; the pair may cross
// into the next thread, the low half then stores its 2 bytes there).
template <bool kSur>
__device__ __forceinline__ void encode_bmp(const uint32_t (&w)[kW + 2], uint8_t *p)
{
#pragma unroll
    for (int j = 1; j <= kW; j++) {
        const uint32_t x = w[j];
        const uint32_t m2 = prmt(ge80_lanes(x), 0, 0xBB99);     // 0xFFFF on lanes >= 0x80
        uint32_t m3 = prmt(ge800_lanes(x), 0, 0xBB99);          // 0xFFFF on lanes >= 0x800
        const uint32_t t = (x & 0x003F003Fu) | 0x00800080u;
        const uint32_t x6 = x >> 6;
        uint32_t f = (((x6 & 0x001F001Fu) | 0x00C000C0u) & m2) | (x & ~m2);
        f = ((((x >> 12) & 0x000F000Fu) | 0x00E000E0u) & m3) | (f & ~m3);
        uint32_t s = (((x6 & 0x003F003Fu) | 0x00800080u) & m3) | (t & ~m3);
        if (kSur) {
            const uint32_t sr = surr_lanes(x);
            const uint32_t ms = prmt(sr, 0, 0xBB99);             // surrogate lanes
            const uint32_t ml = prmt(sr & (x << 5), 0, 0xBB99);  // low-surrogate lanes
            const uint32_t hu = (x & 0x03FF03FFu) + 0x00400040u;  // U of a high surrogate
            const uint32_t fh = ((hu >> 8) & 0x00070007u) | 0x00F000F0u;
            const uint32_t sh = ((hu >> 2) & 0x003F003Fu) | 0x00800080u;
            const uint32_t prev = __funnelshift_l(w[j - 1], x, 16);   // the word before each lane
            const uint32_t fl = ((prev & 0x00030003u) << 4) | (x6 & 0x000F000Fu) | 0x00800080u;
            f = (((fl & ml) | (fh & ~ml)) & ms) | (f & ~ms);
            s = (((t & ml) | (sh & ~ml)) & ms) | (s & ~ms);
            m3 &= ~ms;                                            // surrogates store 2 bytes
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const bool c2 = (m2 >> (16 * h)) & 1u, c3 = (m3 >> (16 * h)) & 1u;
            p[0] = (uint8_t)(f >> (16 * h));
            if (c2) p[1] = (uint8_t)(s >> (16 * h));
            if (c3) p[2] = (uint8_t)(t >> (16 * h));
            p += 1 + (c2 ? 1 : 0) + (c3 ? 1 : 0);
        }
    }
}

// Validation and staging of the thread's bytes at obuf (output offset t_off
// in the chunk; obuf holds the chunk's bytes from offset wb). The warp-uniform
// flags come from phase 1; the per-thread ones are recomputed from the input
// edges.
template <bool kWrite, bool kBE>
__device__ __forceinline__ void chunk16_phase2(St16 st, const uint8_t *stage, bool interior,
                                               uint8_t *obuf, uint32_t t_off, uint32_t wb, int64_t vt,
                                               int64_t lo, int64_t hi, unsigned long long *s_err)
{
    if (st.skip) return;
    uint32_t w[kW + 2];
    Edge e;
    load16<kBE>(w, stage, interior, vt, lo, hi, e);
    st.vmask = (uint32_t)e.vmask;
    st.slow = e.straddle;
    if (st.vmask == 0) return;   // nothing of the input here
    if (!kWrite && !st.sur && !st.slow) return;   // valid and nothing to write
    bool slow = st.slow;
    if (st.sur && !slow) {
        // sequencing (Sec. 7.4): a word is a low surrogate exactly when the
        // word before it is a high one; a thread where this fails for one of
        // its words, or for the word after its last, takes the exact path
        // below
        auto hi_lanes = [](uint32_t x) { return surr_lanes(x) & ~(x << 5); };
        auto lo_lanes = [](uint32_t x) { return surr_lanes(x) & (x << 5); };
        uint32_t v = 0, h_prev = hi_lanes(w[0]);
#pragma unroll
        for (int j = 1; j <= kW; j++) {
            const uint32_t h = hi_lanes(w[j]);
            v |= __funnelshift_l(h_prev, h, 16) ^ lo_lanes(w[j]);
            h_prev = h;
        }
        v |= (h_prev ^ (lo_lanes(w[kW + 1]) << 16)) & 0x80000000u;
        slow = v != 0;
    }
    if (!slow) {
        // every word of this thread is valid
        if (!kWrite) return;
        uint8_t *p = obuf + (t_off - wb);
        if (st.sur) {
            encode_bmp<true>(w, p);
        } else if (st.only12) {
#pragma unroll
            for (int i = 0; i < kU16; i++) {
                const uint32_t u = lane16(w, i);
                const bool big = u >= 0x80u;
                const uint32_t v = big ? enc2(u) : u;
                p[0] = (uint8_t)v;
                if (big) p[1] = (uint8_t)(v >> 8);
                p += big ? 2 : 1;
            }
        } else {
            encode_bmp<false>(w, p);
        }
        return;
    }
    uint64_t key = ~0ull;
    uint32_t o = t_off;
#pragma unroll
    for (int i = 0; i < kU16; i++) {
        const uint32_t u = lane16(w, i), pv = lane16(w, i - 1), nx = lane16(w, i + 1);
        const bool is_hi = (u & 0xFC00u) == 0xD800u;
        const bool is_lo = (u & 0xFC00u) == 0xDC00u;
        uint32_t kind = 0;
        if (is_hi && (nx & 0xFC00u) != 0xDC00u) kind = kLoneHigh;
        if (is_lo && (pv & 0xFC00u) != 0xD800u) kind = kLoneLow;
        const bool c2 = u >= 0x80u, c3 = u >= 0x800u;
        const uint32_t len = (is_hi || is_lo) ? 2u : 1u + (c2 ? 1u : 0u) + (c3 ? 1u : 0u);
        uint32_t v;
        if (is_hi) {            // the first 2 bytes of the pair's 4
            const uint32_t hu = (u & 0x3FFu) + 0x40u;
            v = (0xF0u | (hu >> 8)) | ((0x80u | ((hu >> 2) & 0x3Fu)) << 8);
        } else if (is_lo) {     // the last 2
            v = (0x80u | ((pv & 3u) << 4) | ((u >> 6) & 0xFu)) | ((0x80u | (u & 0x3Fu)) << 8);
        } else {
            v = c3 ? enc3(u) : (c2 ? enc2(u) : u);
        }
        if ((st.vmask >> i) & 1u) {
            if (kWrite && o - wb + len <= kWarpOutBytes) {
                uint8_t *q = obuf + (o - wb);
                q[0] = (uint8_t)v;
                if (len >= 2) q[1] = (uint8_t)(v >> 8);
                if (len >= 3) q[2] = (uint8_t)(v >> 16);
            }
            if (kind != 0 && key == ~0ull) key = err_key((uint64_t)(vt + i - lo), kind, o);
            o += len;
        }
    }
    if (key != ~0ull) atomicMin(s_err, key);
}

// ===========================================================================
// The persistent kernel
// ===========================================================================

struct Ring {
    uint64_t full[kStages];        // mbarrier per stage: TMA completion (producer)
    uint64_t empty[kStages];       // mbarrier per stage: every compute warp is done with it
    Item item[kStages];
    uint32_t chunk[kStages], end[kStages];
};

// What the warps know of one chunk of this CTA (slot: the chunk's number in
// the CTA's sequence, modulo kSlots), from its load to its accounting.
struct ChunkRec {
    uint64_t excl;               // look-back warp: output units of the item before the chunk
    unsigned long long err;      // compute threads (phase 2): first-error key, ~0 if none
    uint8_t *out;                // producer: the item's output, capacity, operation
    uint64_t cap;
    uint32_t op;
    uint32_t chunk, chunk_base, nchunks, itidx;   // producer
    uint32_t agg;                // compute thread 0: the chunk's output units
    uint32_t end;                // producer / compute thread 0: no chunk here
};

// A chunk to load: its global number, its item and the item's descriptor.
struct Next {
    uint32_t c, it;
    Item I;
};

// Producer lane: the descriptor of global chunk c (two dependent global reads
// in a batch, none for one item), fetched ahead of the load where possible.
__device__ __forceinline__ Next describe(const Job &J, uint32_t c)
{
    Next n;
    n.c = c;
    n.it = 0;
    if (c < J.total_chunks) {
        n.it = J.chunk_item ? J.chunk_item[c] : 0u;
        n.I = J.items ? J.items[n.it] : J.item0;
    }
    return n;
}

// Producer lane: load chunk n.c into stage `slot` and describe it in `rec`.
// Returns false (and marks the stage and the record as the end) when the job
// is exhausted.
__device__ __forceinline__ bool produce(const Job &J, const Next &n, int slot, uint8_t *stages,
                                        Ring &R, ChunkRec &rec)
{
    rec.err = ~0ull;
    const uint32_t c = n.c, it = n.it;
    if (c >= J.total_chunks) {
        rec.end = 1;
        R.end[slot] = 1;
        mbar_arrive(&R.full[slot]);
        return false;
    }
    const Item &I = n.I;
    rec.out = I.out;
    rec.cap = I.cap;
    rec.op = I.op;
    rec.chunk = c;
    rec.chunk_base = I.chunk_base;
    rec.nchunks = I.nchunks;
    rec.itidx = it;
    rec.end = 0;
    R.item[slot] = I;
    R.chunk[slot] = c;
    R.end[slot] = 0;
    const int64_t ub = (I.op & kOpUtf16) ? 2 : 1;
    const int64_t v0b = (int64_t)(c - I.chunk_base) * kChunkBytes;   // virtual byte offset
    const int64_t endb = (((int64_t)I.head + (int64_t)I.n) * ub + 15) & ~(int64_t)15;
    int64_t lo_b = v0b - (int64_t)kHalo;
    if (lo_b < 0) lo_b = 0;
    int64_t hi_b = v0b + (int64_t)(kChunkBytes + kHalo);
    if (hi_b > endb) hi_b = endb;
    uint8_t *dst = stages + (size_t)slot * kStageBytes + (lo_b - (v0b - (int64_t)kHalo));
    fence_proxy_async_smem();
    if (hi_b > lo_b) {
        mbar_arrive_expect_tx(&R.full[slot], (uint32_t)(hi_b - lo_b));
        tma_load_1d(dst, I.in_al + lo_b, (uint32_t)(hi_b - lo_b), &R.full[slot]);
    } else {
        mbar_arrive(&R.full[slot]);
    }
    return true;
}

// Every CTA adds the chunks it processed to the job's chunk counter; the last
// CTA out checks that they add up to the job's chunks (a counter left dirty by
// an aborted launch shows here), advances the epoch and resets the job's
// counters for the next launch.
__device__ __forceinline__ void exit_job(const Job &J, uint32_t epoch, uint32_t processed)
{
    atomicAdd(J.chunks_done, processed);
    __threadfence();
    if (atomicAdd(J.exit_count, 1u) != gridDim.x - 1) return;
    __threadfence();   // every other CTA's accounting is visible
    if (!J.items) finalize_item(J, 0, J.item0);
    const unsigned int chunks = atomicExch(J.chunks_done, 0u);
    *J.claim = 0;
    const unsigned int flags = atomicAdd(J.flags, 0u);
    if (chunks != J.total_chunks || flags != 0) {
        // counters were left dirty by an aborted launch, or a wait gave up
        // (chunks may have been skipped, items left unfinished): no item was
        // finished reliably
        const int32_t st = (flags & 1u) ? kDeviceTimeout : kDeviceError;
        for (uint32_t it = 0; it < J.num_items; it++) {
            const Item &X = J.items ? J.items[it] : J.item0;
            volatile ResultSlot *r = X.result;
            r->status = st;
            r->reserved = 0;
            r->in_offset = 0;
            r->out_len = 0;
        }
    }
    const uint32_t next = (epoch + 1) & kEpochMask;
    if (next == 0)   // wrap: stale words of epoch 0 must not look ready
        for (uint32_t i = 0; i < J.status_capacity; i++) J.status[i] = 0;
    *J.epoch = next;
    *J.exit_count = 0;
    *J.flags = 0;
    __threadfence_system();
}

// A chunk staged in iteration i is written out in iteration i + kDepth, so
// its offset has kDepth iterations to arrive; kDepth staging buffers.
#ifndef GBU_DEPTH
#define GBU_DEPTH 2
#endif
constexpr int kDepth = GBU_DEPTH;
static_assert(kStages >= 2, "stages: one in use, at least one loading");
// Chunk records (chunk j of the CTA uses slot j % kSlots): live from the
// chunk's load (kStages chunks ahead of its phase 1) to its accounting.
constexpr int kSlots = 16;
static_assert(kSlots >= kStages + kDepth + kLbWarps + 2, "chunk records");

// How chunks are dealt to CTAs: 0 round-robin (CTA b takes chunks b, b +
// grid, ...); 1 claimed from a counter when a stage frees; 2 as 1, except
// that transcoding claims a chunk once the CTA's previous chunk is counted.
#ifndef GBU_CLAIM
#define GBU_CLAIM 2
#endif
constexpr int kClaim = GBU_CLAIM;

// Look-backs a look-back warp runs at once. One: with chunks claimed just
// ahead of their processing, a chunk's predecessors have published by the
// time its look-back starts, and the warp's shortest round trip per chunk
// wins (two at once: 4 % slower over the eight 1 GiB cases).
#ifndef GBU_LB_SLOTS
#define GBU_LB_SLOTS 1
#endif
constexpr int kLbSlots = GBU_LB_SLOTS;

// kIn: the input encoding of every item when known at launch (1 UTF-8, 2
// UTF-16; the other direction's code is then not in the kernel), 0 any.
template <bool kWrite, int kLook, bool kAnyBE, int kIn = 0>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
transcode_kernel(const Job J)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    uint8_t *const stages = dyn_smem;
    uint8_t *const obufs = dyn_smem + kStages * kStageBytes;   // kDepth output staging buffers
    __shared__ __align__(16) Ring R;
    __shared__ __align__(8) uint64_t pend_bar[kSlots], excl_bar[kSlots], lb_exit;
    __shared__ ChunkRec s_rec[kSlots];
    __shared__ uint32_t s_warp[2][kThreads / 32 + 1];
    __shared__ uint32_t s_epoch;

    const uint32_t tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&R.full[s], 1);
            mbar_init(&R.empty[s], kThreads / 32);
        }
        for (int s = 0; s < kSlots; s++) {
            mbar_init(&pend_bar[s], 1);
            mbar_init(&excl_bar[s], 1);
        }
        mbar_init(&lb_exit, kLbWarps);
        fence_mbar_init();
        s_epoch = *reinterpret_cast<volatile unsigned int *>(J.epoch);
    }
    __syncthreads();
    const uint32_t epoch = s_epoch;
    const uint64_t wlim = J.wait_ns ? J.wait_ns : kWaitNs;   // limit of every bounded wait

    if (tid >= kThreads + 32 * kLbWarps) {
        // ---- producer warp (lane 0): refill the ring, account for chunks ----
        if (tid != kThreads + 32 * kLbWarps) return;
        bool producing = true, ok = true;
        // Transcoding claims a chunk just ahead of its processing, once the
        // CTA's previous chunk is counted: the chunks of all CTAs are then
        // processed about in the order of their numbers, so that look-backs
        // rarely wait for a late predecessor. Validation and length-only
        // calls (short per-chunk work, no offsets to wait for) claim a chunk
        // as soon as a stage frees, its descriptor fetched ahead.
        const bool late = kClaim == 2 && kWrite && !J.validate;
        // the next chunk of this CTA: round-robin (CTA b takes chunks b,
        // b + grid, ...) or claimed from the job's counter
        auto next_chunk = [&](uint32_t n) -> uint32_t {
            if (kClaim == 0) return blockIdx.x + n * gridDim.x;
            return atomicAdd(J.claim, 1u);
        };
        uint32_t np = 0;   // chunks produced (the end marker included)
        for (int s = 0; s < kStages && producing; s++, np++)
            producing = produce(J, describe(J, next_chunk(np)), s, stages, R, s_rec[np % kSlots]);
        Next nx{};
        if (producing && !late) nx = describe(J, next_chunk(np));
        // a multi-chunk item's done count comes back one step later (the
        // atomic's round trip overlaps the next wait); its last chunk
        // finishes the item's result
        bool pend = false;
        uint32_t pend_old = 0, pend_it = 0, pend_n = 0;
        auto settle = [&]() {
            if (pend && pend_old == pend_n - 1) finalize_item(J, pend_it, J.items[pend_it]);
            pend = false;
        };
        if (!producing)   // the other look-back warps stop at the next records
            for (int m = 1; m < kLbWarps; m++) s_rec[(np - 1 + m) % kSlots].end = 1;
        // chunk j's first error and offset are known once its stage is
        // released: record them, count the chunk done, finish its item's
        // result when it is the item's last chunk (a one-item job is finished
        // by its last CTA); then refill the stage
        uint32_t j = 0;
        for (; producing || j + 1 < np; j++) {
            if (!mbar_wait(&R.empty[j % kStages], (j / kStages) & 1u, wlim) ||
                !mbar_wait(&excl_bar[j % kSlots], (j / kSlots) & 1u, wlim)) {
                ok = false;
                break;
            }
            settle();
            const ChunkRec &r = s_rec[j % kSlots];
            const uint64_t key = *reinterpret_cast<const volatile unsigned long long *>(&r.err);
            if (!J.items) {
                if (key != ~0ull) {
                    J.err_prefix[r.chunk] = r.excl + (key & 0x7FFFu);
                    atomicMin(&J.item_err[0], ((key >> 23) << 8) | ((key >> 15) & 0xFFu));
                }
            } else if (r.nchunks == 1) {
                finalize_single(J, J.items[r.itidx], r.agg, key);
            } else {
                if (key != ~0ull) {
                    J.err_prefix[r.chunk] = r.excl + (key & 0x7FFFu);
                    atomicMin(&J.item_err[r.itidx], ((key >> 23) << 8) | ((key >> 15) & 0xFFu));
                }
                pend_old = atomic_add_acq_rel(&J.item_done[r.itidx], 1u);
                pend_it = r.itidx;
                pend_n = r.nchunks;
                pend = true;
            }
            if (producing) {
                if (late) {
                    if (!mbar_wait(&pend_bar[(np - 1) % kSlots], ((np - 1) / kSlots) & 1u, wlim)) {
                        ok = false;
                        break;
                    }
                    nx = describe(J, next_chunk(np));
                }
                producing = produce(J, nx, (int)(j % kStages), stages, R, s_rec[np % kSlots]);
                np++;
                if (producing && !late) nx = describe(J, next_chunk(np));
                if (!producing)
                    for (int m = 1; m < kLbWarps; m++) s_rec[(np - 1 + m) % kSlots].end = 1;
            }
        }
        settle();
        if (!ok) atomicOr(J.flags, 1u);
        // the look-back warps are done (every inclusive prefix is out)
        if (!mbar_wait(&lb_exit, 0, wlim)) atomicOr(J.flags, 1u);
        exit_job(J, epoch, j);
        return;
    }
    if (tid >= kThreads) {
        // ---- look-back warps: warp p handles this CTA's chunks j = p (mod kLbWarps)
        // Once chunk j is counted (and its aggregate published): the
        // look-back, the inclusive prefix published and the offset handed
        // back. Up to kLbSlots look-backs run at once: every
        // round loads the windows of all of them before checking any, so that
        // one L2 round trip serves them all, and a chunk whose predecessors
        // have not all published yet does not hold up the chunks after it.
        constexpr int kSl = kLook * kLbSlots <= 8 ? kLbSlots : (8 / kLook > 0 ? 8 / kLook : 1);
        const uint32_t p = (tid - kThreads) >> 5;
        const bool lead = lane == 0;
        const uint64_t start_word = pack_status(kFlagInclusive, epoch, 0);
        bool failed = false, ending = false;
        uint32_t next = p, live = 0;
        uint32_t s_j[kSl], s_chunk[kSl], s_base0[kSl], s_agg[kSl];
        int64_t s_pos[kSl];    // next predecessor to read (index in the item)
        uint64_t s_acc[kSl];   // sum of the predecessors read so far
#pragma unroll
        for (int m = 0; m < kSl; m++) {
            s_j[m] = s_chunk[m] = s_base0[m] = s_agg[m] = 0;
            s_pos[m] = 0;
            s_acc[m] = 0;
        }
        uint64_t t_idle = 0;
        uint32_t idle_rounds = 0;
        auto finish = [&](uint32_t j, uint64_t excl) {
            __syncwarp();
            if (lead) {
                s_rec[j % kSlots].excl = excl;
                mbar_arrive(&excl_bar[j % kSlots]);
            }
        };
        while (true) {
            // admit the chunks counted since the last round (waiting only
            // when nothing else is in flight)
            while (!ending && __popc(live) < kSl) {
                const int q = next % kSlots;
                const uint32_t par = (next / kSlots) & 1u;
                const bool ready = live == 0 ? __all_sync(kFull, mbar_wait(&pend_bar[q], par, wlim))
                                             : __all_sync(kFull, mbar_test(&pend_bar[q], par));
                if (!ready) {
                    if (live == 0) failed = true;
                    break;
                }
                const ChunkRec &r = s_rec[q];
                if (r.end) {
                    ending = true;
                    break;
                }
                const uint32_t agg = r.agg;
                const uint32_t k = r.chunk - r.chunk_base;
                if (k == 0 || J.validate) {   // validation needs no offsets
                    finish(next, 0);
                } else {
                    const int m = __ffs(~live) - 1;
#pragma unroll
                    for (int mm = 0; mm < kSl; mm++)
                        if (mm == m) {
                            s_j[mm] = next;
                            s_chunk[mm] = r.chunk;
                            s_base0[mm] = r.chunk_base;
                            s_agg[mm] = agg;
                            s_pos[mm] = (int64_t)k - 1;
                            s_acc[mm] = 0;
                        }
                    live |= 1u << m;
                }
                next += kLbWarps;
            }
            if (failed || (live == 0 && ending)) break;
            if (live == 0) continue;
            // one round for every look-back in flight: all loads, then checks
            uint64_t w[kSl][kLook];
#pragma unroll
            for (int m = 0; m < kSl; m++) {
                if (!((live >> m) & 1u)) continue;
#pragma unroll
                for (int i = 0; i < kLook; i++) {
                    const int64_t idx = s_pos[m] - 32 * i - (int64_t)lane;
                    w[m][i] = idx >= 0 ? ld_relaxed(&J.status[s_base0[m] + idx]) : start_word;
                }
            }
            bool progress = false;
#pragma unroll
            for (int m = 0; m < kSl; m++) {
                if (!((live >> m) & 1u)) continue;
                bool ready, found;
                const uint64_t part = lookback_window<kLook>(w[m], epoch, &ready, &found);
                if (!ready) continue;
                progress = true;
                s_acc[m] += warp_sum_u64(part);
                if (found) {
                    if (lead)
                        st_relaxed(&J.status[s_chunk[m]],
                                   pack_status(kFlagInclusive, epoch, s_acc[m] + s_agg[m]));
                    finish(s_j[m], s_acc[m]);
                    live &= ~(1u << m);
                } else {
                    s_pos[m] -= 32 * kLook;
                }
            }
            if (progress) {
                t_idle = 0;
                idle_rounds = 0;
            } else {
                // back off while predecessors are late (the first rounds
                // re-read at once: an L2 round trip paces them)
                if (++idle_rounds > 2) __nanosleep(idle_rounds < 16 ? GBU_LB_SLEEP_SHORT : GBU_LB_SLEEP_LONG);
                // predecessors not ready: give up after the wait limit without
                // progress, or as soon as another CTA of the launch gave up
                const uint64_t now = globaltimer_ns();
                if (t_idle == 0) t_idle = now;
                const bool stop = now - t_idle > wlim ||
                                  *reinterpret_cast<volatile unsigned int *>(J.flags) != 0;
                if (__any_sync(kFull, stop)) {
                    failed = true;
                    break;
                }
            }
        }
        if (lead) {
            if (failed) atomicOr(J.flags, 1u);
            mbar_arrive(&lb_exit);
        }
        return;
    }

    // ---- compute warps ------------------------------------------------------
    // write out chunk jd (staging buffer jd % kDepth) once its offset is known;
    // false if the wait for the offset gave up
    auto write_out = [&](uint32_t jd) -> bool {
        const int q = jd % kSlots;
        if (!mbar_wait(&excl_bar[q], (jd / kSlots) & 1u, wlim)) return false;
        const ChunkRec &r = s_rec[q];
        const uint64_t excl = r.excl;
        if (excl < r.cap) {
            const bool u16 = (r.op & kOpUtf16) != 0;
            const uint32_t ub = u16 ? 1u : 2u;                       // output unit bytes
            uint64_t nw = r.agg;
            if (nw > r.cap - excl) nw = r.cap - excl;
            if (nw * ub > kOutBytes) nw = kOutBytes / ub;
            block_store_bytes(obufs + (size_t)(jd % kDepth) * kOutBuf, r.out + excl * ub,
                              (uint32_t)(nw * ub));
        }
        return true;
    };

    uint32_t iter = 0;
    bool failed = false;
    while (true) {
        const int slot = iter % kStages;
        const bool okw = mbar_wait(&R.full[slot], (iter / kStages) & 1u, wlim);
        const bool end = okw && R.end[slot] != 0;
        const bool live = okw && !end;
        const uint8_t *stage = stages + (size_t)slot * kStageBytes;
        Item I{};
        uint32_t c = 0;
        if (live) {
            I = R.item[slot];
            c = R.chunk[slot];
        }
        const int64_t lo = I.head, hi = (int64_t)I.head + (int64_t)I.n;
        const uint32_t k = c - I.chunk_base;
        const bool u16 = kIn == 2 || (kIn == 0 && (I.op & kOpUtf16) != 0);
        const bool be = kAnyBE && (I.op & kOpBE);
        bool interior;
        int64_t vt;
        uint32_t cnt = 0;
        St8 s8;
        St16 s16;
        if (u16) {
            const int64_t v0 = (int64_t)k * kChunk16;
            interior = v0 - 2 >= lo && v0 + (int64_t)kChunk16 + 2 <= hi;
            vt = v0 + (int64_t)kU16 * tid;
            if (live) cnt = be ? chunk16_phase1<true>(s16, stage, interior, vt, lo, hi)
                               : chunk16_phase1<false>(s16, stage, interior, vt, lo, hi);
        } else {
            const int64_t v0 = (int64_t)k * kChunk8;
            interior = v0 - 4 >= lo && v0 + (int64_t)kChunk8 + 4 <= hi;
            vt = v0 + (int64_t)kBPT * tid;
            if (live) cnt = chunk8_phase1(s8, stage, interior, vt, lo, hi);
        }
        // the scan's barrier also tells every thread whether a wait gave up
        // (here, or in thread 0's previous hand-over)
        uint32_t agg, nfail;
        const uint32_t t_off =
            block_exclusive_scan_flag(cnt, !okw || failed, s_warp[iter & 1], &agg, &nfail);
        if (nfail) {
            failed = true;
            break;
        }
        if (end) break;
        const int q = iter % kSlots;
        if (tid == 0) {
            // publish the chunk's aggregate at once (the look-backs of later
            // chunks, in every CTA, wait for it; a chunk at the start of its
            // item is its own inclusive prefix) and hand the count to its
            // look-back warp
            st_relaxed(&J.status[c], pack_status(k == 0 ? kFlagInclusive : kFlagAggregate, epoch, agg));
            s_rec[q].agg = agg;
            mbar_arrive(&pend_bar[q]);
        }
        if (kWrite && iter >= (uint32_t)kDepth) {
            const bool ok2 = write_out(iter - kDepth);
            // the staging buffer is free once every thread has written it out
            if (cw_sync_count(!ok2)) {
                failed = true;
                iter++;
                break;
            }
        }
        uint8_t *obuf = obufs + (size_t)(iter % kDepth) * kOutBuf;
        unsigned long long *err = &s_rec[q].err;
        if (u16) {
            if (be) chunk16_phase2<kWrite, true>(s16, stage, interior, obuf, t_off, 0, vt, lo, hi, err);
            else chunk16_phase2<kWrite, false>(s16, stage, interior, obuf, t_off, 0, vt, lo, hi, err);
        } else {
            uint16_t *pu = reinterpret_cast<uint16_t *>(obuf) + t_off;
            if (be) chunk8_phase2<kWrite, true>(s8, stage, interior, pu, t_off, vt, lo, hi, err);
            else chunk8_phase2<kWrite, false>(s8, stage, interior, pu, t_off, vt, lo, hi, err);
        }
        // this warp is done with the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[slot]);
        iter++;
    }
    // iter chunks were handed over; the end (or a failure) goes to every
    // look-back warp as hand-overs iter .. iter + kLbWarps - 1
    if (tid == 0) {
        for (uint32_t h = iter; h < iter + kLbWarps; h++) {
            s_rec[h % kSlots].end = 1;
            mbar_arrive(&pend_bar[h % kSlots]);
        }
        if (failed) atomicOr(J.flags, 1u);
    }
    // drain: write out the last kDepth chunks (unless any thread failed)
    if (kWrite && cw_sync_count(failed) == 0) {
        for (int m = kDepth; m > 0; m--) {
            if (iter < (uint32_t)m) continue;
            const bool ok2 = write_out(iter - m);
            if (cw_sync_count(!ok2)) break;
        }
    }
}

// ===========================================================================
// One-launch path for inputs of a few chunks
//
// An input of at most kSmallMaxChunks chunks is converted by one thread-block
// cluster with one CTA per chunk and no persistent machinery: each CTA loads
// its chunk (with the same 16 bytes of context on either side) by plain
// 16-byte loads, runs the chunk body of the persistent kernel (phase 1, the
// CTA scan, phase 2 into shared memory), and learns the output offset of its
// chunk from the aggregates of the chunks before it, which every CTA writes
// into the shared memory of every CTA of the cluster before the cluster
// barrier. The first error and the result are gathered the same way in CTA 0.
// Nothing is kept in global memory between launches (no status words,
// counters or fences), and there is no wait other than the two hardware
// cluster barriers.
// ===========================================================================

__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}
// Store into the shared memory of CTA `rank` of the cluster, at the address
// that `local` has in this CTA.
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_u32(const void *local, uint32_t rank, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr(local, rank)), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_u64(const void *local, uint32_t rank, uint64_t v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(cluster_addr(local, rank)), "l"(v) : "memory");
}

constexpr size_t kSmallSmem = (size_t)kStageBytes + kOutBuf;

// Static shared memory of a one-launch CTA (the same layout in every CTA of
// a cluster, which the distributed shared-memory stores rely on).
struct SmallSmem {
    uint32_t warp[kThreads / 32 + 1];
    uint32_t agg[kSmallMaxChunks];              // every chunk's output units
    unsigned long long key[kSmallMaxChunks];    // CTA 0: every chunk's first error
    unsigned long long err;
};

// Chunk k of nct (the CTA's rank in its cluster) of item I: load, the chunk
// body, the aggregates and first errors through the cluster, the output and
// (CTA 0) the result. `validate`: the validation-only form (out_len 0).
template <bool kWrite, bool kBE>
__device__ __forceinline__ void small_body(const Item &I, uint32_t k, uint32_t nct,
                                           uint32_t validate, SmallSmem &S, uint8_t *stage,
                                           uint8_t *obuf)
{
    uint32_t *const s_warp = S.warp;
    uint32_t *const s_agg = S.agg;
    unsigned long long *const s_key = S.key;
    unsigned long long &s_err = S.err;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) s_err = ~0ull;
    const bool u16 = (I.op & kOpUtf16) != 0;
    // the window of the persistent kernel's TMA load (16-byte aligned, whole
    // 16-byte blocks)
    {
        const int64_t ub = u16 ? 2 : 1;
        const int64_t v0b = (int64_t)k * kChunkBytes;
        const int64_t endb = (((int64_t)I.head + (int64_t)I.n) * ub + 15) & ~(int64_t)15;
        int64_t lo_b = v0b - (int64_t)kHalo;
        if (lo_b < 0) lo_b = 0;
        int64_t hi_b = v0b + (int64_t)(kChunkBytes + kHalo);
        if (hi_b > endb) hi_b = endb;
        uint8_t *dst = stage + (lo_b - (v0b - (int64_t)kHalo));
        for (int64_t b = lo_b + 16 * (int64_t)tid; b < hi_b; b += 16 * kThreads)
            *reinterpret_cast<uint4 *>(dst + (b - lo_b)) =
                __ldg(reinterpret_cast<const uint4 *>(I.in_al + b));
    }
    __syncthreads();
    const int64_t lo = I.head, hi = (int64_t)I.head + (int64_t)I.n;
    bool interior;
    int64_t vt;
    uint32_t cnt;
    St8 s8;
    St16 s16;
    if (u16) {
        const int64_t v0 = (int64_t)k * kChunk16;
        interior = v0 - 2 >= lo && v0 + (int64_t)kChunk16 + 2 <= hi;
        vt = v0 + (int64_t)kU16 * tid;
        cnt = chunk16_phase1<kBE>(s16, stage, interior, vt, lo, hi);
    } else {
        const int64_t v0 = (int64_t)k * kChunk8;
        interior = v0 - 4 >= lo && v0 + (int64_t)kChunk8 + 4 <= hi;
        vt = v0 + (int64_t)kBPT * tid;
        cnt = chunk8_phase1(s8, stage, interior, vt, lo, hi);
    }
    uint32_t agg, nflag;
    const uint32_t t_off = block_exclusive_scan_flag(cnt, false, s_warp, &agg, &nflag);
    if (nct > 1) {
        // the chunk's aggregate into every CTA of the cluster (the barrier
        // completes while phase 2 runs)
        if (tid == 0)
            for (uint32_t r = 0; r < nct; r++) st_cluster_u32(&s_agg[k], r, agg);
        cluster_arrive_release();
    }
    if (u16) {
        chunk16_phase2<kWrite, kBE>(s16, stage, interior, obuf, t_off, 0, vt, lo, hi, &s_err);
    } else {
        uint16_t *pu = reinterpret_cast<uint16_t *>(obuf) + t_off;
        chunk8_phase2<kWrite, kBE>(s8, stage, interior, pu, t_off, vt, lo, hi, &s_err);
    }
    uint64_t excl = 0, total = agg;
    if (nct > 1) {
        cluster_wait_acquire();
        total = 0;
        for (uint32_t r = 0; r < nct; r++) {
            if (r == k) excl = total;
            total += s_agg[r];
        }
    }
    __syncthreads();   // the staged output and the chunk's first error are complete
    if (kWrite && excl < I.cap) {
        const uint32_t ub = u16 ? 1u : 2u;   // output unit bytes
        uint64_t nw = agg;
        if (nw > I.cap - excl) nw = I.cap - excl;
        block_store_bytes(obuf, I.out + excl * ub, (uint32_t)(nw * ub));
    }
    uint64_t key = s_err;
    uint64_t prefix = excl;   // output units before the chunk holding the first error
    if (nct > 1) {
        // every chunk's first error into CTA 0 (its output units counted
        // from the chunk's start; CTA 0 adds the chunks before it)
        if (tid == 0) st_cluster_u64(&s_key[k], 0, key);
        cluster_arrive_release();
        cluster_wait_acquire();
        if (k != 0) return;
        key = ~0ull;
        uint64_t run = 0;
        for (uint32_t r = 0; r < nct; r++) {
            if (s_key[r] != ~0ull) {   // chunks hold increasing positions
                key = s_key[r];
                prefix = run;
                break;
            }
            run += s_agg[r];
        }
    }
    if (tid != 0) return;
    const bool v = validate != 0;
    if (key != ~0ull)
        write_result(I, (int32_t)((key >> 15) & 0xFFu), key >> 23, prefix + (key & 0x7FFFu), v);
    else
        write_result(I, ((I.op & kOpWrite) && total > I.cap) ? kOutputTooSmall : kOk, I.n, total, v);
}

// Grid = cluster = the item's chunks (1 .. kSmallMaxChunks); CTA k converts
// chunk k. `validate`: the validation-only form (out_len reported as 0).
template <bool kWrite, bool kBE>
__global__ void __launch_bounds__(kThreads, 1) small_kernel(const Item I, uint32_t validate)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ SmallSmem S;
    small_body<kWrite, kBE>(I, blockIdx.x, gridDim.x, validate, S, dyn_smem, dyn_smem + kStageBytes);
}

// A batch's one-chunk items, one CTA each (no cluster, no scratch): CTA b
// converts items[b] and writes its result. kAnyBE: some item is UTF-16BE.
template <bool kWrite, bool kAnyBE>
__global__ void __launch_bounds__(kThreads, 1) small_items_kernel(const Item *items)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ SmallSmem S;
    const Item I = items[blockIdx.x];
    if (kAnyBE && (I.op & kOpBE))
        small_body<kWrite, true>(I, 0, 1, 0, S, dyn_smem, dyn_smem + kStageBytes);
    else
        small_body<kWrite, false>(I, 0, 1, 0, S, dyn_smem, dyn_smem + kStageBytes);
}

template <bool W>
const void *small_fn(bool be)
{
    return be ? reinterpret_cast<const void *>(&small_kernel<W, true>)
              : reinterpret_cast<const void *>(&small_kernel<W, false>);
}

template <bool W>
const void *small_items_fn(bool any_be)
{
    return any_be ? reinterpret_cast<const void *>(&small_items_kernel<W, true>)
                  : reinterpret_cast<const void *>(&small_items_kernel<W, false>);
}

int g_max_per_sm[64] = {0};
int g_sms[64] = {0};

}  // namespace

size_t job_smem_bytes(bool write)
{
    return (size_t)kStages * kStageBytes + (write ? (size_t)kDepth * kOutBuf : 0);
}

// Every instantiation of the kernel: (write, look-back width, whether any
// item is UTF-16BE; the UTF-16LE-only kernels carry no byte-order code; for
// little-endian transcoding of one encoding at the default look-back width,
// kernels with that encoding's code only, half the code to fetch).
#ifndef GBU_DIR_SPLIT
#define GBU_DIR_SPLIT 1
#endif
template <bool W, int L>
const void *kernel_fn(bool be, int in)
{
    if constexpr (W && L == GBU_DEFAULT_LOOK && GBU_DIR_SPLIT) {
        if (!be && in == 1) return reinterpret_cast<const void *>(&transcode_kernel<W, L, false, 1>);
        if (!be && in == 2) return reinterpret_cast<const void *>(&transcode_kernel<W, L, false, 2>);
    }
    return be ? reinterpret_cast<const void *>(&transcode_kernel<W, L, true>)
              : reinterpret_cast<const void *>(&transcode_kernel<W, L, false>);
}

// in: 1 / 2 when every item's input is UTF-8 / UTF-16, else 0
const void *kernel_for(bool write, int look, bool be, int in = 0)
{
    switch (look) {
    case 1: return write ? kernel_fn<true, 1>(be, in) : kernel_fn<false, 1>(be, in);
    case 2: return write ? kernel_fn<true, 2>(be, in) : kernel_fn<false, 2>(be, in);
    case 8: return write ? kernel_fn<true, 8>(be, in) : kernel_fn<false, 8>(be, in);
    case 16: return write ? kernel_fn<true, 16>(be, in) : kernel_fn<false, 16>(be, in);
    default: return write ? kernel_fn<true, 4>(be, in) : kernel_fn<false, 4>(be, in);
    }
}

int job_max_ctas_per_sm(int device)
{
    if (device < 0 || device >= 64) return 0;
    if (g_max_per_sm[device]) return g_max_per_sm[device];
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    for (const int look : kLookWidths)
        for (int w = 0; w < 2; w++)
            for (int be = 0; be < 2; be++)
                for (int in = 0; in < 3; in++)
                    if (cudaFuncSetAttribute(kernel_for(w != 0, look, be != 0, in),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)job_smem_bytes(w != 0)) != cudaSuccess)
                        return 0;
    for (int be = 0; be < 2; be++)
        if (cudaFuncSetAttribute(small_fn<true>(be != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmallSmem) != cudaSuccess ||
            cudaFuncSetAttribute(small_fn<false>(be != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmallSmem) != cudaSuccess ||
            cudaFuncSetAttribute(small_items_fn<true>(be != 0),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem) != cudaSuccess ||
            cudaFuncSetAttribute(small_items_fn<false>(be != 0),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem) != cudaSuccess)
            return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel_for(true, GBU_DEFAULT_LOOK, false), kBlock,
                                                      job_smem_bytes(true)) != cudaSuccess ||
        per < 1)
        per = 1;
    g_sms[device] = sms;
    g_max_per_sm[device] = per;
    return per;
}

int job_grid(int device, const Tune &t)
{
    const int per = job_max_ctas_per_sm(device);
    if (per <= 0) return 0;
    const int use = t.ctas_per_sm > 0 && t.ctas_per_sm < per ? t.ctas_per_sm : per;
    return g_sms[device] * use;
}

cudaError_t launch_job(const Job &J, bool write, int grid, cudaStream_t stream, int look, bool be,
                       int in)
{
    void *args[] = {const_cast<Job *>(&J)};
    return cudaLaunchKernel(kernel_for(write, look, be, in), dim3(grid), dim3(kBlock), args,
                            job_smem_bytes(write), stream);
}

cudaError_t launch_small(const Item &I, bool write, bool validate, cudaStream_t stream)
{
    const uint32_t nct = I.nchunks;
    if (nct < 1 || nct > (uint32_t)kSmallMaxChunks) return cudaErrorInvalidValue;
    if (kSmallSmem > 48 * 1024) {   // the attribute is set once per device
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || job_max_ctas_per_sm(dev) <= 0)
            return cudaErrorInvalidValue;
    }
    const void *fn = write ? small_fn<true>((I.op & kOpBE) != 0) : small_fn<false>((I.op & kOpBE) != 0);
    Item item = I;
    uint32_t v = validate ? 1u : 0u;
    void *args[] = {&item, &v};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nct);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmallSmem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nct;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = nct > 1 ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_small_items(const Item *items, uint32_t count, bool write, bool any_be,
                               cudaStream_t stream)
{
    if (count == 0) return cudaSuccess;
    if (kSmallSmem > 48 * 1024) {   // the attribute is set once per device
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || job_max_ctas_per_sm(dev) <= 0)
            return cudaErrorInvalidValue;
    }
    const void *fn = write ? small_items_fn<true>(any_be) : small_items_fn<false>(any_be);
    const Item *arg = items;
    void *args[] = {&arg};
    return cudaLaunchKernel(fn, dim3(count), dim3(kThreads), args, kSmallSmem, stream);
}

Item make_item(const void *in, uint64_t n, bool utf16, void *out, uint64_t cap, bool write,
               ResultSlot *result, uint32_t chunk_base, bool big_endian)
{
    Item I{};
    const uintptr_t p = reinterpret_cast<uintptr_t>(in);
    if (n == 0) {
        I.in_al = nullptr;
        I.head = 0;
    } else {
        I.in_al = reinterpret_cast<const uint8_t *>(p & ~(uintptr_t)15u);
        I.head = (uint32_t)(utf16 ? (p & 15u) >> 1 : (p & 15u));
    }
    I.n = n;
    I.out = static_cast<uint8_t *>(out);
    I.cap = write ? cap : 0;
    I.result = result;
    I.op = (utf16 ? kOpUtf16 : 0u) | (write ? kOpWrite : 0u) | (big_endian ? kOpBE : 0u);
    I.chunk_base = chunk_base;
    const uint64_t units = utf16 ? kChunk16 : kChunk8;
    const uint64_t nch = n ? (I.head + n + units - 1) / units : 1;
    I.nchunks = (uint32_t)nch;
    return I;
}

}  // namespace GBU_VNS

const Variant &GBU_VARIANT_FN()
{
    static const Variant v = {kThreads,
                              kBPT,
                              kMinBlocks,
                              kChunkBytes,
                              &GBU_VNS::make_item,
                              &GBU_VNS::job_smem_bytes,
                              &GBU_VNS::job_max_ctas_per_sm,
                              &GBU_VNS::job_grid,
                              &GBU_VNS::launch_job,
                              &GBU_VNS::launch_small,
                              &GBU_VNS::launch_small_items};
    return v;
}

}  // namespace gbu
