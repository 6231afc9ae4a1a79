// Persistent, validating UTF-8 <-> UTF-16LE transcoding kernel (paper Sec. 6
// and Sec. 7) over a job of one or more inputs.
//
// Work decomposition. Every input ("item") is cut into 8 KiB chunks; the
// chunks of all items of a job are numbered globally and handed out in order
// by an atomic counter. A persistent grid (a few CTAs per SM) loops over them:
//   * thread 0 claims chunks ahead and loads each one, with 16 bytes of
//     context on either side, into a ring of kStages shared-memory stages by
//     a 1-D TMA bulk copy completing on the stage's mbarrier;
//   * the 256 threads classify the chunk (thread t owns bytes [32t, 32t+32)),
//     count its output, scan the counts across the CTA and publish the
//     chunk's aggregate for the decoupled look-back;
//   * a ninth warp looks back for the chunk's offset as soon as its aggregate
//     is out and publishes the inclusive prefix;
//   * the compute threads assemble the chunk's output into one of kDepth
//     shared-memory staging buffers and write it out with 16-byte stores
//     kDepth iterations later, when its offset is long known.
// The compute warps thus practically never wait on a look-back, and the TMA
// ring loads the next chunk while the current one is processed.
//
// Ownership: a UTF-8 unit belongs to the thread holding its end position
// (see chunk8 below); a UTF-16 surrogate pair belongs to the owner of its
// high surrogate. Errors are located by the exact local rules described with
// each chunk body; the minimum (position, kind) over a chunk and then over
// the item is the sequential decoder's first error (the paper's ell).
#include "kernels.h"

namespace gbu {

namespace {

constexpr uint32_t kB7 = 0x80808080u;

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

// Exact local rule for every owned position of a flagged thread (rare path).
// Re-reads the thread's bytes (positions -4 .. 35) from the stage and
// recomputes the end positions, so the hot path keeps its words in
// registers. Returns the key of the first error, or ~0.
__device__ __noinline__ uint64_t first_error_exact8(const uint8_t *stage, int64_t vt, int64_t lo,
                                                    int64_t hi, uint32_t t_off)
{
    const uint8_t *sp = stage + kHalo + 32 * threadIdx.x;
    uint32_t w[10];
    for (int j = 0; j < 10; j++)
        w[j] = mask_word_bytes(*reinterpret_cast<const uint32_t *>(sp - 4 + 4 * j), vt - 4 + 4 * j,
                               lo, hi);
    uint32_t units = 0;
    for (int i = 0; i < 32; i++) {
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

struct St8 {
    uint32_t w[10];    // w[0]: bytes -4..-1, w[1..8]: own bytes 0..31, w[9]: 32..35
    uint32_t end[8];   // end-position indicators (bit 7 of each byte)
    uint32_t vmask;    // owned positions inside the input
    uint32_t bad;      // the fast check fired
    bool skip;         // the whole warp lies outside the input (warp-uniform)
    bool warp3, warp4;
};

// Structure check (expected continuations = continuations), C0/C1 check
// and end positions of one thread (Sec. 6.1, 6.4); returns its unit count.
// k3: the warp holds >= E0 leads (else every >= E0 / >= F0 term is zero and
// dropped). ORs its >= F0 leads into any4.
template <bool k3>
__device__ __forceinline__ uint32_t structure8(St8 &st, const uint32_t *w, bool wmasked,
                                               uint32_t &bad, uint32_t &any4)
{
    Cls cl[10];
#pragma unroll
    for (int j = 0; j < 10; j++) {
        cl[j] = classify(w[j]);
        if (!k3) cl[j].c3 = cl[j].c4 = 0;
    }
    // leads in the look-behind word shape the units at the first positions
    any4 = cl[0].c4;
    uint32_t ec[9], cnt = 0;
#pragma unroll
    for (int j = 1; j <= 8; j++) {
        const uint32_t exp = back(cl[j - 1].c2, cl[j].c2, 8) | back(cl[j - 1].c3, cl[j].c3, 16) |
                             back(cl[j - 1].c4, cl[j].c4, 24);
        bad |= exp ^ cl[j].ct;
        ec[j - 1] = exp & cl[j].ct;
        // C0 / C1: 2-byte leads whose bits 4..1 are zero
        bad |= cl[j].c2 & ~cl[j].c3 & zero_bytes(w[j] & 0x1E1E1E1Eu);
        any4 |= cl[j].c4;
    }
    // continuations the last leads expect at positions 32..34
    const uint32_t exp9 = (cl[8].c2 >> 24) | (cl[8].c3 >> 16) | (cl[8].c4 >> 8);
    bad |= exp9 & ~cl[9].ct;
    ec[8] = exp9 & cl[9].ct;
    if (!wmasked) {
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t e = (~ahead(ec[j - 1], ec[j], 8) | back(cl[j - 1].c4, cl[j].c4, 16)) & kB7;
            st.end[j - 1] = e;
            cnt += __popc(e);
        }
    } else {
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            uint32_t e = (~ahead(ec[j - 1], ec[j], 8) | back(cl[j - 1].c4, cl[j].c4, 16)) & kB7;
            e &= spread4((st.vmask >> (4 * (j - 1))) & 0xFu);
            st.end[j - 1] = e;
            cnt += __popc(e);
        }
    }
    return cnt;
}

// Load, classify, check structure, count units. Returns the thread's count.
__device__ __forceinline__ uint32_t chunk8_phase1(St8 &st, const uint8_t *stage, int64_t vt,
                                                  int64_t lo, int64_t hi)
{
    const uint8_t *sp = stage + kHalo + 32 * threadIdx.x;
    const uint4 a = *reinterpret_cast<const uint4 *>(sp);
    const uint4 b = *reinterpret_cast<const uint4 *>(sp + 16);
    uint32_t *w = st.w;
    w[1] = a.x; w[2] = a.y; w[3] = a.z; w[4] = a.w;
    w[5] = b.x; w[6] = b.y; w[7] = b.z; w[8] = b.w;
    w[0] = *reinterpret_cast<const uint32_t *>(sp - 4);
    w[9] = *reinterpret_cast<const uint32_t *>(sp + 32);
    st.bad = 0;
    st.vmask = 0xFFFFFFFFu;
    bool masked = false;
    // A chunk whose bytes and context all lie inside the input (the common
    // case; the test is the same for every thread) needs none of the edge
    // handling below.
    const int64_t v0 = vt - 32 * (int64_t)threadIdx.x;
    const bool interior = v0 - 4 >= lo && v0 + (int64_t)kChunk8 + 4 <= hi;
    if (!interior) {
        // threads wholly outside the input (the tail of an item's last chunk)
        // count nothing; a warp wholly outside skips the chunk body
        const bool outside = vt + 32 <= lo || vt >= hi;
        st.skip = __all_sync(kFull, outside);
        if (st.skip) {
            st.vmask = 0;
            st.warp3 = st.warp4 = false;
            return 0;
        }
        if (outside) {
#pragma unroll
            for (int j = 0; j < 10; j++) w[j] = 0;
            st.vmask = 0;
            masked = true;
        } else if (vt < lo || vt + 32 > hi) {   // straddles an end of the input
            masked = true;
            st.vmask = 0;
#pragma unroll
            for (int i = 0; i < 32; i++)
                if (vt + i >= lo && vt + i < hi) st.vmask |= 1u << i;
#pragma unroll
            for (int j = 0; j < 8; j++) w[1 + j] = mask_word_bytes(w[1 + j], vt + 4 * j, lo, hi);
        }
        if (!outside && (vt - 4 < lo || vt + 36 > hi)) {
            w[0] = mask_word_bytes(w[0], vt - 4, lo, hi);
            w[9] = mask_word_bytes(w[9], vt + 32, lo, hi);
        }
    } else {
        st.skip = false;
    }
    // some thread of the warp masks its end positions (warp-uniform, so the
    // unmasked warps branch around that work instead of predicating it)
    const bool wmasked = !interior && __any_sync(kFull, masked);

    // leads >= E0 (3/4-byte) anywhere in the warp, the look-behind word
    // included: without them the phase below drops their terms
    uint32_t any3 = 0;
#pragma unroll
    for (int j = 0; j < 9; j++) any3 |= w[j] & (w[j] << 1) & (w[j] << 2);
    st.warp3 = __any_sync(kFull, (any3 & kB7) != 0);
    uint32_t bad = 0, any4 = 0, cnt;
    if (st.warp3) {
        cnt = structure8<true>(st, w, wmasked, bad, any4);
        st.warp4 = __any_sync(kFull, any4 != 0);
    } else {
        cnt = structure8<false>(st, w, wmasked, bad, any4);
        st.warp4 = false;
    }
    if (st.warp3) {
        // E0 + 80..9F (overlong), ED + A0..BF (surrogate): a byte that is E0
        // when bit 5 of the next byte is clear, or ED when it is set
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t y5 = ahead(w[j], w[j + 1], 8) << 2;   // bit 5 of the next byte, at bit 7
            const uint32_t m = ((y5 >> 7) & 0x01010101u) * 0x0Du;  // 0x0D where it is set
            bad |= zero_bytes(w[j] ^ 0xE0E0E0E0u ^ m);
        }
    }
    if (st.warp4) {
        // F0 + 80..8F (overlong), F4 + 90..BF (too large): a byte that is F0
        // when bits 5 and 4 of the next byte are clear, or F4 when one is
        // set; and F5..FF (the low 7 bits reach 0x80 when 0x0B is added)
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t y = ahead(w[j], w[j + 1], 8);
            const uint32_t y54 = (y << 2) | (y << 3);              // bit 7: bit 5 or 4 of the next byte
            const uint32_t m = (y54 >> 5) & 0x04040404u;           // 0x04 where set
            bad |= zero_bytes(w[j] ^ 0xF0F0F0F0u ^ m);
            bad |= ((w[j] & 0x7F7F7F7Fu) + 0x0B0B0B0Bu) & w[j] & 0x80808080u;
        }
    }
    st.bad = bad;
    return cnt;
}

// Exact first error (flagged threads) and staging of the units.
// Units at the end positions (Eq. W_sum, W_out), four positions at a time
// on two registers of 16-bit lanes, stored at p in order. k3 / k4: the warp
// holds 3- or 4-byte leads (4-byte leads are also >= E0, so k4 implies k3).
template <bool k3, bool k4, bool kBE>
__device__ __forceinline__ void assemble8(const St8 &st, uint16_t *p)
{
    const uint32_t *w = st.w;
    uint32_t s[9], c3[9], c4[9];
#pragma unroll
    for (int j = 0; j < 9; j++) {
        // >= E0 / >= F0 at bit 7 of each byte (the other bits are not
        // used: the masks below replicate bit 7)
        if (k3) c3[j] = w[j] & (w[j] << 1) & (w[j] << 2);
        if (k4) c4[j] = c3[j] & (w[j] << 3);
        const uint32_t na = prmt(w[j], 0, 0xBA98);        // 0xFF where byte >= 0x80
        s[j] = w[j] & ~(na & 0xC0C0C0C0u);                // tag bits stripped
    }
#pragma unroll
    for (int j = 1; j <= 8; j++) {
        const uint32_t na = prmt(w[j], 0, 0xBA98);
        const uint32_t s1 = back(s[j - 1], s[j], 8) & na;          // W_-1 where end byte is not ASCII
        uint32_t wa = prmt(s[j], 0, 0x4140) + (prmt(s1, 0, 0x4140) << 6);
        uint32_t wb = prmt(s[j], 0, 0x4342) + (prmt(s1, 0, 0x4342) << 6);
        if (k3) {
            // W_-2 (low 4 bits) where the byte two back is a 3/4-byte lead
            const uint32_t m3 = prmt(c3[j - 1], c3[j], 0xDCBA);
            const uint32_t s2 = back(s[j - 1], s[j], 16) & m3 & 0x0F0F0F0Fu;
            wa += prmt(s2, 0, 0x4140) << 12;
            wb += prmt(s2, 0, 0x4342) << 12;
        }
        if (k4) {
            // surrogates: high at the third byte of a 4-byte sequence,
            // low at its fourth byte (Eq. W_out)
            const uint32_t hma = prmt(c4[j - 1], c4[j], 0xBBAA);
            const uint32_t hmb = prmt(c4[j - 1], c4[j], 0xDDCC);
            const uint32_t lma = prmt(c4[j - 1], c4[j], 0xAA99);
            const uint32_t lmb = prmt(c4[j - 1], c4[j], 0xCCBB);
            const uint32_t ha = ((wa >> 4) & 0x0FFF0FFFu) + 0xD7C0D7C0u;
            const uint32_t hb = ((wb >> 4) & 0x0FFF0FFFu) + 0xD7C0D7C0u;
            wa = ((ha & hma) | (wa & ~hma)) | (lma & 0xDC00DC00u);
            wb = ((hb & hmb) | (wb & ~hmb)) | (lmb & 0xDC00DC00u);
        }
        if (kBE) {   // UTF-16BE output
            wa = prmt(wa, 0, 0x2301);
            wb = prmt(wb, 0, 0x2301);
        }
        const uint32_t e = st.end[j - 1];
        if (e & 0x00000080u) *p++ = (uint16_t)wa;
        if (e & 0x00008000u) *p++ = (uint16_t)(wa >> 16);
        if (e & 0x00800000u) *p++ = (uint16_t)wb;
        if (e & 0x80000000u) *p++ = (uint16_t)(wb >> 16);
    }
}

template <bool kWrite, bool kBE>
__device__ __forceinline__ void chunk8_phase2(St8 &st, const uint8_t *stage, uint8_t *obuf,
                                              uint32_t t_off, int64_t vt, int64_t lo, int64_t hi,
                                              unsigned long long *s_err)
{
    if (st.skip) return;
    // Threads straddling an end of the input see the bytes outside it as
    // zeros (ASCII), which neither create nor hide an error inside it, so
    // the fast check covers them as well.
    if (st.bad) {
        const uint64_t key = first_error_exact8(stage, vt, lo, hi, t_off);
        if (key != ~0ull) atomicMin(s_err, key);
    }
    if (!kWrite) return;
    // the 3/4-byte parts only in warps that hold such leads (warp-uniform)
    uint16_t *p = reinterpret_cast<uint16_t *>(obuf) + t_off;
    if (st.warp4)
        assemble8<true, true, kBE>(st, p);
    else if (st.warp3)
        assemble8<true, false, kBE>(st, p);
    else
        assemble8<false, false, kBE>(st, p);
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

__device__ __forceinline__ uint32_t lane16(const uint32_t *w, int i)   // word i, i in [-2, 18)
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
    uint32_t w[10];    // w[0]: words -2,-1; w[1..8]: own words 0..15; w[9]: words 16,17
    uint32_t vmask;
    bool slow;         // the thread straddles an end of the input
    bool skip;         // the whole warp lies outside the input (warp-uniform)
    bool sur, only12;  // the warp holds surrogates / only words below U+0800 (warp-uniform)
};

__device__ __forceinline__ uint32_t unit_keep(int64_t u, int64_t lo, int64_t hi)
{
    return (u >= lo && u < hi) ? 0xFFFFu : 0u;
}

template <bool kBE>
__device__ __forceinline__ uint32_t chunk16_phase1(St16 &st, const uint8_t *stage, int64_t vt,
                                                   int64_t lo, int64_t hi)
{
    const uint8_t *sp = stage + kHalo + 32 * threadIdx.x;
    const uint4 a = *reinterpret_cast<const uint4 *>(sp);
    const uint4 b = *reinterpret_cast<const uint4 *>(sp + 16);
    uint32_t *w = st.w;
    w[1] = a.x; w[2] = a.y; w[3] = a.z; w[4] = a.w;
    w[5] = b.x; w[6] = b.y; w[7] = b.z; w[8] = b.w;
    w[0] = *reinterpret_cast<const uint32_t *>(sp - 4);
    w[9] = *reinterpret_cast<const uint32_t *>(sp + 32);
    st.vmask = 0xFFFFu;
    bool edge = false, masked = false;
    // A chunk whose words and context all lie inside the input (the common
    // case; the same test for every thread) needs none of the edge handling.
    const int64_t v0 = vt - 16 * (int64_t)threadIdx.x;
    const bool interior = v0 - 2 >= lo && v0 + (int64_t)kChunk16 + 2 <= hi;
    if (!interior) {
        // threads wholly outside the input count nothing; a warp wholly
        // outside skips the chunk body
        const bool outside = vt + 16 <= lo || vt >= hi;
        st.skip = __all_sync(kFull, outside);
        if (st.skip) {
            st.vmask = 0;
            st.slow = st.sur = st.only12 = false;
            return 0;
        }
        if (outside) {
#pragma unroll
            for (int j = 0; j < 10; j++) w[j] = 0;
            st.vmask = 0;
            masked = true;
        } else if (vt < lo || vt + 16 > hi) {   // straddles an end of the input
            edge = masked = true;
            st.vmask = 0;
#pragma unroll
            for (int i = 0; i < 16; i++)
                if (vt + i >= lo && vt + i < hi) st.vmask |= 1u << i;
#pragma unroll
            for (int j = 0; j < 8; j++)
                w[1 + j] &= unit_keep(vt + 2 * j, lo, hi) | (unit_keep(vt + 2 * j + 1, lo, hi) << 16);
        }
        if (!outside && (vt - 2 < lo || vt + 18 > hi)) {
            w[0] &= unit_keep(vt - 2, lo, hi) | (unit_keep(vt - 1, lo, hi) << 16);
            w[9] &= unit_keep(vt + 16, lo, hi) | (unit_keep(vt + 17, lo, hi) << 16);
        }
    } else {
        st.skip = false;
    }
    // some thread of the warp counts only part of its words (warp-uniform)
    const bool wmasked = !interior && __any_sync(kFull, masked);
    if (kBE) {   // UTF-16BE: swap the bytes of every word once, then as UTF-16LE
#pragma unroll
        for (int j = 0; j < 10; j++) w[j] = prmt(w[j], 0, 0x2301);
    }
    // does the warp hold words of U+0800 and above? (warp-uniform; words
    // outside the input are zero)
    uint32_t top5 = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) top5 |= w[1 + j] & 0xF800F800u;
    st.only12 = !__any_sync(kFull, top5 != 0);
    // per word: 1 + [>=80] + [>=800] - [surrogate]: 1-3 bytes, 2 for either
    // half of a pair
    uint32_t cnt = 0, anysur = 0;
    if (!wmasked && st.only12) {
        cnt = 16;
#pragma unroll
        for (int j = 0; j < 8; j++) cnt += __popc(ge80_lanes(w[1 + j]));
    } else if (!wmasked) {
        cnt = 16;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint32_t x = w[1 + j];
            const uint32_t ga = ge80_lanes(x), gb = ge800_lanes(x), s = surr_lanes(x);
            cnt += __popc(ga) + __popc(gb) - __popc(s);
            anysur |= s;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint32_t x = w[1 + j];
            const uint32_t ga = ge80_lanes(x), gb = ge800_lanes(x), s = surr_lanes(x);
            const uint32_t vm = (((st.vmask >> (2 * j)) & 1u) << 15) | (((st.vmask >> (2 * j + 1)) & 1u) << 31);
            cnt += __popc(vm) + __popc(ga & vm) + __popc(gb & vm) - __popc(s & vm);
            anysur |= s;
        }
    }
    st.sur = __any_sync(kFull, anysur != 0);
    st.slow = edge;
    return cnt;
}

// UTF-8 bytes of 16 units, two units at a time on 16-bit lanes
// (Fig. 1(a)): lead F (the unit itself, C0 | u >> 6, or E0 | u >> 12),
// second byte S (80 | u & 3F, or 80 | (u >> 6) & 3F in the 3-byte form) and
// third byte T (80 | u & 3F); each unit stores its 1-3 bytes at p.
// A surrogate pair's 4 bytes (Sec. 7.3) are split between its halves, 2
// each: with U = (high & 3FF) + 40 (the code point >> 10), the high
// surrogate stores F0 | U >> 8 and 80 | (U >> 2) & 3F, the low one
// 80 | (high & 3) << 4 | (low >> 6) & F and 80 | low & 3F.
// kSur: the units may hold surrogates (validly paired; the pair may cross
// into the next thread, the low half then stores its 2 bytes there).
template <bool kSur>
__device__ __forceinline__ void encode_bmp(const uint32_t *w, uint8_t *p)
{
#pragma unroll
    for (int j = 1; j <= 8; j++) {
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
            const uint32_t prev = __funnelshift_l(w[j - 1], x, 16);   // the unit before each lane
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

template <bool kWrite>
__device__ __forceinline__ void chunk16_phase2(const St16 &st, uint8_t *obuf, uint32_t t_off,
                                               int64_t vt, int64_t lo, unsigned long long *s_err)
{
    if (st.skip || st.vmask == 0) return;   // nothing of the input here
    const uint32_t *w = st.w;
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
        for (int j = 1; j <= 8; j++) {
            const uint32_t h = hi_lanes(w[j]);
            v |= __funnelshift_l(h_prev, h, 16) ^ lo_lanes(w[j]);
            h_prev = h;
        }
        v |= (h_prev ^ (lo_lanes(w[9]) << 16)) & 0x80000000u;
        slow = v != 0;
    }
    if (!slow) {
        // every word of this thread is valid
        if (!kWrite) return;
        uint8_t *p = obuf + t_off;
        if (st.sur) {
            encode_bmp<true>(w, p);
        } else if (st.only12) {
#pragma unroll
            for (int i = 0; i < 16; i++) {
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
    for (int i = 0; i < 16; i++) {
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
            if (kWrite && o + len <= kStage16Bytes) {
                uint8_t *q = obuf + o;
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
    uint64_t full[kStages];        // mbarrier per stage (TMA completion)
    Item item[kStages];
    uint32_t chunk[kStages], itidx[kStages], end[kStages];
};

// Thread 0: start the TMA load of chunk c (claimed earlier) into `slot`; `it`
// is its item index and, in a batch, *pre its descriptor, both fetched
// earlier (the descriptor by cp.async, waited for here).
// Returns false (and marks the slot as the end) when the job is exhausted.
__device__ __forceinline__ bool produce(const Job &J, uint32_t c, uint32_t it, const Item *pre,
                                        int slot, uint8_t *stages, Ring &R)
{
    if (c >= J.total_chunks) {
        R.end[slot] = 1;
        mbar_arrive(&R.full[slot]);
        return false;
    }
    if (J.items) {
        cp_async_wait_all();
        R.item[slot] = *pre;
    } else {
        R.item[slot] = J.item0;
    }
    const Item I = R.item[slot];
    R.chunk[slot] = c;
    R.itidx[slot] = it;
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

struct Pending {                 // a processed chunk waiting for its offset
    Item item;
    uint32_t chunk, itidx, agg, end;
};

struct Done {                    // what the look-back warp keeps of a chunk until it is written
    uint64_t excl;
    uint32_t chunk, itidx, nchunks, agg;
};

// The last CTA out checks that every chunk id was handed out exactly once,
// advances the epoch and resets the job's counters for the next launch.
__device__ __forceinline__ void exit_job(const Job &J, uint32_t epoch)
{
    __threadfence();
    if (atomicAdd(J.exit_count, 1u) != gridDim.x - 1) return;
    __threadfence();   // every other CTA's accounting is visible
    if (!J.items) finalize_item(J, 0, J.item0);
    const unsigned int claims = atomicExch(J.claim, 0u);
    const unsigned int flags = atomicAdd(J.flags, 0u);
    if (claims != J.total_chunks + gridDim.x || flags != 0) {
        // counters were left dirty by an aborted launch, or a wait gave up
        // (chunks may have been skipped, items left unfinished): no item was
        // finished reliably
        const int32_t st = claims != J.total_chunks + gridDim.x || (flags & 2u) ? kDeviceError
                                                                               : kDeviceTimeout;
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

// Warps 0-7 (compute): at iteration i, wait for chunk i's stage, classify and
// count it, scan, publish its aggregate and hand it to the look-back warp
// (pend_bar). Then write out chunk i-kDepth from staging buffer i % kDepth
// (its offset was computed meanwhile) and signal it (written_bar), and
// assemble chunk i's output into the same buffer. Thread 0 also feeds the TMA
// ring, claiming chunk ids one iteration ahead so that the claim's latency is
// hidden. Warp 8 (look-back): for every handed-over chunk, as soon as its
// aggregate is out, look back, publish the inclusive prefix and hand the
// offset back (excl_bar); once the chunk is written, record its first error
// and count it done, finishing its item's result when it is the item's last
// chunk (a one-item job is finished by its last CTA). None of the global
// atomics and fences of this bookkeeping sit on the compute path.
// Output staging depth: a chunk staged in iteration i is written out in
// iteration i + kDepth, so its offset has kDepth iterations to arrive.
#ifndef GBU_OUT_DEPTH
#define GBU_OUT_DEPTH 3
#endif
constexpr int kDepth = GBU_OUT_DEPTH;
// Hand-over slots (chunk j uses j % kSlots): more than the kDepth + 1
// chunks between a hand-over and the write-out that retires it.
constexpr int kSlots = 8;
static_assert(kSlots > kDepth + 1, "hand-over slots");

template <bool kWrite, int kLook, bool kAnyBE>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
transcode_kernel(const Job J)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    uint8_t *const stages = dyn_smem;
    uint8_t *const obufs = dyn_smem + kStages * kStageBytes;
    __shared__ __align__(16) Ring R;
    __shared__ __align__(16) Item s_next_item;
    __shared__ __align__(8) uint64_t pend_bar[kSlots], excl_bar[kSlots], written_bar[kSlots];
    __shared__ Pending s_pend[kSlots];
    __shared__ unsigned long long s_excl[kSlots], s_errsnap[kSlots], s_err[kDepth];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_epoch;

    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(&R.full[s], 1);
        for (int s = 0; s < kSlots; s++) {
            mbar_init(&pend_bar[s], 1);
            mbar_init(&excl_bar[s], 1);
            mbar_init(&written_bar[s], 1);
        }
        for (int s = 0; s < kDepth; s++) s_err[s] = ~0ull;
        fence_mbar_init();
        s_epoch = *reinterpret_cast<volatile unsigned int *>(J.epoch);
    }
    __syncthreads();
    const uint32_t epoch = s_epoch;

    if (tid >= kThreads) {
        // ---- look-back warp -------------------------------------------------
        const bool lead = tid == kThreads;
        bool failed = false;
        Done dq[kDepth] = {};   // dq[m]: chunk j-1-m
        // chunk j was written: merge its first error, count it done
        auto account = [&](const Done &d, uint32_t j) -> bool {
            if (!mbar_wait(&written_bar[j % kSlots], (j / kSlots) & 1u)) return false;
            if (lead) {
                const uint64_t key = s_errsnap[j % kSlots];
                if (!J.items) {
                    // one item: its result is finished by the last CTA out
                    if (key != ~0ull) {
                        J.err_prefix[d.chunk] = d.excl + (key & 0x7FFFu);
                        atomicMin(&J.item_err[0], ((key >> 23) << 8) | ((key >> 15) & 0xFFu));
                    }
                } else if (d.nchunks == 1) {
                    finalize_single(J, J.items ? J.items[d.itidx] : J.item0, d.agg, key);
                } else {
                    if (key != ~0ull) {
                        J.err_prefix[d.chunk] = d.excl + (key & 0x7FFFu);
                        atomicMin(&J.item_err[d.itidx], ((key >> 23) << 8) | ((key >> 15) & 0xFFu));
                    }
                    if (atomic_add_acq_rel(&J.item_done[d.itidx], 1u) == d.nchunks - 1)
                        finalize_item(J, d.itidx, J.items ? J.items[d.itidx] : J.item0);
                }
            }
            return true;
        };
        uint32_t j = 0;
        for (;; j++) {
            const int q = j % kSlots;
            if (!mbar_wait(&pend_bar[q], (j / kSlots) & 1u)) {
                failed = true;
                break;
            }
            const Pending &P = s_pend[q];
            if (P.end) break;
            const uint32_t k = P.chunk - P.item.chunk_base;
            uint64_t excl = 0;
            if (k > 0 && !J.validate) {   // validation needs no offsets
                excl = lookback<kLook>(J.status + P.item.chunk_base, k, epoch, J.flags);
                if (lead)
                    st_relaxed(&J.status[P.chunk], pack_status(kFlagInclusive, epoch, excl + P.agg));
            }
            Done d0;
            d0.excl = excl;
            d0.chunk = P.chunk;
            d0.itidx = P.itidx;
            d0.nchunks = P.item.nchunks;
            d0.agg = P.agg;
            __syncwarp();
            if (lead) {
                s_excl[q] = excl;
                mbar_arrive(&excl_bar[q]);
            }
            if (j >= kDepth && !account(dq[kDepth - 1], j - kDepth)) {
                failed = true;
                break;
            }
#pragma unroll
            for (int m = kDepth - 1; m > 0; m--) dq[m] = dq[m - 1];
            dq[0] = d0;
        }
        // the compute warps stop after writing out their last kDepth chunks
#pragma unroll
        for (int m = kDepth; m > 0; m--)
            if (!failed && j >= (uint32_t)m && !account(dq[m - 1], j - m)) failed = true;
        if (lead) {
            if (failed) atomicOr(J.flags, 1u);
            exit_job(J, epoch);
        }
        return;
    }

    // ---- compute warps ------------------------------------------------------
    // write out chunk j (staging buffer j&1) once its offset is known; false
    // if the wait for the offset gave up
    auto write_out = [&](uint32_t j) -> bool {
        const int q = j % kSlots;
        if (!mbar_wait(&excl_bar[q], (j / kSlots) & 1u)) return false;
        if (kWrite) {
            const Pending &P = s_pend[q];
            const uint64_t excl = s_excl[q];
            const bool u16 = (P.item.op & kOpUtf16) != 0;
            const uint32_t ub = u16 ? 1u : 2u;                       // output unit bytes
            const uint32_t stage_units = u16 ? kStage16Bytes : kStage8Units;
            if (excl < P.item.cap) {
                const uint64_t room = P.item.cap - excl;
                uint32_t nw = P.agg < stage_units ? P.agg : stage_units;
                if (nw > room) nw = (uint32_t)room;
                block_store_bytes(obufs + (size_t)(j % kDepth) * kOutBufBytes, P.item.out + excl * ub,
                                  nw * ub);
            }
        }
        if (tid == 0) {
            s_errsnap[q] = s_err[j % kDepth];
            s_err[j % kDepth] = ~0ull;
            mbar_arrive(&written_bar[q]);
        }
        return true;
    };

    // Thread 0 feeds the ring. The chunk it loads at the top of iteration i
    // was claimed at the top of iteration i-1, its item index fetched in the
    // middle and its item descriptor at the end of iteration i-1, so none of
    // these global round trips stalls the CTA.
    bool producing = true;   // meaningful in thread 0 only
    uint32_t next_claim = 0, next_it = 0;
    auto fetch_it = [&]() {
        if (J.chunk_item && next_claim < J.total_chunks) next_it = J.chunk_item[next_claim];
    };
    // the descriptor of the next load, fetched asynchronously
    auto fetch_item = [&]() {
        if (J.items && next_claim < J.total_chunks) {
            const uint8_t *src = reinterpret_cast<const uint8_t *>(J.items + next_it);
            uint8_t *dst = reinterpret_cast<uint8_t *>(&s_next_item);
#pragma unroll
            for (int q = 0; q < (int)sizeof(Item); q += 16) cp_async16(dst + q, src + q);
        }
    };
    if (tid == 0) {
        for (int s = 0; s < kStages - 1 && producing; s++) {
            next_claim = atomicAdd(J.claim, 1u);
            fetch_it();
            fetch_item();
            producing = produce(J, next_claim, next_it, &s_next_item, s, stages, R);
        }
        if (producing) {   // the chunk loaded in iteration 0
            next_claim = atomicAdd(J.claim, 1u);
            fetch_it();
            fetch_item();
        }
    }

    uint32_t iter = 0, handed = 0;
    bool failed = false;
    while (true) {
        const int slot = iter % kStages;
        const int p = iter % kDepth;
        const bool ok = mbar_wait(&R.full[slot], (iter / kStages) & 1u);
        if (cw_sync_or(!ok)) {
            failed = true;
            break;
        }
        // every compute thread is done with iteration iter-1: its stage can
        // be refilled
        if (tid == 0 && producing) {
            producing = produce(J, next_claim, next_it, &s_next_item, (iter + kStages - 1) % kStages,
                                stages, R);
            if (producing) next_claim = atomicAdd(J.claim, 1u);   // used next iteration
        }
        if (R.end[slot]) break;
        const Item I = R.item[slot];
        const uint32_t c = R.chunk[slot];
        const uint32_t it = R.itidx[slot];
        const uint8_t *stage = stages + (size_t)slot * kStageBytes;
        uint8_t *obuf = obufs + (size_t)p * kOutBufBytes;
        const int64_t lo = I.head, hi = (int64_t)I.head + (int64_t)I.n;
        const uint32_t k = c - I.chunk_base;
        uint32_t agg, t_off;
        auto hand_over = [&]() {
            if (tid == 0) {
                st_relaxed(&J.status[c], pack_status(k == 0 ? kFlagInclusive : kFlagAggregate, epoch, agg));
                Pending &P = s_pend[iter % kSlots];
                P.item = I;
                P.chunk = c;
                P.itidx = it;
                P.agg = agg;
                P.end = 0;
                mbar_arrive(&pend_bar[iter % kSlots]);
                if (producing) fetch_it();
            }
            handed++;
        };
        if (I.op & kOpUtf16) {
            const int64_t vt = (int64_t)k * kChunk16 + 16 * tid;
            St16 st;
            const uint32_t cnt = (kAnyBE && (I.op & kOpBE))
                                     ? chunk16_phase1<true>(st, stage, vt, lo, hi)
                                     : chunk16_phase1<false>(st, stage, vt, lo, hi);
            t_off = block_exclusive_scan(cnt, s_warp, &agg);
            hand_over();
            if (iter >= kDepth && cw_sync_or(!write_out(iter - kDepth))) {
                failed = true;
                break;
            }
            chunk16_phase2<kWrite>(st, obuf, t_off, vt, lo, &s_err[p]);
        } else {
            const int64_t vt = (int64_t)k * kChunk8 + 32 * tid;
            St8 st;
            const uint32_t cnt = chunk8_phase1(st, stage, vt, lo, hi);
            t_off = block_exclusive_scan(cnt, s_warp, &agg);
            hand_over();
            if (iter >= kDepth && cw_sync_or(!write_out(iter - kDepth))) {
                failed = true;
                break;
            }
            if (kAnyBE && (I.op & kOpBE))
                chunk8_phase2<kWrite, true>(st, stage, obuf, t_off, vt, lo, hi, &s_err[p]);
            else
                chunk8_phase2<kWrite, false>(st, stage, obuf, t_off, vt, lo, hi, &s_err[p]);
        }
        // every thread read this iteration's R.item[slot] at its start: the
        // slot's descriptor can be replaced by the one the next load needs
        if (tid == 0 && producing) fetch_item();
        iter++;
    }
    // drain: write out the last kDepth chunks, then stop the look-back warp
    for (int m = kDepth; m > 0 && !failed; m--)
        if (iter >= (uint32_t)m && cw_sync_or(!write_out(iter - m))) failed = true;
    if (tid == 0) {
        if (failed) atomicOr(J.flags, 1u);
        Pending &P = s_pend[handed % kSlots];
        P.end = 1;
        mbar_arrive(&pend_bar[handed % kSlots]);
    }
}

int g_max_per_sm[64] = {0};
int g_sms[64] = {0};

}  // namespace

size_t job_smem_bytes(bool write)
{
    return (size_t)kStages * kStageBytes + (write ? (size_t)kDepth * kOutBufBytes : 0);
}

// Every instantiation of the kernel: (write, look-back width, whether any
// item is UTF-16BE; the UTF-16LE-only kernels carry no byte-order code).
template <bool W, int L>
const void *kernel_fn(bool be)
{
    return be ? reinterpret_cast<const void *>(&transcode_kernel<W, L, true>)
              : reinterpret_cast<const void *>(&transcode_kernel<W, L, false>);
}

const void *kernel_for(bool write, int look, bool be)
{
    switch (look) {
    case 1: return write ? kernel_fn<true, 1>(be) : kernel_fn<false, 1>(be);
    case 2: return write ? kernel_fn<true, 2>(be) : kernel_fn<false, 2>(be);
    case 8: return write ? kernel_fn<true, 8>(be) : kernel_fn<false, 8>(be);
    case 16: return write ? kernel_fn<true, 16>(be) : kernel_fn<false, 16>(be);
    default: return write ? kernel_fn<true, 4>(be) : kernel_fn<false, 4>(be);
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
                if (cudaFuncSetAttribute(kernel_for(w != 0, look, be != 0),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)job_smem_bytes(w != 0)) != cudaSuccess)
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

int job_max_grid(int device)
{
    return job_grid(device, Tune{});
}

cudaError_t launch_job(const Job &J, bool write, int grid, cudaStream_t stream, int look, bool be)
{
    void *args[] = {const_cast<Job *>(&J)};
    return cudaLaunchKernel(kernel_for(write, look, be), dim3(grid), dim3(kBlock), args,
                            job_smem_bytes(write), stream);
}

__global__ void write_result_kernel(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                    uint64_t out_len)
{
    volatile ResultSlot *r = dst;
    r->status = status;
    r->reserved = 0;
    r->in_offset = in_offset;
    r->out_len = out_len;
    __threadfence_system();
}

cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream)
{
    write_result_kernel<<<1, 1, 0, stream>>>(dst, status, in_offset, out_len);
    return cudaGetLastError();
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

}  // namespace gbu
