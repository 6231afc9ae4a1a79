// UTF-8 -> UTF-16LE, validating, single pass (paper Sec. 6).
//
// Work decomposition: the input is cut into chunks of kChunk8 bytes, one CTA
// per chunk (claimed in order from an atomic counter so that the look-back
// always waits on CTAs that are already running). Each of the 256 threads owns
// 32 consecutive byte positions and sees 4 bytes on each side.
//
// Classification (Sec. 6.1) is done four bytes at a time on 32-bit words:
// indicator bit 7 of each byte for "continuation" (80-BF), ">= C0", ">= E0"
// and ">= F0" (the paper's complement of m_1234, m_234, m_34, m_4).
//
// Units are produced at the *end* positions of the sequences, as in the
// paper (Sec. 6.1-6.2): every last byte of a character, and the third byte of
// a 4-byte character, ends one UTF-16 unit, assembled from the last, second
// last and third last bytes with their tag bits stripped:
//   W = W_-2 << 12 | W_-1 << 6 | W_end   (Eq. W_sum, 16-bit),
// where W_-1 is used when the end byte is not ASCII and W_-2 when the byte two
// back is a 3/4-byte lead; high surrogates become (W >> 4) + 0xD7C0 and low
// surrogates W | 0xDC00 (Eq. W_out). Here four end positions are assembled at
// once on two registers of 16-bit lanes. A position p is an end when the byte
// after it does not continue a sequence, or when it is the third byte of a
// 4-byte sequence. "Continues" means a continuation byte that a lead at p-1,
// p-2 or p-3 expects (the paper's m_c); with that definition a stray
// continuation byte also ends the valid prefix before it, so the units of the
// valid prefix are exact even in a chunk that holds an error. Each position
// ends at most one unit, so a thread's count is the population count of its
// end mask and a chunk never produces more units than bytes.
//
// Validation (Sec. 6.4), two levels:
//  * fast, for every thread: the structure check is exact (expected
//    continuation positions, from the leads at p-1/p-2/p-3, must equal the
//    continuation positions: rules 2-3); bad bytes and out-of-range values
//    (rules 1, 4-6: C0/C1, F5-FF, E0+80..9F, ED+A0..BF, F0+80..8F, F4+90..BF)
//    are caught by a check that never misses an error but may flag a valid
//    word (the E0/ED and F0/F4/F5+ parts run only in warps holding such
//    bytes);
//  * exact, only in threads that were flagged: for every position p the rule
//    the sequential decoder applies if a character starts at p (stray
//    continuation -> TOO_LONG; C0/C1 -> OVERLONG; F5-FF -> HEADER_BITS; lead
//    without its continuations -> TOO_SHORT; then OVERLONG / SURROGATE /
//    TOO_LARGE from the value). The smallest such p is exactly where the
//    sequential decoder stops (every earlier position is a validated
//    character start or a continuation inside one), so the block-wide and
//    grid-wide minimum of (p, kind) is the paper's error position ell.
#include "kernels.h"

namespace gbu {

namespace {

constexpr int kPer8 = kChunk8 / kThreads;   // 32 bytes per thread
static_assert(kPer8 == 32, "one 32-bit position mask per thread");
// Staging capacity in units: at most one unit per input byte (see above).
constexpr uint32_t kStage8 = kChunk8 + 8;

constexpr uint32_t kB7 = 0x80808080u;

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
// w: 10 words (positions -4 .. 35); end: the 8 end-indicator words. Returns
// the key of the first error, or ~0.
__device__ __noinline__ uint64_t first_error_exact(const uint32_t *w, const uint32_t *end,
                                                   uint32_t vmask, int64_t pos0, uint32_t t_off)
{
    uint32_t units = 0;
    for (int i = 0; i < kPer8; i++) {
        const int j = (i >> 2) + 1;
        const int sh = (i & 3) * 8;
        const uint32_t xf = __funnelshift_r(w[j], w[j + 1], sh);   // bytes i .. i+3
        const uint32_t xb = __funnelshift_r(w[j - 1], w[j], sh);   // bytes i-4 .. i-1
        const uint32_t b0 = xf & 0xFFu;
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
        if (kind != 0 && ((vmask >> i) & 1u)) return err_key((uint64_t)(pos0 + i), kind, t_off + units);
        units += (end[i >> 2] >> (8 * (i & 3) + 7)) & 1u;
    }
    return ~0ull;
}

template <bool kWrite>
__global__ void __launch_bounds__(kThreads)
utf8_to_utf16_kernel(const uint8_t *__restrict__ in_al, uint16_t *__restrict__ out, Launch L)
{
    __shared__ __align__(16) uint8_t s_out[kWrite ? 2 * kStage8 + 16 : 16];
    __shared__ uint32_t s_first[kThreads], s_last[kThreads];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_chunk, s_halo_prev, s_halo_next;
    __shared__ unsigned long long s_err, s_excl;

    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        s_chunk = atomicAdd(L.s.claim, 1u);
        s_err = ~0ull;
    }
    __syncthreads();
    const uint32_t chunk = s_chunk;
    if (chunk >= L.num_chunks) {   // counter left dirty by an aborted launch
        if (tid == 0) {
            atomicOr(L.s.flags, 2u);
            finish_launch<kWrite>(L, kChunk8);
        }
        return;
    }
    const int64_t lo = L.head, hi = (int64_t)L.head + (int64_t)L.n;
    const int64_t v0 = (int64_t)chunk * kChunk8;
    const int64_t vt = v0 + (int64_t)tid * kPer8;

    // ---- load 32 bytes (two aligned 16-byte blocks) ------------------------
    uint32_t w[10];   // w[0]: bytes -4..-1, w[1..8]: own bytes 0..31, w[9]: 32..35
    {
        uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
        if (vt < hi) a = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt));
        if (vt + 16 < hi) b = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt + 16));
        w[1] = a.x; w[2] = a.y; w[3] = a.z; w[4] = a.w;
        w[5] = b.x; w[6] = b.y; w[7] = b.z; w[8] = b.w;
    }
    uint32_t vmask = 0xFFFFFFFFu;
    const bool edge = vt < lo || vt + kPer8 > hi;
    if (edge) {   // buffer edges only
        vmask = 0;
#pragma unroll
        for (int i = 0; i < kPer8; i++)
            if (vt + i >= lo && vt + i < hi) vmask |= 1u << i;
#pragma unroll
        for (int j = 0; j < 8; j++) w[1 + j] = mask_word_bytes(w[1 + j], vt + 4 * j, lo, hi);
    }
    s_first[tid] = w[1];
    s_last[tid] = w[8];
    if (tid == 0) {
        uint32_t h = 0;
        if (v0 >= 4 && v0 - 4 < hi) h = *reinterpret_cast<const uint32_t *>(in_al + v0 - 4);
        s_halo_prev = mask_word_bytes(h, v0 - 4, lo, hi);
    }
    if (tid == kThreads - 1) {
        uint32_t h = 0;
        const int64_t vn = v0 + kChunk8;
        if (vn < hi) h = *reinterpret_cast<const uint32_t *>(in_al + vn);
        s_halo_next = mask_word_bytes(h, vn, lo, hi);
    }
    __syncthreads();
    w[0] = tid ? s_last[tid - 1] : s_halo_prev;
    w[9] = tid + 1 < kThreads ? s_first[tid + 1] : s_halo_next;

    // ---- pass 1: classes, structure check, end mask, unit count ------------
    uint32_t c3[9], c4[9], end[8];
    uint32_t bad = 0, any3 = 0, any4 = 0, cnt = 0;
    {
        Cls cl[10];
#pragma unroll
        for (int j = 0; j < 10; j++) cl[j] = classify(w[j]);
        // leads in the look-behind word shape the units at my first positions
        any3 = cl[0].c3;
        any4 = cl[0].c4;
        uint32_t ec[9];
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t exp = back(cl[j - 1].c2, cl[j].c2, 8) | back(cl[j - 1].c3, cl[j].c3, 16) |
                                 back(cl[j - 1].c4, cl[j].c4, 24);
            bad |= exp ^ cl[j].ct;
            ec[j - 1] = exp & cl[j].ct;
            // C0 / C1: 2-byte leads whose bits 4..1 are zero
            bad |= cl[j].c2 & ~cl[j].c3 & zero_bytes(w[j] & 0x1E1E1E1Eu);
            any3 |= cl[j].c3;
            any4 |= cl[j].c4;
        }
        // continuations my last leads expect at positions 32..34
        const uint32_t exp9 = (cl[8].c2 >> 24) | (cl[8].c3 >> 16) | (cl[8].c4 >> 8);
        bad |= exp9 & ~cl[9].ct;
        ec[8] = exp9 & cl[9].ct;
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            uint32_t e = (~ahead(ec[j - 1], ec[j], 8) | back(cl[j - 1].c4, cl[j].c4, 16)) & kB7;
            if (edge) e &= spread4((vmask >> (4 * (j - 1))) & 0xFu);
            end[j - 1] = e;
            cnt += __popc(e);
        }
#pragma unroll
        for (int j = 0; j < 9; j++) {
            c3[j] = cl[j].c3;
            c4[j] = cl[j].c4;
        }
    }
    const bool warp3 = __any_sync(kFull, any3 != 0);
    const bool warp4 = __any_sync(kFull, any4 != 0);
    if (warp3) {
        // E0 + 80..9F (overlong), ED + A0..BF (surrogate); may over-flag
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t y5 = ahead(w[j], w[j + 1], 8) << 2;   // bit 5 of the next byte
            bad |= zero_bytes(w[j] ^ 0xE0E0E0E0u) & ~y5;
            bad |= zero_bytes(w[j] ^ 0xEDEDEDEDu) & y5;
        }
    }
    if (warp4) {
        // F0 + 80..8F (overlong), F4 + 90..BF (too large), F5..FF; may over-flag
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t y = ahead(w[j], w[j + 1], 8);
            const uint32_t y54 = (y << 2) | (y << 3);              // bits 5 or 4 of the next byte
            bad |= zero_bytes(w[j] ^ 0xF0F0F0F0u) & ~y54;
            bad |= zero_bytes(w[j] ^ 0xF4F4F4F4u) & y54;
            bad |= c4[j] & (((w[j] & 0x0F0F0F0Fu) + 0x0B0B0B0Bu) << 3);
        }
    }

    uint32_t agg;
    const uint32_t t_off = block_exclusive_scan(cnt, s_warp, &agg);
    if (tid == 0)
        st_relaxed(&L.s.status[chunk],
                   pack_status(chunk == 0 ? kFlagInclusive : kFlagAggregate, L.epoch, agg));

    // ---- chunk offset: warp 0 looks back first, the others start staging --
    if (tid < 32) {
        uint64_t excl = 0;
        if (chunk > 0) {
            excl = lookback(L, chunk);
            if (tid == 0)
                st_relaxed(&L.s.status[chunk], pack_status(kFlagInclusive, L.epoch, excl + agg));
        }
        if (tid == 0) s_excl = excl;
    }

    // ---- exact first error, only where the fast check fired ----------------
    if (bad || edge) {
        const uint64_t key = first_error_exact(w, end, vmask, vt - lo, t_off);
        if (key != ~0ull) atomicMin(&s_err, key);
    }

    // ---- pass 2: assemble units at end positions and stage them ------------
    if (kWrite) {
        uint32_t s[9];
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const uint32_t na = prmt(w[j], 0, 0xBA98);        // 0xFF where byte >= 0x80
            s[j] = w[j] & ~(na & 0xC0C0C0C0u);                       // tag bits stripped
        }
        uint16_t *p = reinterpret_cast<uint16_t *>(s_out) + t_off;
#pragma unroll
        for (int j = 1; j <= 8; j++) {
            const uint32_t na = prmt(w[j], 0, 0xBA98);
            const uint32_t s1 = back(s[j - 1], s[j], 8) & na;          // W_-1 where end byte is not ASCII
            uint32_t wa = prmt(s[j], 0, 0x4140) + (prmt(s1, 0, 0x4140) << 6);
            uint32_t wb = prmt(s[j], 0, 0x4342) + (prmt(s1, 0, 0x4342) << 6);
            if (warp3) {
                // W_-2 (low 4 bits) where the byte two back is a 3/4-byte lead
                const uint32_t m3 = prmt(c3[j - 1], c3[j], 0xDCBA);
                const uint32_t s2 = back(s[j - 1], s[j], 16) & m3 & 0x0F0F0F0Fu;
                wa += prmt(s2, 0, 0x4140) << 12;
                wb += prmt(s2, 0, 0x4342) << 12;
            }
            if (warp4) {
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
            const uint32_t e = end[j - 1];
            if (e & 0x00000080u) *p++ = (uint16_t)wa;
            if (e & 0x00008000u) *p++ = (uint16_t)(wa >> 16);
            if (e & 0x00800000u) *p++ = (uint16_t)wb;
            if (e & 0x80000000u) *p++ = (uint16_t)(wb >> 16);
        }
    }
    __syncthreads();
    const uint64_t excl = s_excl;

    if (kWrite && excl < L.cap) {
        const uint64_t room = L.cap - excl;
        uint32_t nw = agg < kStage8 ? agg : kStage8;
        if (nw > room) nw = (uint32_t)room;
        block_store_bytes(s_out, reinterpret_cast<uint8_t *>(out + excl), 2u * nw);
    }
    if (tid == 0) {
        publish_error(L, chunk, s_err, excl);
        finish_launch<kWrite>(L, kChunk8);
    }
}

}  // namespace

const uint8_t *plan_utf8(const uint8_t *in, uint64_t n, Launch &L)
{
    const uintptr_t p = reinterpret_cast<uintptr_t>(in);
    L.head = (uint32_t)(p & 15u);
    L.n = n;
    L.num_chunks = (uint32_t)((L.head + n + kChunk8 - 1) / kChunk8);
    return reinterpret_cast<const uint8_t *>(p - L.head);
}

cudaError_t launch_utf8_to_utf16(const uint8_t *in_aligned, uint16_t *out, bool write,
                                 const Launch &L, cudaStream_t stream)
{
    if (write)
        utf8_to_utf16_kernel<true><<<L.num_chunks, kThreads, 0, stream>>>(in_aligned, out, L);
    else
        utf8_to_utf16_kernel<false><<<L.num_chunks, kThreads, 0, stream>>>(in_aligned, out, L);
    return cudaGetLastError();
}

}  // namespace gbu
