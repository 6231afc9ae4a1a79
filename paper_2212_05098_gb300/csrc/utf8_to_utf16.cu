// UTF-8 -> UTF-16LE, validating, single pass (paper Sec. 6).
//
// Work decomposition: the input is cut into chunks of kChunk8 bytes, one CTA
// per chunk (claimed in order from an atomic counter so that the look-back
// always waits on CTAs that are already running). Each of the 256 threads owns
// 32 consecutive byte positions and sees 4 bytes on each side.
//
// Ownership: a character belongs to the thread (and chunk) that holds its
// first byte. This replaces the paper's "advance by complete sequences" rule
// (Sec. 6, plan of attack) and its output-straddle guard (Sec. 6.2, M_out):
// no character is ever split between two owners.
//
// Validation is local. For every position p the kernel evaluates the rule
// that the sequential decoder would apply if it started a character at p:
//   continuation byte 80-BF: TOO_LONG unless a lead at p-1 (>= C0), p-2
//     (>= E0) or p-3 (>= F0) expects it (Sec. 6.4, rules 2-3; the paper's m_c
//     mask of Eqs. m_+1, m_+2, m_c);
//   C0/C1: OVERLONG (Sec. 6.4, the overlong 2-byte check);
//   F5-FF: HEADER_BITS (rule 1);
//   lead C2-F4: TOO_SHORT unless the next len-1 bytes are continuations,
//     then OVERLONG / SURROGATE / TOO_LARGE from the assembled value
//     (rules 4-6; the M_<800, M_3s, M_4s checks of Sec. 6.4).
// The smallest p with a violation is exactly where the sequential decoder
// stops (every position before it is either a validated character start or a
// continuation inside a validated character), so the block-wide and then
// grid-wide minimum of (p, kind) is the first error, and the output offsets of
// all characters before it are exact.
//
// Output: characters are assembled from their bytes per Fig. 1(a); 4-byte
// characters become the surrogate pair (0xD7C0 + (cp >> 10), 0xDC00 | low 10
// bits), the constant of Sec. 6.2. Units are staged in shared memory at the
// thread's scanned offset and written with 16-byte stores.
#include "kernels.h"

namespace gbu {

namespace {

constexpr int kPer8 = kChunk8 / kThreads;   // 32 bytes per thread
static_assert(kPer8 == 32, "one 32-bit position mask per thread");
// Staging capacity in units. A chunk's valid characters need at most
// kChunk8 + 1 units (each valid character has no more units than bytes, and
// a 4-byte character whose lead is the chunk's last byte adds 2 units for 1
// byte). Offsets past an error can grow up to 2 units per byte, so stores and
// the write-out are bounded by this capacity; what lies past an error is
// unspecified output anyway.
constexpr uint32_t kStage8 = kChunk8 + 8;

// Continuation bytes (10xxxxxx), one indicator bit per byte at bit 7.
__device__ __forceinline__ uint32_t cont_bits(uint32_t x)
{
    return x & ~(x << 1) & 0x80808080u;
}

// Bytes >= F0, one indicator bit per byte at bit 7 (exact: the low nibble of
// every byte of t is zero, so no borrow crosses into a non-zero byte).
__device__ __forceinline__ uint32_t ge_f0_bits(uint32_t x)
{
    const uint32_t t = ~x & 0xF0F0F0F0u;
    return (t - 0x01010101u) & ~t & 0x80808080u;
}

// 4 bits of a position mask -> bit 7 of the 4 bytes of a word.
__device__ __forceinline__ uint32_t spread4(uint32_t m4)
{
    return ((m4 * 0x00204081u) & 0x01010101u) << 7;
}

template <bool kWrite>
__global__ void __launch_bounds__(kThreads)
utf8_to_utf16_kernel(const uint8_t *__restrict__ in_al, uint16_t *__restrict__ out, Launch L)
{
    __shared__ __align__(16) uint8_t s_out[kWrite ? 2 * kStage8 + 16 : 16];
    __shared__ uint32_t s_first[kThreads], s_last[kThreads];
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_chunk, s_halo_prev, s_halo_next, s_err_units;
    __shared__ unsigned long long s_err, s_excl;

    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        s_chunk = atomicAdd(L.s.claim, 1u);
        s_err = ~0ull;
    }
    __syncthreads();
    const uint32_t chunk = s_chunk;
    if (chunk >= L.num_chunks) {   // counter left dirty by an aborted launch
        if (tid == 0) atomicOr(L.s.flags, 2u);
        finish_launch<kWrite>(L, kChunk8);
        return;
    }
    const int64_t lo = L.head, hi = (int64_t)L.head + (int64_t)L.n;
    const int64_t v0 = (int64_t)chunk * kChunk8;
    const int64_t vt = v0 + (int64_t)tid * kPer8;

    // ---- load 32 bytes (two aligned 16-byte blocks) ------------------------
    uint32_t w[10];
    {
        uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
        if (vt < hi) a = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt));
        if (vt + 16 < hi) b = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt + 16));
        w[1] = a.x; w[2] = a.y; w[3] = a.z; w[4] = a.w;
        w[5] = b.x; w[6] = b.y; w[7] = b.z; w[8] = b.w;
    }
    uint32_t vmask = 0xFFFFFFFFu;
    if (vt < lo || vt + kPer8 > hi) {          // buffer edges only
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

    // ---- pass 1: output units per thread (1 per non-continuation byte, +1 for >= F0)
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t x = w[1 + j];
        const uint32_t vm = spread4((vmask >> (4 * j)) & 0xFu);
        cnt += __popc(~cont_bits(x) & vm) + __popc(ge_f0_bits(x) & vm);
    }
    __syncthreads();   // s_first / s_last / halos visible
    w[0] = tid ? s_last[tid - 1] : s_halo_prev;
    w[9] = tid + 1 < kThreads ? s_first[tid + 1] : s_halo_next;

    uint32_t agg;
    const uint32_t t_off = block_exclusive_scan(cnt, s_warp, &agg);
    if (tid == 0)
        st_relaxed(&L.s.status[chunk],
                   pack_status(chunk == 0 ? kFlagInclusive : kFlagAggregate, L.epoch, agg));

    // ---- pass 2: decode, validate, stage -----------------------------------
    uint16_t *s16 = reinterpret_cast<uint16_t *>(s_out);
    uint32_t o = t_off;
    int e_kind = 0, e_pos = 0;
    uint32_t e_units = 0;
#pragma unroll
    for (int i = 0; i < kPer8; i++) {
        const int j = (i >> 2) + 1;
        const int sh = (i & 3) * 8;
        const uint32_t xf = __funnelshift_r(w[j], w[j + 1], sh);   // bytes i .. i+3
        const uint32_t xb = __funnelshift_r(w[j - 1], w[j], sh);   // bytes i-4 .. i-1
        const uint32_t b0 = xf & 0xFFu;
        const bool cont = (b0 & 0xC0u) == 0x80u;
        const uint32_t nunits = cont ? 0u : (b0 >= 0xF0u ? 2u : 1u);
        int kind = 0;
        uint32_t u1 = b0, u2 = 0;
        if (cont) {
            const uint32_t p1 = xb >> 24, p2 = (xb >> 16) & 0xFFu, p3 = (xb >> 8) & 0xFFu;
            if (!(p1 >= 0xC0u || p2 >= 0xE0u || p3 >= 0xF0u)) kind = kTooLong;
        } else if (b0 >= 0x80u) {
            if (b0 < 0xC2u) {
                kind = kOverlong;
            } else if (b0 >= 0xF5u) {
                kind = kHeaderBits;
            } else {
                const uint32_t len = b0 < 0xE0u ? 2u : (b0 < 0xF0u ? 3u : 4u);
                const uint32_t c = (xf ^ 0x80808080u) & 0xC0C0C0C0u;   // zero byte = continuation
                const uint32_t need = len == 2 ? 0x0000FF00u : (len == 3 ? 0x00FFFF00u : 0xFFFFFF00u);
                if (c & need) {
                    kind = kTooShort;
                } else {
                    const uint32_t b1 = (xf >> 8) & 0x3Fu, b2 = (xf >> 16) & 0x3Fu, b3 = xf >> 24 & 0x3Fu;
                    uint32_t cp;
                    if (len == 2) cp = ((b0 & 0x1Fu) << 6) | b1;
                    else if (len == 3) cp = ((b0 & 0x0Fu) << 12) | (b1 << 6) | b2;
                    else cp = ((b0 & 0x07u) << 18) | (b1 << 12) | (b2 << 6) | b3;
                    if (len == 3 && cp < 0x800u) kind = kOverlong;
                    else if (len == 3 && (cp & 0xF800u) == 0xD800u) kind = kSurrogate;
                    else if (len == 4 && cp < 0x10000u) kind = kOverlong;
                    else if (len == 4 && cp > 0x10FFFFu) kind = kTooLarge;
                    if (len == 4) {
                        u1 = 0xD7C0u + (cp >> 10);
                        u2 = 0xDC00u | (cp & 0x3FFu);
                    } else {
                        u1 = cp;
                    }
                }
            }
        }
        if ((vmask >> i) & 1u) {
            if (kWrite && kind == 0 && nunits && o + nunits <= kStage8) {
                s16[o] = (uint16_t)u1;
                if (nunits == 2) s16[o + 1] = (uint16_t)u2;
            }
            if (kind != 0 && e_kind == 0) {
                e_kind = kind;
                e_pos = i;
                e_units = o;
            }
            o += nunits;
        }
    }

    // ---- first error of the chunk -------------------------------------------
    if (e_kind) {
        const uint64_t pos = (uint64_t)(vt + e_pos - lo);
        atomicMin(&s_err, (pos << 8) | (uint64_t)e_kind);
    }
    __syncthreads();
    const unsigned long long blk_err = s_err;
    if (blk_err != ~0ull && e_kind) {
        const uint64_t pos = (uint64_t)(vt + e_pos - lo);
        if (((pos << 8) | (uint64_t)e_kind) == blk_err) s_err_units = e_units;
    }

    // ---- chunk offset: decoupled look-back ---------------------------------
    if (tid < 32) {
        uint64_t excl = 0;
        if (chunk > 0) {
            excl = lookback(L, chunk);
            if (tid == 0)
                st_relaxed(&L.s.status[chunk], pack_status(kFlagInclusive, L.epoch, excl + agg));
        }
        if (tid == 0) s_excl = excl;
    }
    __syncthreads();
    const uint64_t excl = s_excl;

    if (kWrite && excl < L.cap) {
        const uint64_t room = L.cap - excl;
        uint32_t nw = agg < kStage8 ? agg : kStage8;
        if (nw > room) nw = (uint32_t)room;
        block_store_bytes(s_out, reinterpret_cast<uint8_t *>(out + excl), 2u * nw);
    }
    if (tid == 0 && blk_err != ~0ull) {
        L.s.err_prefix[chunk] = excl + s_err_units;
        __threadfence();
        atomicMin(L.s.err, blk_err);
    }
    finish_launch<kWrite>(L, kChunk8);
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
