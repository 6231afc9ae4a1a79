// UTF-16LE -> UTF-8, validating, single pass (paper Sec. 7).
//
// Work decomposition: chunks of kChunk16 words, one CTA per chunk (claimed
// in order from an atomic counter), 16 words per thread plus one word of
// look-behind and one of look-ahead (the paper's surrogate carry c and
// look-ahead word L of Sec. 7 and Sec. 7.4).
//
// Ownership: a surrogate pair belongs to the owner of its high surrogate,
// which emits all four bytes; its low surrogate emits nothing.
//
// Output length per word (Sec. 7, plan of attack): 1 byte below U+0080, 2
// below U+0800, 3 for other BMP words, 4 for a high surrogate (the pair), 0
// for a low surrogate. Counted two words at a time on 16-bit lanes.
//
// Paths: like the paper's fast paths (ASCII / 1-2 byte / no surrogates /
// default, Sec. 7.1), each warp picks one from its own words: all below
// U+0800 (1-2 byte encoder, no validation needed), no surrogates (1-3 byte
// encoder, no validation needed), or the general path with the surrogate
// join and the sequencing check. The choice is warp-uniform, so lanes never
// diverge on it.
//
// Validation (Sec. 7.4), general path only: a high surrogate not followed by
// a low one is LONE_HIGH at the high, a low surrogate not preceded by a high
// one is LONE_LOW at the low. The smallest offending position is where the
// sequential decoder stops, so the block-wide and grid-wide minimum of
// (position, kind) is the first error and all output offsets before it are
// exact.
//
// Encoding (Fig. 1(a), Sec. 7.2-7.3): pairs are joined with
// (hi << 10) + lo + 0xFCA02400 (32-bit wrap); the 6-bit groups of the code
// point get the tag bits C0/E0/F0 (lead) and 80 (continuation). Bytes are
// staged in shared memory at the thread's scanned offset and written with
// 16-byte stores after the look-back has placed the chunk.
#include "kernels.h"

namespace gbu {

namespace {

constexpr int kPer16 = kChunk16 / kThreads;   // 16 words per thread
static_assert(kPer16 == 16, "one 16-bit position mask per thread");
// Staging capacity in bytes. A chunk's valid words need at most
// 3 * kChunk16 + 1 bytes (3 per BMP word; a pair gives 4 bytes for 2 words,
// and a high surrogate that is the chunk's last word adds 4 for 1). Offsets
// past an error can grow up to 4 bytes per word, so stores and the write-out
// are bounded by this capacity; what lies past an error is unspecified.
constexpr uint32_t kStage16 = 3 * kChunk16 + 8;

// Indicator bit 15 of each 16-bit lane of w (two words per register).
__device__ __forceinline__ uint32_t ge80_lanes(uint32_t w)    // word >= 0x0080
{
    return (((w & 0x7F807F80u) + 0x7F807F80u) | w) & 0x80008000u;
}
__device__ __forceinline__ uint32_t ge800_lanes(uint32_t w)   // word >= 0x0800
{
    return (((w & 0x78007800u) + 0x78007800u) | w) & 0x80008000u;
}
__device__ __forceinline__ uint32_t surr_lanes(uint32_t w)    // D800-DFFF (exact:
{                                                              // low 11 bits zero)
    const uint32_t v = (w & 0xF800F800u) ^ 0xD800D800u;
    return (v - 0x00010001u) & ~v & 0x80008000u;
}

__device__ __forceinline__ uint32_t lane(const uint32_t *w, int i)   // word i, i in [-2, 18)
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

template <bool kWrite>
__global__ void __launch_bounds__(kThreads)
utf16_to_utf8_kernel(const uint16_t *__restrict__ in_al, uint8_t *__restrict__ out, Launch L)
{
    __shared__ __align__(16) uint8_t s_out[kWrite ? kStage16 + 16 : 16];
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
            finish_launch<kWrite>(L, kChunk16);
        }
        return;
    }
    const int64_t lo = L.head, hi = (int64_t)L.head + (int64_t)L.n;   // in words
    const int64_t v0 = (int64_t)chunk * kChunk16;
    const int64_t vt = v0 + (int64_t)tid * kPer16;

    // w[0]: words -2,-1; w[1..8]: own words 0..15; w[9]: words 16,17
    uint32_t w[10];
    {
        uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
        if (vt < hi) a = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt));
        if (vt + 8 < hi) b = __ldcs(reinterpret_cast<const uint4 *>(in_al + vt + 8));
        w[1] = a.x; w[2] = a.y; w[3] = a.z; w[4] = a.w;
        w[5] = b.x; w[6] = b.y; w[7] = b.z; w[8] = b.w;
    }
    uint32_t vmask = 0xFFFFu;
    const bool edge = vt < lo || vt + kPer16 > hi;
    if (edge) {
        vmask = 0;
#pragma unroll
        for (int i = 0; i < kPer16; i++)
            if (vt + i >= lo && vt + i < hi) vmask |= 1u << i;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            uint32_t keep = 0;
            if ((vmask >> (2 * j)) & 1u) keep |= 0xFFFFu;
            if ((vmask >> (2 * j + 1)) & 1u) keep |= 0xFFFF0000u;
            w[1 + j] &= keep;
        }
    }
    s_first[tid] = w[1];
    s_last[tid] = w[8];
    if (tid == 0) {
        uint32_t h = 0;
        if (v0 >= 2 && v0 - 2 < hi) h = *reinterpret_cast<const uint32_t *>(in_al + v0 - 2);
        uint32_t keep = 0;
        if (v0 - 2 >= lo && v0 - 2 < hi) keep |= 0xFFFFu;
        if (v0 - 1 >= lo && v0 - 1 < hi) keep |= 0xFFFF0000u;
        s_halo_prev = h & keep;
    }
    if (tid == kThreads - 1) {
        uint32_t h = 0;
        const int64_t vn = v0 + kChunk16;
        if (vn < hi) h = *reinterpret_cast<const uint32_t *>(in_al + vn);
        uint32_t keep = 0;
        if (vn < hi) keep |= 0xFFFFu;
        if (vn + 1 < hi) keep |= 0xFFFF0000u;
        s_halo_next = h & keep;
    }

    // ---- pass 1: output bytes per thread, path flags ------------------------
    uint32_t cnt = 0, any800 = 0, anysur = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t x = w[1 + j];
        const uint32_t a = ge80_lanes(x), b = ge800_lanes(x), s = surr_lanes(x);
        const uint32_t lo_bit = (x << 5) & 0x80008000u;   // bit 10: low surrogate
        uint32_t vm = 0x80008000u;
        if (edge) vm = (((vmask >> (2 * j)) & 1u) << 15) | (((vmask >> (2 * j + 1)) & 1u) << 31);
        // 1 + [>=80] + [>=800] + [high] - 3 [low]
        cnt += __popc(vm) + __popc(a & vm) + __popc(b & vm) + __popc(s & ~lo_bit & vm) -
               3u * __popc(s & lo_bit & vm);
        any800 |= b;
        anysur |= s;
    }
    __syncthreads();
    w[0] = tid ? s_last[tid - 1] : s_halo_prev;
    w[9] = tid + 1 < kThreads ? s_first[tid + 1] : s_halo_next;

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

    // ---- pass 2: encode (and validate) ------------------------------------
    const bool warp_general = __any_sync(kFull, anysur != 0 || edge);
    const bool warp_12 = !__any_sync(kFull, any800 != 0);
    if (!warp_general) {
        // no surrogates in this warp: every word is valid
        if (kWrite) {
            uint8_t *p = s_out + t_off;
            if (warp_12) {
#pragma unroll
                for (int i = 0; i < kPer16; i++) {
                    const uint32_t u = lane(w, i);
                    const bool big = u >= 0x80u;
                    const uint32_t v = big ? enc2(u) : u;
                    p[0] = (uint8_t)v;
                    if (big) p[1] = (uint8_t)(v >> 8);
                    p += big ? 2 : 1;
                }
            } else {
#pragma unroll
                for (int i = 0; i < kPer16; i++) {
                    const uint32_t u = lane(w, i);
                    const bool c2 = u >= 0x80u, c3 = u >= 0x800u;
                    const uint32_t v = c3 ? enc3(u) : (c2 ? enc2(u) : u);
                    p[0] = (uint8_t)v;
                    if (c2) p[1] = (uint8_t)(v >> 8);
                    if (c3) p[2] = (uint8_t)(v >> 16);
                    p += 1 + (c2 ? 1 : 0) + (c3 ? 1 : 0);
                }
            }
        }
    } else {
        uint64_t key = ~0ull;
        uint32_t o = t_off;
#pragma unroll
        for (int i = 0; i < kPer16; i++) {
            const uint32_t u = lane(w, i), pv = lane(w, i - 1), nx = lane(w, i + 1);
            const bool is_hi = (u & 0xFC00u) == 0xD800u;
            const bool is_lo = (u & 0xFC00u) == 0xDC00u;
            uint32_t kind = 0;
            if (is_hi && (nx & 0xFC00u) != 0xDC00u) kind = kLoneHigh;
            if (is_lo && (pv & 0xFC00u) != 0xD800u) kind = kLoneLow;
            const bool c2 = u >= 0x80u, c3 = u >= 0x800u;
            const uint32_t len = is_lo ? 0u : (is_hi ? 4u : 1u + (c2 ? 1u : 0u) + (c3 ? 1u : 0u));
            uint32_t v;
            if (is_hi) {
                const uint32_t cp = (u << 10) + nx + 0xFCA02400u;
                v = (cp >> 18) | ((cp >> 4) & 0x3F00u) | ((cp << 10) & 0x3F0000u) |
                    ((cp << 24) & 0x3F000000u) | 0x808080F0u;
            } else {
                v = c3 ? enc3(u) : (c2 ? enc2(u) : u);
            }
            if ((vmask >> i) & 1u) {
                if (kWrite && o + len <= kStage16) {
                    uint8_t *q = s_out + o;
                    if (len >= 1) q[0] = (uint8_t)v;
                    if (len >= 2) q[1] = (uint8_t)(v >> 8);
                    if (len >= 3) q[2] = (uint8_t)(v >> 16);
                    if (len >= 4) q[3] = (uint8_t)(v >> 24);
                }
                if (kind != 0 && key == ~0ull)
                    key = err_key((uint64_t)(vt + i - lo), kind, o);
                o += len;
            }
        }
        if (key != ~0ull) atomicMin(&s_err, key);
    }
    __syncthreads();
    const uint64_t excl = s_excl;

    if (kWrite && excl < L.cap) {
        const uint64_t room = L.cap - excl;
        uint32_t nw = agg < kStage16 ? agg : kStage16;
        if (nw > room) nw = (uint32_t)room;
        block_store_bytes(s_out, out + excl, nw);
    }
    if (tid == 0) {
        publish_error(L, chunk, s_err, excl);
        finish_launch<kWrite>(L, kChunk16);
    }
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

}  // namespace

const uint16_t *plan_utf16(const uint16_t *in, uint64_t n, Launch &L)
{
    const uintptr_t p = reinterpret_cast<uintptr_t>(in);
    L.head = (uint32_t)((p & 15u) >> 1);
    L.n = n;
    L.num_chunks = (uint32_t)((L.head + n + kChunk16 - 1) / kChunk16);
    return reinterpret_cast<const uint16_t *>(p & ~(uintptr_t)15u);
}

cudaError_t launch_utf16_to_utf8(const uint16_t *in_aligned, uint8_t *out, bool write,
                                 const Launch &L, cudaStream_t stream)
{
    if (write)
        utf16_to_utf8_kernel<true><<<L.num_chunks, kThreads, 0, stream>>>(in_aligned, out, L);
    else
        utf16_to_utf8_kernel<false><<<L.num_chunks, kThreads, 0, stream>>>(in_aligned, out, L);
    return cudaGetLastError();
}

cudaError_t launch_write_result(ResultSlot *dst, int32_t status, uint64_t in_offset,
                                uint64_t out_len, cudaStream_t stream)
{
    write_result_kernel<<<1, 1, 0, stream>>>(dst, status, in_offset, out_len);
    return cudaGetLastError();
}

}  // namespace gbu
