// UTF-16LE -> UTF-8, validating, single pass (paper Sec. 7).
//
// Work decomposition: chunks of kChunk16 words, one CTA per chunk (claimed
// in order from an atomic counter), 16 words per thread plus one word of
// look-ahead and one of look-behind (the paper's look-ahead word L and
// surrogate carry c of Sec. 7 and Sec. 7.4).
//
// Ownership: a surrogate pair belongs to the owner of its high surrogate,
// which emits all four bytes; its low surrogate emits nothing.
//
// Validation is local (Sec. 7.4): a high surrogate not followed by a low one
// is LONE_HIGH at the high, a low surrogate not preceded by a high one is
// LONE_LOW at the low. The smallest offending position is where the
// sequential decoder stops, so the block-wide and grid-wide minimum of
// (position, kind) is the first error and all output offsets before it are
// exact.
//
// Encoding (Fig. 1(a), Sec. 7.2-7.3): pairs are joined with
// (hi << 10) + lo + 0xFCA02400 (32-bit wrap); the 6-bit groups of the code
// point get the tag bits C0/E0/F0 (lead) and 80 (continuation). Bytes are
// staged in shared memory at the thread's scanned offset and written with
// 16-byte stores.
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

__device__ __forceinline__ uint32_t out_len8(uint32_t u)
{
    // bytes emitted by the owner of word u: 1 / 2 / 3, 4 for a high surrogate
    // (the pair), 0 for a low surrogate (Sec. 7, output sizes)
    if (u < 0x80u) return 1;
    if (u < 0x800u) return 2;
    if ((u & 0xF800u) != 0xD800u) return 3;
    return (u & 0x0400u) ? 0u : 4u;
}

template <bool kWrite>
__global__ void __launch_bounds__(kThreads)
utf16_to_utf8_kernel(const uint16_t *__restrict__ in_al, uint8_t *__restrict__ out, Launch L)
{
    __shared__ __align__(16) uint8_t s_out[kWrite ? kStage16 + 16 : 16];
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
        finish_launch<kWrite>(L, kChunk16);
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
    if (vt < lo || vt + kPer16 > hi) {
        vmask = 0;
#pragma unroll
        for (int i = 0; i < kPer16; i++)
            if (vt + i >= lo && vt + i < hi) vmask |= 1u << i;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            uint32_t keep = 0;
            if (vt + 2 * j >= lo && vt + 2 * j < hi) keep |= 0xFFFFu;
            if (vt + 2 * j + 1 >= lo && vt + 2 * j + 1 < hi) keep |= 0xFFFF0000u;
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

    // ---- pass 1: output bytes per thread -----------------------------------
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kPer16; i++) {
        const uint32_t u = (w[1 + (i >> 1)] >> (16 * (i & 1))) & 0xFFFFu;
        if ((vmask >> i) & 1u) cnt += out_len8(u);
    }
    __syncthreads();
    w[0] = tid ? s_last[tid - 1] : s_halo_prev;
    w[9] = tid + 1 < kThreads ? s_first[tid + 1] : s_halo_next;

    uint32_t agg;
    const uint32_t t_off = block_exclusive_scan(cnt, s_warp, &agg);
    if (tid == 0)
        st_relaxed(&L.s.status[chunk],
                   pack_status(chunk == 0 ? kFlagInclusive : kFlagAggregate, L.epoch, agg));

    // ---- pass 2: encode, validate, stage -----------------------------------
    uint32_t o = t_off;
    int e_kind = 0, e_pos = 0;
    uint32_t e_units = 0;
#pragma unroll
    for (int i = 0; i < kPer16; i++) {
        const uint32_t u = (w[1 + (i >> 1)] >> (16 * (i & 1))) & 0xFFFFu;
        const uint32_t pv = (w[(i + 1) >> 1] >> (16 * ((i + 1) & 1))) & 0xFFFFu;   // word i-1
        const uint32_t nx = (w[1 + ((i + 1) >> 1)] >> (16 * ((i + 1) & 1))) & 0xFFFFu; // word i+1
        const bool is_hi = (u & 0xFC00u) == 0xD800u;
        const bool is_lo = (u & 0xFC00u) == 0xDC00u;
        int kind = 0;
        if (is_hi && (nx & 0xFC00u) != 0xDC00u) kind = kLoneHigh;
        if (is_lo && (pv & 0xFC00u) != 0xD800u) kind = kLoneLow;
        const uint32_t len = out_len8(u);
        uint32_t enc;
        if (len == 1) {
            enc = u;
        } else if (len == 2) {
            enc = (0xC0u | (u >> 6)) | ((0x80u | (u & 0x3Fu)) << 8);
        } else if (len == 3) {
            enc = (0xE0u | (u >> 12)) | ((0x80u | ((u >> 6) & 0x3Fu)) << 8) |
                  ((0x80u | (u & 0x3Fu)) << 16);
        } else {
            const uint32_t cp = (u << 10) + nx + 0xFCA02400u;
            enc = (0xF0u | (cp >> 18)) | ((0x80u | ((cp >> 12) & 0x3Fu)) << 8) |
                  ((0x80u | ((cp >> 6) & 0x3Fu)) << 16) | ((0x80u | (cp & 0x3Fu)) << 24);
        }
        if ((vmask >> i) & 1u) {
            if (kWrite && kind == 0 && o + len <= kStage16) {
                if (len >= 1) s_out[o] = (uint8_t)enc;
                if (len >= 2) s_out[o + 1] = (uint8_t)(enc >> 8);
                if (len >= 3) s_out[o + 2] = (uint8_t)(enc >> 16);
                if (len >= 4) s_out[o + 3] = (uint8_t)(enc >> 24);
            }
            if (kind != 0 && e_kind == 0) {
                e_kind = kind;
                e_pos = i;
                e_units = o;
            }
            o += len;
        }
    }

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
        uint32_t nw = agg < kStage16 ? agg : kStage16;
        if (nw > room) nw = (uint32_t)room;
        block_store_bytes(s_out, out + excl, nw);
    }
    if (tid == 0 && blk_err != ~0ull) {
        L.s.err_prefix[chunk] = excl + s_err_units;
        __threadfence();
        atomicMin(L.s.err, blk_err);
    }
    finish_launch<kWrite>(L, kChunk16);
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
