/*
 * Oracle: plain, slow, obviously-correct scalar UTF-8 <-> UTF-16LE transcoder
 * (and UTF-8 <-> UTF-32LE, the third format of Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header, table or constant with the CUDA
 * library: every rule below is written out from the paper's statement of the
 * encodings (Clausecker & Lemire, "Transcoding Unicode Characters with AVX-512
 * Instructions", arXiv 2212.05098):
 *
 *   - Fig. 1(a): bit-by-bit correspondence of the ASCII, 2-byte, 3-byte and
 *     4-byte cases between UTF-16 and UTF-8.
 *   - Sec. 2.1 (UTF-16): BMP code points are stored as one 16-bit word;
 *     others have 0x10000 subtracted, are split into two 10-bit halves tagged
 *     0xD800 (high) and 0xDC00 (low), high first; every high surrogate must be
 *     followed by a low surrogate and vice versa. Little-endian words; no BOM
 *     handling.
 *   - Sec. 2.2 (UTF-8) and Table 1: byte types (ASCII 00-7F, continuation
 *     80-BF, 2-byte lead C2-DF, 3-byte lead E0-EF, 4-byte lead F0-F4);
 *     shortest form only; nothing above U+10FFFF; C0, C1, F5-FF never occur.
 *   - Sec. 6.4 (Input Validation), rules 1-6: bad bytes, lead/continuation
 *     matching, no stray continuations, overlong forms, > U+10FFFF, surrogates.
 *   - Sec. 6.4 and Sec. 7.4/7.5: on an encoding error the valid prefix is
 *     transcoded and the number of input units before the first error is
 *     reported.
 *
 * Readings where the paper is silent (error kinds, precedence, capacity) are
 * the library's documented conventions:
 *   - a byte-level class error is reported first (stray continuation ->
 *     TOO_LONG, C0/C1 -> OVERLONG, F5-FF -> HEADER_BITS), then structure
 *     (missing continuation or end of input -> TOO_SHORT at the lead byte),
 *     then value (OVERLONG / SURROGATE / TOO_LARGE at the lead byte);
 *   - UTF-16: an unpaired high surrogate -> LONE_HIGH_SURROGATE at it, an
 *     unpaired low surrogate -> LONE_LOW_SURROGATE at it;
 *   - output units are written only below the capacity; an encoding error
 *     takes precedence over a too-small output; OUTPUT_TOO_SMALL reports the
 *     full required length.
 *
 * UTF-16LE data is handled as bytes (low byte first) so that the oracle does
 * not depend on the host's byte order.
 */
#include <stddef.h>
#include <stdint.h>

/* Status codes, numerically identical to the library's public enum so the
 * test-suite can compare them directly (the only thing the two share is this
 * numbering, restated here). */
enum {
    OR_OK = 0,
    OR_HEADER_BITS = 1,
    OR_TOO_SHORT = 2,
    OR_TOO_LONG = 3,
    OR_OVERLONG = 4,
    OR_TOO_LARGE = 5,
    OR_SURROGATE = 6,
    OR_LONE_HIGH_SURROGATE = 7,
    OR_LONE_LOW_SURROGATE = 8,
    OR_OUTPUT_TOO_SMALL = 16
};

typedef struct {
    int32_t status;
    uint64_t in_offset; /* input units consumed (n) or index of first error */
    uint64_t out_len;   /* output units of the whole input / the valid prefix */
} oracle_result;

static int is_continuation(uint8_t b) { return b >= 0x80 && b <= 0xBF; }

static void put16(uint8_t *out, uint64_t cap_units, uint64_t *o, uint32_t w)
{
    /* One UTF-16LE word: low byte first (Sec. 2.1, little-endian). */
    if (out && *o < cap_units) {
        out[2 * *o] = (uint8_t)(w & 0xFF);
        out[2 * *o + 1] = (uint8_t)(w >> 8);
    }
    (*o)++;
}

static void put8(uint8_t *out, uint64_t cap_bytes, uint64_t *o, uint32_t b)
{
    if (out && *o < cap_bytes) out[*o] = (uint8_t)b;
    (*o)++;
}

static void finish(oracle_result *r, int32_t err, uint64_t p, uint64_t n,
                   uint64_t o, uint64_t cap, int check_cap)
{
    if (err != OR_OK) {
        r->status = err;
        r->in_offset = p;
        r->out_len = o;
    } else {
        r->status = (check_cap && o > cap) ? OR_OUTPUT_TOO_SMALL : OR_OK;
        r->in_offset = n;
        r->out_len = o;
    }
}

/*
 * UTF-8 -> UTF-16LE, one character at a time from the start (Sec. 2.2,
 * Table 1, Fig. 1(a); validation rules of Sec. 6.4).
 * out: cap_units 16-bit words as 2*cap_units bytes (may be NULL when counting).
 */
static void u8_to_u16(const uint8_t *in, uint64_t n, uint8_t *out,
                      uint64_t cap_units, int check_cap, oracle_result *r)
{
    uint64_t p = 0, o = 0;
    int32_t err = OR_OK;
    while (p < n) {
        uint8_t b = in[p];
        uint32_t len, cp, k;
        if (b <= 0x7F) {                 /* ASCII lead byte */
            put16(out, cap_units, &o, b);
            p += 1;
            continue;
        }
        if (b <= 0xBF) { err = OR_TOO_LONG; break; }     /* stray continuation */
        if (b <= 0xC1) { err = OR_OVERLONG; break; }     /* C0/C1: 2-byte overlong */
        if (b <= 0xDF) len = 2;
        else if (b <= 0xEF) len = 3;
        else if (b <= 0xF4) len = 4;
        else { err = OR_HEADER_BITS; break; }            /* F5-FF never used */

        /* Structure: the lead must be followed by len-1 continuation bytes. */
        if (n - p < len) { err = OR_TOO_SHORT; break; }
        for (k = 1; k < len; k++)
            if (!is_continuation(in[p + k])) break;
        if (k < len) { err = OR_TOO_SHORT; break; }

        /* Payload bits per Fig. 1(a): lead keeps 5/4/3 bits, each continuation 6. */
        if (len == 2) {
            cp = ((uint32_t)(b & 0x1F) << 6) | (in[p + 1] & 0x3F);
        } else if (len == 3) {
            cp = ((uint32_t)(b & 0x0F) << 12) | ((uint32_t)(in[p + 1] & 0x3F) << 6)
               | (in[p + 2] & 0x3F);
        } else {
            cp = ((uint32_t)(b & 0x07) << 18) | ((uint32_t)(in[p + 1] & 0x3F) << 12)
               | ((uint32_t)(in[p + 2] & 0x3F) << 6) | (in[p + 3] & 0x3F);
        }

        /* Value: shortest form, no surrogates, at most U+10FFFF (rules 4-6). */
        if (len == 3 && cp < 0x800) { err = OR_OVERLONG; break; }
        if (len == 3 && cp >= 0xD800 && cp <= 0xDFFF) { err = OR_SURROGATE; break; }
        if (len == 4 && cp < 0x10000) { err = OR_OVERLONG; break; }
        if (len == 4 && cp > 0x10FFFF) { err = OR_TOO_LARGE; break; }

        if (cp <= 0xFFFF) {
            put16(out, cap_units, &o, cp);
        } else {
            /* Sec. 2.1: subtract 0x10000, split 10/10, tag D800 / DC00. */
            uint32_t v = cp - 0x10000;
            put16(out, cap_units, &o, 0xD800 + (v >> 10));
            put16(out, cap_units, &o, 0xDC00 + (v & 0x3FF));
        }
        p += len;
    }
    finish(r, err, p, n, o, cap_units, check_cap);
}

/*
 * UTF-16LE -> UTF-8, one word at a time from the start (Sec. 2.1 surrogate
 * rules; Fig. 1(a) byte layouts; sequencing check of Sec. 7.4).
 * in: n_units words as 2*n_units bytes, low byte first.
 */
static void u16_to_u8(const uint8_t *in, uint64_t n, uint8_t *out,
                      uint64_t cap_bytes, int check_cap, oracle_result *r)
{
    uint64_t p = 0, o = 0;
    int32_t err = OR_OK;
    while (p < n) {
        uint32_t u = (uint32_t)in[2 * p] | ((uint32_t)in[2 * p + 1] << 8);
        uint32_t cp;
        uint64_t used = 1;
        if (u >= 0xD800 && u <= 0xDBFF) {            /* high surrogate */
            uint32_t v;
            if (p + 1 >= n) { err = OR_LONE_HIGH_SURROGATE; break; }
            v = (uint32_t)in[2 * p + 2] | ((uint32_t)in[2 * p + 3] << 8);
            if (v < 0xDC00 || v > 0xDFFF) { err = OR_LONE_HIGH_SURROGATE; break; }
            cp = 0x10000 + ((u - 0xD800) << 10) + (v - 0xDC00);
            used = 2;
        } else if (u >= 0xDC00 && u <= 0xDFFF) {     /* low surrogate, unpaired */
            err = OR_LONE_LOW_SURROGATE;
            break;
        } else {
            cp = u;
        }

        if (cp <= 0x7F) {
            put8(out, cap_bytes, &o, cp);
        } else if (cp <= 0x7FF) {
            put8(out, cap_bytes, &o, 0xC0 | (cp >> 6));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        } else if (cp <= 0xFFFF) {
            put8(out, cap_bytes, &o, 0xE0 | (cp >> 12));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 6) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        } else {
            put8(out, cap_bytes, &o, 0xF0 | (cp >> 18));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 12) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 6) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        }
        p += used;
    }
    finish(r, err, p, n, o, cap_bytes, check_cap);
}

/* ---- UTF-32LE ---------------------------------------------------------- */

static void put32(uint8_t *out, uint64_t cap_units, uint64_t *o, uint32_t cp)
{
    /* One UTF-32LE unit: the code point itself, low byte first (Sec. 2). */
    if (out && *o < cap_units) {
        out[4 * *o] = (uint8_t)(cp & 0xFF);
        out[4 * *o + 1] = (uint8_t)((cp >> 8) & 0xFF);
        out[4 * *o + 2] = (uint8_t)((cp >> 16) & 0xFF);
        out[4 * *o + 3] = (uint8_t)(cp >> 24);
    }
    (*o)++;
}

/*
 * UTF-8 -> UTF-32LE: the same character-by-character decoding and the same
 * validation as UTF-8 -> UTF-16LE above (Sec. 2.2, Table 1, Fig. 1(a),
 * Sec. 6.4); every character becomes one 32-bit unit holding its code point.
 */
static void u8_to_u32(const uint8_t *in, uint64_t n, uint8_t *out,
                      uint64_t cap_units, int check_cap, oracle_result *r)
{
    uint64_t p = 0, o = 0;
    int32_t err = OR_OK;
    while (p < n) {
        uint8_t b = in[p];
        uint32_t len, cp, k;
        if (b <= 0x7F) {
            put32(out, cap_units, &o, b);
            p += 1;
            continue;
        }
        if (b <= 0xBF) { err = OR_TOO_LONG; break; }
        if (b <= 0xC1) { err = OR_OVERLONG; break; }
        if (b <= 0xDF) len = 2;
        else if (b <= 0xEF) len = 3;
        else if (b <= 0xF4) len = 4;
        else { err = OR_HEADER_BITS; break; }
        if (n - p < len) { err = OR_TOO_SHORT; break; }
        for (k = 1; k < len; k++)
            if (!is_continuation(in[p + k])) break;
        if (k < len) { err = OR_TOO_SHORT; break; }
        if (len == 2) {
            cp = ((uint32_t)(b & 0x1F) << 6) | (in[p + 1] & 0x3F);
        } else if (len == 3) {
            cp = ((uint32_t)(b & 0x0F) << 12) | ((uint32_t)(in[p + 1] & 0x3F) << 6)
               | (in[p + 2] & 0x3F);
        } else {
            cp = ((uint32_t)(b & 0x07) << 18) | ((uint32_t)(in[p + 1] & 0x3F) << 12)
               | ((uint32_t)(in[p + 2] & 0x3F) << 6) | (in[p + 3] & 0x3F);
        }
        if (len == 3 && cp < 0x800) { err = OR_OVERLONG; break; }
        if (len == 3 && cp >= 0xD800 && cp <= 0xDFFF) { err = OR_SURROGATE; break; }
        if (len == 4 && cp < 0x10000) { err = OR_OVERLONG; break; }
        if (len == 4 && cp > 0x10FFFF) { err = OR_TOO_LARGE; break; }
        put32(out, cap_units, &o, cp);
        p += len;
    }
    finish(r, err, p, n, o, cap_units, check_cap);
}

/*
 * UTF-32LE -> UTF-8, one unit at a time (Sec. 2: a UTF-32 unit is the code
 * point). A unit above U+10FFFF is TOO_LARGE and one in D800-DFFF is
 * SURROGATE (the library's convention, named like the UTF-8 value errors of
 * Sec. 6.4, rules 5 and 6), at the unit's index. Bytes per Fig. 1(a).
 */
static void u32_to_u8(const uint8_t *in, uint64_t n, uint8_t *out,
                      uint64_t cap_bytes, int check_cap, oracle_result *r)
{
    uint64_t p = 0, o = 0;
    int32_t err = OR_OK;
    while (p < n) {
        uint32_t cp = (uint32_t)in[4 * p] | ((uint32_t)in[4 * p + 1] << 8)
                    | ((uint32_t)in[4 * p + 2] << 16) | ((uint32_t)in[4 * p + 3] << 24);
        if (cp > 0x10FFFF) { err = OR_TOO_LARGE; break; }
        if (cp >= 0xD800 && cp <= 0xDFFF) { err = OR_SURROGATE; break; }
        if (cp <= 0x7F) {
            put8(out, cap_bytes, &o, cp);
        } else if (cp <= 0x7FF) {
            put8(out, cap_bytes, &o, 0xC0 | (cp >> 6));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        } else if (cp <= 0xFFFF) {
            put8(out, cap_bytes, &o, 0xE0 | (cp >> 12));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 6) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        } else {
            put8(out, cap_bytes, &o, 0xF0 | (cp >> 18));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 12) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | ((cp >> 6) & 0x3F));
            put8(out, cap_bytes, &o, 0x80 | (cp & 0x3F));
        }
        p += 1;
    }
    finish(r, err, p, n, o, cap_bytes, check_cap);
}

/* ---- exported entry points (ctypes) ------------------------------------ */

void oracle_utf8_to_utf16le(const uint8_t *in, uint64_t n_bytes, uint8_t *out,
                            uint64_t cap_units, oracle_result *r)
{
    u8_to_u16(in, n_bytes, out, cap_units, 1, r);
}

void oracle_utf16le_to_utf8(const uint8_t *in, uint64_t n_units, uint8_t *out,
                            uint64_t cap_bytes, oracle_result *r)
{
    u16_to_u8(in, n_units, out, cap_bytes, 1, r);
}

/* Length-only: the same scan, nothing written, no capacity. */
void oracle_utf16_length_from_utf8(const uint8_t *in, uint64_t n_bytes, oracle_result *r)
{
    u8_to_u16(in, n_bytes, NULL, 0, 0, r);
}

void oracle_utf8_length_from_utf16le(const uint8_t *in, uint64_t n_units, oracle_result *r)
{
    u16_to_u8(in, n_units, NULL, 0, 0, r);
}

void oracle_utf8_to_utf32le(const uint8_t *in, uint64_t n_bytes, uint8_t *out,
                            uint64_t cap_units, oracle_result *r)
{
    u8_to_u32(in, n_bytes, out, cap_units, 1, r);
}

void oracle_utf32le_to_utf8(const uint8_t *in, uint64_t n_units, uint8_t *out,
                            uint64_t cap_bytes, oracle_result *r)
{
    u32_to_u8(in, n_units, out, cap_bytes, 1, r);
}

void oracle_utf32_length_from_utf8(const uint8_t *in, uint64_t n_bytes, oracle_result *r)
{
    u8_to_u32(in, n_bytes, NULL, 0, 0, r);
}

void oracle_utf8_length_from_utf32le(const uint8_t *in, uint64_t n_units, oracle_result *r)
{
    u32_to_u8(in, n_units, NULL, 0, 0, r);
}
