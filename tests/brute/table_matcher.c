/*
 * Exhaustive check of the oracle against an independent formulation.
 *
 * UTF-8: every string of 1, 2, 3 and 4 bytes is run through the oracle and
 * through a matcher of the well-formed byte-sequence table of the Unicode
 * Standard (Chapter 3, Table 3-7: each row gives the allowed range of every
 * byte position; the lead-byte ranges restate Table 1 of the paper). The
 * matcher never assembles a code point: it only compares bytes with ranges.
 * Status, first-error offset and output length must agree.
 *
 * UTF-16: every string of 1 and 2 units is run through the oracle and a
 * pairing matcher (Sec. 2.1: high D800-DBFF must be followed by low
 * DC00-DFFF and vice versa).
 *
 * Error kinds follow the library's convention: byte class first, then
 * structure (TOO_SHORT), then the restricted second-byte ranges of the table
 * (E0 -> OVERLONG, ED -> SURROGATE, F0 -> OVERLONG, F4 -> TOO_LARGE).
 *
 * Usage: table_matcher utf8|utf16 THREADS ; prints "mismatches N" and exits
 * non-zero on any mismatch.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t status; uint64_t in_offset; uint64_t out_len; } res_t;
void oracle_utf8_to_utf16le(const uint8_t *, uint64_t, uint8_t *, uint64_t, res_t *);
void oracle_utf16le_to_utf8(const uint8_t *, uint64_t, uint8_t *, uint64_t, res_t *);

enum { OK = 0, HEADER_BITS = 1, TOO_SHORT = 2, TOO_LONG = 3, OVERLONG = 4,
       TOO_LARGE = 5, SURROGATE = 6, LONE_HIGH = 7, LONE_LOW = 8 };

/* Table 3-7: {len, lo1, hi1, lo2, hi2, lo3, hi3, lo4, hi4, utf16 units} */
static const int T37[9][10] = {
    {1, 0x00, 0x7F, 0, 0, 0, 0, 0, 0, 1},
    {2, 0xC2, 0xDF, 0x80, 0xBF, 0, 0, 0, 0, 1},
    {3, 0xE0, 0xE0, 0xA0, 0xBF, 0x80, 0xBF, 0, 0, 1},
    {3, 0xE1, 0xEC, 0x80, 0xBF, 0x80, 0xBF, 0, 0, 1},
    {3, 0xED, 0xED, 0x80, 0x9F, 0x80, 0xBF, 0, 0, 1},
    {3, 0xEE, 0xEF, 0x80, 0xBF, 0x80, 0xBF, 0, 0, 1},
    {4, 0xF0, 0xF0, 0x90, 0xBF, 0x80, 0xBF, 0x80, 0xBF, 2},
    {4, 0xF1, 0xF3, 0x80, 0xBF, 0x80, 0xBF, 0x80, 0xBF, 2},
    {4, 0xF4, 0xF4, 0x80, 0x8F, 0x80, 0xBF, 0x80, 0xBF, 2},
};

static int in_range(int b, int lo, int hi) { return b >= lo && b <= hi; }

static void match8(const uint8_t *s, int n, res_t *r)
{
    int p = 0;
    uint64_t o = 0;
    while (p < n) {
        int row, hit = -1;
        for (row = 0; row < 9 && hit < 0; row++) {
            int len = T37[row][0], k, good = 1;
            if (p + len > n) continue;
            for (k = 0; k < len && good; k++)
                good = in_range(s[p + k], T37[row][1 + 2 * k], T37[row][2 + 2 * k]);
            if (good) hit = row;
        }
        if (hit >= 0) {
            o += T37[hit][9];
            p += T37[hit][0];
            continue;
        }
        /* no row matches at p: classify by the convention */
        {
            int b = s[p], kind;
            if (in_range(b, 0x80, 0xBF)) kind = TOO_LONG;
            else if (in_range(b, 0xC0, 0xC1)) kind = OVERLONG;
            else if (b >= 0xF5) kind = HEADER_BITS;
            else {
                int len = b <= 0xDF ? 2 : b <= 0xEF ? 3 : 4, k, conts = 1;
                if (p + len > n) conts = 0;
                for (k = 1; k < len && conts; k++) conts = in_range(s[p + k], 0x80, 0xBF);
                if (!conts) kind = TOO_SHORT;
                else if (b == 0xE0 || b == 0xF0) kind = OVERLONG;
                else if (b == 0xED) kind = SURROGATE;
                else kind = TOO_LARGE; /* F4 with second byte above 8F */
            }
            r->status = kind;
            r->in_offset = (uint64_t)p;
            r->out_len = o;
            return;
        }
    }
    r->status = OK;
    r->in_offset = (uint64_t)n;
    r->out_len = o;
}

static void match16(const uint16_t *u, int n, res_t *r)
{
    int p = 0;
    uint64_t o = 0;
    while (p < n) {
        int w = u[p];
        if (in_range(w, 0xD800, 0xDBFF)) {
            if (p + 1 < n && in_range(u[p + 1], 0xDC00, 0xDFFF)) { o += 4; p += 2; continue; }
            r->status = LONE_HIGH; r->in_offset = p; r->out_len = o; return;
        }
        if (in_range(w, 0xDC00, 0xDFFF)) {
            r->status = LONE_LOW; r->in_offset = p; r->out_len = o; return;
        }
        o += w < 0x80 ? 1 : w < 0x800 ? 2 : 3;
        p += 1;
    }
    r->status = OK; r->in_offset = n; r->out_len = o;
}

typedef struct { int mode, tid, nthreads; uint64_t bad, checked; char first[160]; } job_t;

static void compare(job_t *j, const res_t *a, const res_t *b, const char *what)
{
    j->checked++;
    if (a->status != b->status || a->in_offset != b->in_offset || a->out_len != b->out_len) {
        if (!j->bad)
            snprintf(j->first, sizeof j->first,
                     "%s: oracle (%d,%llu,%llu) matcher (%d,%llu,%llu)", what,
                     a->status, (unsigned long long)a->in_offset, (unsigned long long)a->out_len,
                     b->status, (unsigned long long)b->in_offset, (unsigned long long)b->out_len);
        j->bad++;
    }
}

static void *run(void *arg)
{
    job_t *j = (job_t *)arg;
    uint8_t out[64];
    res_t a, b;
    char what[64];
    if (j->mode == 8) {
        uint8_t s[4];
        /* lengths 1-3: thread 0 only (16.8 M strings) */
        if (j->tid == 0) {
            for (int len = 1; len <= 3; len++) {
                uint32_t total = 1u << (8 * len);
                for (uint32_t v = 0; v < total; v++) {
                    for (int k = 0; k < len; k++) s[k] = (uint8_t)(v >> (8 * (len - 1 - k)));
                    oracle_utf8_to_utf16le(s, len, out, 32, &a);
                    match8(s, len, &b);
                    if (a.status != b.status || a.in_offset != b.in_offset || a.out_len != b.out_len) {
                        snprintf(what, sizeof what, "utf8 len %d %06x", len, v);
                        compare(j, &a, &b, what);
                    } else j->checked++;
                }
            }
        }
        /* length 4: lead bytes split over threads */
        for (uint32_t lead = (uint32_t)j->tid; lead < 256; lead += (uint32_t)j->nthreads) {
            s[0] = (uint8_t)lead;
            for (uint32_t rest = 0; rest < (1u << 24); rest++) {
                s[1] = (uint8_t)(rest >> 16); s[2] = (uint8_t)(rest >> 8); s[3] = (uint8_t)rest;
                oracle_utf8_to_utf16le(s, 4, out, 32, &a);
                match8(s, 4, &b);
                if (a.status != b.status || a.in_offset != b.in_offset || a.out_len != b.out_len) {
                    snprintf(what, sizeof what, "utf8 len 4 %02x%06x", lead, rest);
                    compare(j, &a, &b, what);
                } else j->checked++;
            }
        }
    } else {
        uint16_t u[2];
        uint8_t bytes[4];
        if (j->tid == 0) {
            for (uint32_t v = 0; v < 65536; v++) {
                u[0] = (uint16_t)v; bytes[0] = (uint8_t)v; bytes[1] = (uint8_t)(v >> 8);
                oracle_utf16le_to_utf8(bytes, 1, out, 64, &a);
                match16(u, 1, &b);
                snprintf(what, sizeof what, "utf16 len 1 %04x", v);
                compare(j, &a, &b, what);
            }
        }
        for (uint32_t first = (uint32_t)j->tid; first < 65536; first += (uint32_t)j->nthreads) {
            u[0] = (uint16_t)first; bytes[0] = (uint8_t)first; bytes[1] = (uint8_t)(first >> 8);
            for (uint32_t second = 0; second < 65536; second++) {
                u[1] = (uint16_t)second; bytes[2] = (uint8_t)second; bytes[3] = (uint8_t)(second >> 8);
                oracle_utf16le_to_utf8(bytes, 2, out, 64, &a);
                match16(u, 2, &b);
                if (a.status != b.status || a.in_offset != b.in_offset || a.out_len != b.out_len) {
                    snprintf(what, sizeof what, "utf16 len 2 %04x %04x", first, second);
                    compare(j, &a, &b, what);
                } else j->checked++;
            }
        }
    }
    return NULL;
}

int main(int argc, char **argv)
{
    int mode = (argc > 1 && strcmp(argv[1], "utf16") == 0) ? 16 : 8;
    int nt = argc > 2 ? atoi(argv[2]) : 4;
    if (nt < 1) nt = 1;
    if (nt > 256) nt = 256;
    pthread_t th[256];
    job_t jobs[256];
    memset(jobs, 0, sizeof jobs);
    for (int t = 0; t < nt; t++) {
        jobs[t].mode = mode; jobs[t].tid = t; jobs[t].nthreads = nt;
        pthread_create(&th[t], NULL, run, &jobs[t]);
    }
    uint64_t bad = 0, checked = 0;
    const char *first = NULL;
    for (int t = 0; t < nt; t++) {
        pthread_join(th[t], NULL);
        bad += jobs[t].bad;
        checked += jobs[t].checked;
        if (jobs[t].bad && !first) first = jobs[t].first;
    }
    printf("checked %llu mismatches %llu\n", (unsigned long long)checked, (unsigned long long)bad);
    if (first) printf("first: %s\n", first);
    return bad ? 1 : 0;
}
