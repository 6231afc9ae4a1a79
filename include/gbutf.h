/*
 * gbutf: validating UTF-8 <-> UTF-16LE transcoding on NVIDIA GB300 (sm_103a).
 *
 * A C ABI over hand-written CUDA kernels. The operations are those of
 * Clausecker & Lemire, "Transcoding Unicode Characters with AVX-512
 * Instructions" (arXiv 2212.05098): transcode a buffer of UTF-8 into UTF-16LE
 * (Sec. 6) or UTF-16LE into UTF-8 (Sec. 7), validating the input throughout
 * (Sec. 6.4, Sec. 7.4); on an encoding error, transcode the valid prefix and
 * report the number of input units before the first error (Sec. 6.4,
 * Sec. 7.5). The length-only calls run the same validation and count the
 * output without writing it.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units. UTF-8 is counted in bytes, UTF-16LE in 16-bit words (little endian,
 *   no byte-order mark generated, checked or stripped; Sec. 2.1).
 * - Validity. UTF-8 follows Table 1 and rules 1-6 of Sec. 6.4 (shortest form,
 *   no surrogates, nothing above U+10FFFF, C0/C1/F5-FF never valid). UTF-16LE
 *   requires every high surrogate to be followed by a low surrogate and every
 *   low surrogate to be preceded by a high one. Noncharacters (U+FFFE ...) and
 *   U+0000 are valid.
 * - Result (gbu_result):
 *     GBU_OK                in_offset = n, out_len = output units written.
 *     encoding error kind   in_offset = index of the first invalid input unit
 *                           (the lead byte of a malformed or truncated
 *                           sequence, a stray continuation byte, or the
 *                           unpaired surrogate); out_len = output units of
 *                           the valid prefix [0, in_offset). An encoding error
 *                           takes precedence over a too-small output.
 *     GBU_OUTPUT_TOO_SMALL  the input is valid but needs out_len > cap units;
 *                           in_offset = n.
 *     GBU_INVALID_ARG, GBU_DEVICE_ERROR, GBU_DEVICE_TIMEOUT: in_offset = 0,
 *                           out_len = 0, output contents unspecified.
 *   Output: units [0, min(out_len, cap)) are written exactly; units from
 *   out_len to cap are unspecified; nothing at or beyond cap is written.
 *   Error kinds are this library's convention (the paper defines only the
 *   error position): byte class first, then structure, then value.
 * - Memory. d_in / d_out are device pointers owned by the caller (any
 *   allocation the current CUDA context can read / write; e.g. torch
 *   tensors). UTF-8 buffers may have any alignment; UTF-16 buffers must be
 *   2-byte aligned (else GBU_INVALID_ARG). Input and output must not overlap.
 *   The kernels read whole aligned 16-byte blocks that overlap the input
 *   range (never a block disjoint from it).
 * - Worst-case capacity: UTF-8 -> UTF-16 needs at most n_bytes units;
 *   UTF-16 -> UTF-8 at most 3 * n_units bytes.
 * - Size limit: n < 2^39 input units per call (else GBU_INVALID_ARG).
 * - Streams. `stream` is a cudaStream_t (0 = legacy default stream). The
 *   synchronous calls enqueue on it and wait for that stream only.
 * - Contexts. A gbu_ctx owns device scratch memory (scan state, error word,
 *   result slot). Calls on one context must not overlap on the GPU: use one
 *   context per stream (or per concurrently running call). Contexts are not
 *   thread-safe.
 * - No exceptions cross this interface; CUDA errors become GBU_DEVICE_ERROR.
 */
#ifndef GBUTF_H
#define GBUTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gbu_status {
    GBU_OK = 0,
    GBU_HEADER_BITS = 1,          /* byte F5-FF (UTF-8 rule 1)                      */
    GBU_TOO_SHORT = 2,            /* lead byte without all its continuation bytes    */
    GBU_TOO_LONG = 3,             /* continuation byte with no lead (rule 3)         */
    GBU_OVERLONG = 4,             /* C0/C1, or a 3/4-byte form of a smaller value    */
    GBU_TOO_LARGE = 5,            /* value above U+10FFFF (rule 5)                   */
    GBU_SURROGATE = 6,            /* UTF-8 encoding of U+D800-U+DFFF (rule 6)        */
    GBU_LONE_HIGH_SURROGATE = 7,  /* UTF-16 high surrogate not followed by a low     */
    GBU_LONE_LOW_SURROGATE = 8,   /* UTF-16 low surrogate not preceded by a high     */
    GBU_OUTPUT_TOO_SMALL = 16,
    GBU_INVALID_ARG = 17,
    GBU_DEVICE_ERROR = 18,
    GBU_DEVICE_TIMEOUT = 19       /* a bounded wait inside a kernel gave up          */
} gbu_status;

typedef struct gbu_result {
    int32_t status;      /* gbu_status                                          */
    uint32_t reserved;   /* zero                                                */
    uint64_t in_offset;  /* see "Result" above                                  */
    uint64_t out_len;    /* output units (UTF-16: words; UTF-8: bytes)          */
} gbu_result;

typedef struct gbu_ctx gbu_ctx;

/* Create a context on CUDA device `device` (that device becomes current for
 * the calling thread). Returns NULL on failure. Free with gbu_destroy. */
gbu_ctx *gbu_create(int device);
void gbu_destroy(gbu_ctx *ctx);

/* Pre-size the context's scratch memory for inputs of up to `max_input_bytes`
 * bytes, so that later calls allocate nothing. Scratch grows on demand
 * otherwise (a growth synchronises the device). Returns a gbu_status. */
int32_t gbu_reserve(gbu_ctx *ctx, uint64_t max_input_bytes);

/* UTF-8 -> UTF-16LE (Sec. 6). d_in: n_bytes bytes; d_out: cap_units words. */
gbu_result gbu_utf8_to_utf16le(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                               uint16_t *d_out, uint64_t cap_units, void *stream);

/* UTF-16LE -> UTF-8 (Sec. 7). d_in: n_units words; d_out: cap_bytes bytes. */
gbu_result gbu_utf16le_to_utf8(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                               uint8_t *d_out, uint64_t cap_bytes, void *stream);

/* Validating length-only calls: out_len = UTF-16 words (resp. UTF-8 bytes) of
 * the whole input, or of its valid prefix on an encoding error. */
gbu_result gbu_utf16_length_from_utf8(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                      void *stream);
gbu_result gbu_utf8_length_from_utf16le(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                        void *stream);

/* UTF-16BE forms (the byte order the paper's Sec. 2.1 mentions beside
 * UTF-16LE): identical to the UTF-16LE calls except that every UTF-16 word
 * is read or written with its high byte first. d_in / d_out as for the
 * UTF-16LE calls (2-byte aligned, units of words). */
gbu_result gbu_utf8_to_utf16be(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                               uint16_t *d_out, uint64_t cap_units, void *stream);
gbu_result gbu_utf16be_to_utf8(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                               uint8_t *d_out, uint64_t cap_bytes, void *stream);
gbu_result gbu_utf8_length_from_utf16be(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                        void *stream);
gbu_result gbu_validate_utf16be(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                void *stream);
int32_t gbu_utf8_to_utf16be_async(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                  uint16_t *d_out, uint64_t cap_units, gbu_result *result,
                                  void *stream);
int32_t gbu_utf16be_to_utf8_async(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                  uint8_t *d_out, uint64_t cap_bytes, gbu_result *result,
                                  void *stream);

/* UTF-32LE forms (Sec. 2: a UTF-32 unit is the code point itself, little-
 * endian 32-bit words; UTF-8 bytes per Fig. 1(a)). Synchronous; results as
 * for the UTF-16 calls, with units of 32-bit words on the UTF-32 side.
 *
 * gbu_utf8_to_utf32le: d_in any alignment; d_out 4-byte aligned, cap_units
 *   32-bit units (n_bytes is never too small). The UTF-8 is validated by the
 *   rules of Sec. 6.4 exactly as by gbu_utf8_to_utf16le (same status and
 *   in_offset); out_len counts code points.
 * gbu_utf32le_to_utf8: d_in 4-byte aligned, n_units 32-bit units; d_out any
 *   alignment, cap_bytes bytes (4 * n_units is never too small). A unit above
 *   U+10FFFF is GBU_TOO_LARGE and one in D800-DFFF is GBU_SURROGATE, at its
 *   index (the library's convention; the paper defines no UTF-32 errors).
 * Length-only and validation calls as for UTF-16. A misaligned pointer is
 * GBU_INVALID_ARG. Each call runs short launches on `stream` (the UTF-8 side
 * first runs the UTF-8 validation) and waits for them; workspace is the
 * context's. */
gbu_result gbu_utf8_to_utf32le(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                               uint32_t *d_out, uint64_t cap_units, void *stream);
gbu_result gbu_utf32le_to_utf8(gbu_ctx *ctx, const uint32_t *d_in, uint64_t n_units,
                               uint8_t *d_out, uint64_t cap_bytes, void *stream);
gbu_result gbu_utf32_length_from_utf8(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                      void *stream);
gbu_result gbu_utf8_length_from_utf32le(gbu_ctx *ctx, const uint32_t *d_in, uint64_t n_units,
                                        void *stream);
gbu_result gbu_validate_utf32le(gbu_ctx *ctx, const uint32_t *d_in, uint64_t n_units,
                                void *stream);

/* Validation only (the paper's validation, Sec. 6.4 and 7.4, without the
 * transcoding): status and in_offset as for the transcoding calls (the
 * first invalid unit), out_len always 0. No output offsets are computed, so
 * the chunks' look-back is skipped. */
gbu_result gbu_validate_utf8(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes, void *stream);
gbu_result gbu_validate_utf16le(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                void *stream);

/* Asynchronous forms: enqueue the work on `stream` and return at once. The
 * gbu_result is stored to `result` (device memory, or pinned host memory
 * mapped into the device's address space) when the stream reaches the end of
 * the work. Return value: GBU_OK if enqueued, else GBU_INVALID_ARG /
 * GBU_DEVICE_ERROR (nothing enqueued, `result` untouched). */
int32_t gbu_utf8_to_utf16le_async(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                  uint16_t *d_out, uint64_t cap_units,
                                  gbu_result *result, void *stream);
int32_t gbu_utf16le_to_utf8_async(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                  uint8_t *d_out, uint64_t cap_bytes,
                                  gbu_result *result, void *stream);
int32_t gbu_utf16_length_from_utf8_async(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                         gbu_result *result, void *stream);
int32_t gbu_utf8_length_from_utf16le_async(gbu_ctx *ctx, const uint16_t *d_in,
                                           uint64_t n_units, gbu_result *result,
                                           void *stream);
int32_t gbu_validate_utf8_async(gbu_ctx *ctx, const uint8_t *d_in, uint64_t n_bytes,
                                gbu_result *result, void *stream);
int32_t gbu_validate_utf16le_async(gbu_ctx *ctx, const uint16_t *d_in, uint64_t n_units,
                                   gbu_result *result, void *stream);

/* Host-buffer forms: h_in / h_out are host memory (pinned memory gives the
 * fastest copies). The call copies the input to device scratch owned by the
 * context, transcodes it there, and copies min(out_len, cap) output units
 * back into h_out, all on `stream`, and returns when done. */
gbu_result gbu_utf8_to_utf16le_host(gbu_ctx *ctx, const uint8_t *h_in, uint64_t n_bytes,
                                    uint16_t *h_out, uint64_t cap_units, void *stream);
gbu_result gbu_utf16le_to_utf8_host(gbu_ctx *ctx, const uint16_t *h_in, uint64_t n_units,
                                    uint8_t *h_out, uint64_t cap_bytes, void *stream);

/* ---- Batches: many independent inputs in one launch of the work ------------
 *
 * The paper transcodes one buffer per call; a batch runs many such calls (any
 * mix of directions and of transcoding / length-only) together: the chunks of
 * all inputs are numbered consecutively (grouped by operation, the items with
 * the most chunks first within a group) and handed out in order to ONE
 * launch of the persistent kernel; every input keeps its own prefix scan,
 * first error and result, so each result equals that of the single-buffer
 * call on the same input. A batch of at least 512 MiB of input instead runs
 * its one-chunk items in a kernel of one CTA per item and the rest as one
 * persistent launch per input encoding (up to three launches, in order on
 * the stream; faster for large batches, more latency for small ones). */
typedef enum gbu_op {
    GBU_OP_UTF8_TO_UTF16LE = 0,           /* as gbu_utf8_to_utf16le            */
    GBU_OP_UTF16LE_TO_UTF8 = 1,           /* as gbu_utf16le_to_utf8            */
    GBU_OP_UTF16_LENGTH_FROM_UTF8 = 2,    /* as gbu_utf16_length_from_utf8     */
    GBU_OP_UTF8_LENGTH_FROM_UTF16LE = 3,  /* as gbu_utf8_length_from_utf16le   */
    GBU_OP_UTF8_TO_UTF16BE = 4,           /* as gbu_utf8_to_utf16be            */
    GBU_OP_UTF16BE_TO_UTF8 = 5,           /* as gbu_utf16be_to_utf8            */
    GBU_OP_UTF8_LENGTH_FROM_UTF16BE = 6   /* as gbu_utf8_length_from_utf16be   */
} gbu_op;

typedef struct gbu_batch_item {
    const void *in;      /* device pointer: UTF-8 bytes or UTF-16LE words (2-byte aligned) */
    uint64_t n;          /* input units                                                  */
    void *out;           /* device pointer, or NULL for the length-only ops              */
    uint64_t cap;        /* output capacity in units (ignored for length-only ops)       */
    int32_t op;          /* gbu_op                                                        */
    uint32_t reserved;   /* zero                                                          */
} gbu_batch_item;

/* Plan a batch on the context: validate the `count` host-side items, lay out
 * their chunks and upload the plan to device memory owned by the context
 * (allocated or grown here; returns after the upload). Results of the batch
 * go to `results[i]` (device memory, or pinned host memory mapped into the
 * device's address space), one gbu_result per item, with the semantics of the
 * corresponding single-buffer call. A plan stays valid until the next plan on
 * the context and may be launched any number of times. Returns GBU_OK,
 * GBU_INVALID_ARG (bad item: index not reported) or GBU_DEVICE_ERROR. */
int32_t gbu_batch_plan(gbu_ctx *ctx, const gbu_batch_item *items, uint32_t count,
                       gbu_result *results, void *stream);

/* Enqueue the planned batch on `stream` (one launch, or up to three for a
 * batch of 512 MiB or more; no host work, no allocation; it may be captured
 * into a CUDA graph by the caller). Results are stored when the stream
 * reaches the end of the work. */
int32_t gbu_batch_launch(gbu_ctx *ctx, void *stream);

/* Same, through a CUDA graph the context captures once per plan and replays
 * on `stream` (lowest launch overhead for repeated batches). */
int32_t gbu_batch_launch_graph(gbu_ctx *ctx, void *stream);

/* Launch parameters of a context (a tuning, not part of the paper's method:
 * results never depend on them). look_width: status words each lane of the
 * look-back warp reads per round (1, 2, 4, 8 or 16; the 32 * look_width nearest
 * predecessors per round). ctas_per_sm: resident CTAs per SM of the
 * persistent grid (0: as many as fit, 1..that maximum otherwise).
 * small_chunks: a single-buffer call whose input spans at most this many
 * chunks (counted from the 16-byte boundary at or before the input) runs as
 * one thread-block cluster with one CTA per chunk instead of the persistent
 * grid: no scratch, no counters, one launch (0: never; at most
 * GBU_SMALL_MAX_CHUNKS). Batches always use the persistent grid.
 * chunk_bytes, compute_threads: the kernel shape, one of those that
 * gbu_tune_shapes lists (input bytes per chunk, i.e. UTF-8 bytes or twice
 * the UTF-16 words, and compute threads per CTA); both 0: single-buffer calls
 * pick the shape from the input's size and batches use the default shape
 * (12288 bytes, 256 threads). A planned batch is counted again for a new
 * shape at its next launch. */
#define GBU_SMALL_MAX_CHUNKS 8
typedef struct gbu_tune {
    int32_t look_width;
    int32_t ctas_per_sm;
    int32_t small_chunks;
    int32_t chunk_bytes;
    int32_t compute_threads;
} gbu_tune;

/* Read / set the context's launch parameters (default {1, 0, 8, 0, 0}). Setting them
 * drops the context's captured batch graph. GBU_INVALID_ARG for values
 * outside the ranges above. */
int32_t gbu_get_tune(gbu_ctx *ctx, gbu_tune *tune);
int32_t gbu_set_tune(gbu_ctx *ctx, const gbu_tune *tune);

/* The compiled kernel shapes: writes up to `max_shapes` of them to `shapes`
 * (chunk_bytes and compute_threads set; the other fields at their defaults)
 * and returns how many there are (GBU_INVALID_ARG, a negative count, for bad
 * arguments). The first is the default shape. */
int32_t gbu_tune_shapes(gbu_tune *shapes, int32_t max_shapes);

/* The launch parameters a single-buffer call on `ctx` with `input_bytes`
 * bytes of input uses (the kernel shape filled in even when the context
 * picks it by size: up to 1 MiB 8192 x 256, above 12288 x 256). Such a call
 * runs as one cluster launch when its input spans at most small_chunks
 * chunks of chunk_bytes (counted from the 16-byte boundary at or before it).
 * Returns GBU_OK or GBU_INVALID_ARG. */
int32_t gbu_call_shape(gbu_ctx *ctx, uint64_t input_bytes, gbu_tune *tune);

/* Bounded waits. Every wait inside the kernels (for a TMA copy, for a
 * predecessor chunk's prefix, for another warp of the CTA) gives up after
 * `ns` nanoseconds of GPU global time (0 restores the default, 1 s). A wait
 * that gives up makes every result of that launch GBU_DEVICE_TIMEOUT (or
 * GBU_DEVICE_ERROR when chunks were left unprocessed); the kernel returns,
 * the CUDA context stays usable and the next call on the context starts from
 * clean scan state. Not part of the paper's method: failure detection of the
 * single-pass scan. Returns GBU_OK or GBU_INVALID_ARG (ns above 60 s). Drops
 * the context's captured batch graph. */
int32_t gbu_set_wait_limit(gbu_ctx *ctx, uint64_t ns);

/* Failure-detection test hook (not part of the paper's method). The next
 * single-buffer launch on this context hands out its chunks starting at chunk
 * `first_chunk` instead of 0, so chunks 0 .. first_chunk - 1 are never
 * processed: the look-back of the chunk after them waits for their prefix
 * until the wait limit runs out, and that launch reports GBU_DEVICE_TIMEOUT
 * (or GBU_DEVICE_ERROR if no chunk was processed at all). Nothing faults and
 * no wait is unbounded. One-shot; the chunk counter is written by a copy on
 * the call's stream. Returns GBU_OK or GBU_INVALID_ARG. */
int32_t gbu_test_skip_chunks(gbu_ctx *ctx, uint32_t first_chunk);

/* Autotune the planned batch: time one warm-up and three launches of it on
 * `stream` for every kernel shape (the batch counted again for each), every
 * look_width and every ctas_per_sm the shape fits, keep the combination with
 * the lowest median time on the context (small_chunks unchanged) and store it
 * in *chosen (may be NULL). The batch's outputs and results are written by
 * every timed launch (the same values each time). If `cache_path` is not
 * NULL, a text file of lines "<key> <look_width> <ctas_per_sm> <chunk_bytes>
 * <compute_threads> <ms>" is consulted first (key: device name, SM count, and
 * the batch's item count and input bytes in powers of two and UTF-16 /
 * transcoding shares in tenths) and the new choice is appended to it; a
 * cached key skips the timing. Blocks until done. Returns GBU_OK,
 * GBU_INVALID_ARG or GBU_DEVICE_ERROR (a failing launch). */
int32_t gbu_batch_autotune(gbu_ctx *ctx, void *stream, const char *cache_path, gbu_tune *chosen);

/* ---- Serving: requests as they arrive, continuous batching ------------------
 *
 * Not a construct of the paper (which transcodes one buffer per call): a
 * server that takes transcode requests of any size and direction as they
 * arrive. A dispatcher thread keeps up to `slots` batches in flight on the
 * GPU, each on its own stream and context. Whenever a slot is free it admits
 * queued requests in arrival order while their bytes fit into a device memory
 * pool of `pool_bytes` (each request holds a block for a copy of its input and
 * its worst-case output until it completes), copies their inputs into the
 * pool and runs them as one batch (see gbu_batch_plan). Requests that arrive
 * while batches run are admitted as soon as a slot and pool space free up, so
 * their work overlaps with the batches in flight. Each request's result is
 * that of the single-buffer call on the same input (gbu_result semantics).
 * The library owns the pool, streams and thread; the caller owns request
 * inputs (device memory, read during the request's batch) and the optional
 * output destinations. */
typedef struct gbu_server gbu_server;

typedef struct gbu_request {
    int32_t op;                   /* gbu_op                                                    */
    uint32_t reserved;            /* zero                                                      */
    const void *in;               /* device pointer: UTF-8 bytes or UTF-16LE words (2-aligned) */
    uint64_t n;                   /* input units                                               */
    void *out_copy;               /* device pointer receiving the output, or NULL (discarded)  */
    uint64_t out_copy_cap_bytes;  /* bytes available at out_copy (the worst-case output,
                                     2n for UTF-8 -> UTF-16LE and 3n for UTF-16LE -> UTF-8,
                                     is copied when it fits; bytes past out_len unspecified)  */
    uint64_t tag;                 /* caller's identifier, returned in the completion           */
} gbu_request;

typedef struct gbu_completion {
    uint64_t tag;
    gbu_result result;
    double t_submit, t_admit, t_launch, t_done;   /* seconds (server clock, or replay start) */
    uint32_t batch;                               /* batch number                             */
    uint32_t batch_items;                         /* requests in that batch                   */
} gbu_completion;

typedef struct gbu_server_stats_t {
    uint64_t submitted, completed, batches, pool_bytes, pool_high_water;
} gbu_server_stats_t;

/* Create a server on `device`: a pool of pool_bytes (>= 1 MiB), 1..16 slots,
 * at most max_batch_items requests per batch. NULL on failure. */
gbu_server *gbu_server_create(int device, uint64_t pool_bytes, uint32_t slots,
                              uint32_t max_batch_items);
/* Stop the dispatcher (queued requests are dropped) and free everything. */
void gbu_server_destroy(gbu_server *srv);
/* Queue one request (copied). GBU_INVALID_ARG: bad op, null or misaligned
 * input, or a request whose block can never fit into the pool. */
int32_t gbu_server_submit(gbu_server *srv, const gbu_request *req);
/* Move up to `max` completions (in completion order) into `out`; returns how
 * many. */
uint32_t gbu_server_poll(gbu_server *srv, gbu_completion *out, uint32_t max);
/* Wait until every submitted request has completed (GBU_DEVICE_TIMEOUT after
 * timeout_s seconds). */
int32_t gbu_server_wait_idle(gbu_server *srv, double timeout_s);
/* Submit reqs[i] at t_arrival[i] seconds after the call (non-decreasing
 * times, from this thread), collect every completion and return them in
 * request order in out[i] (times relative to the call). Must not be mixed
 * with concurrent gbu_server_submit / gbu_server_poll calls. Returns GBU_OK,
 * GBU_INVALID_ARG (bad request; nothing submitted) or GBU_DEVICE_TIMEOUT (not
 * all completed within timeout_s after the last arrival). */
int32_t gbu_server_replay(gbu_server *srv, const gbu_request *reqs, const double *t_arrival,
                          uint32_t count, gbu_completion *out, double timeout_s);
/* Counters of the server. */
int32_t gbu_server_stats(gbu_server *srv, gbu_server_stats_t *stats);

/* No-allocation form of gbu_utf8_to_utf16le. The paper has no counterpart to
 * this call: it is for callers that may not allocate device memory (another
 * component owns the device's memory, or an allocation's implicit device
 * synchronisation is not acceptable on their path), whereas gbu_create /
 * gbu_reserve allocate scratch. It takes no context: the kernel's scratch is
 * one fixed-size device array inside this library, held by every GPU that
 * loads the library until the process exits, so inputs are limited to
 * GBU_NOALLOC_MAX_BYTES bytes (larger inputs: GBU_INVALID_ARG, nothing run).
 * The first call on a device looks up the array's device address (the array
 * starts zeroed when the library's device code loads); make that first call
 * before any stream capture. The call works on the current device: `stream`
 * must belong to it (a stream of another device gives GBU_INVALID_ARG). All
 * calls share the array: calls that overlap on the GPU (other streams, other
 * host threads on the same device) race and must not be issued. Same
 * arguments, result and output rules as gbu_utf8_to_utf16le; calls no
 * cudaMalloc / cudaFree; waits for `stream`. Inputs of at most
 * GBU_SMALL_MAX_CHUNKS chunks take the one-launch path, which uses the array
 * only for the result. */
#define GBU_NOALLOC_MAX_BYTES (64ull << 20)
gbu_result gbu_utf8_to_utf16le_noalloc(const uint8_t *d_in, uint64_t n_bytes,
                                       uint16_t *d_out, uint64_t cap_units, void *stream);

/* Name of a gbu_status value ("GBU_OK", ...); "GBU_UNKNOWN" otherwise. */
const char *gbu_status_name(int32_t status);

/* Number of kernels this library has launched in the calling process
 * (diagnostics; counts every launch of every entry point). */
uint64_t gbu_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GBUTF_H */
