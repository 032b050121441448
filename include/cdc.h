/*
 * cdc.h -- C ABI of the GB300 hashless content-defined chunking library.
 *
 * The library finds chunk boundaries with the hashless algorithms RAM,
 * AE (AE-Max and AE-Min) and MAXP of arxiv 2508.05797 ("VectorCDC"):
 *   RAM  -- Section 2.1 (RAM paragraph), Section 3.3: the maximum of the
 *           w-byte window at the chunk start, then the first later byte that
 *           is >= that maximum ends the chunk (the byte is inside the chunk).
 *   AE   -- Section 2.1 (AE paragraph), Section 3.3: a target is a byte
 *           beyond (greater for AE-Max, lower for AE-Min) all bytes before it
 *           in the chunk; once the w bytes after a target hold nothing beyond
 *           it, the chunk ends right after those w bytes.
 *   MAXP -- Section 2.1 (MAXP paragraph), Section 3.3: a target is strictly
 *           greater than every byte within distance w on both sides (both
 *           windows inside the data); the chunk ends right after the first
 *           target that gives at least `min` bytes.
 * min / max bound the chunk size as in Section 2.1 (hash-based paragraph):
 * no cut before min bytes, a forced cut at max bytes; the last chunk ends at
 * the end of the data and may be shorter than min.
 *
 * Output: the increasing list of chunk ends b_1 < ... < b_k = len (offsets
 * from the start of the data), so chunk i is [b_{i-1}, b_i) with b_0 = 0.
 * The boundaries equal, bit for bit, those of the plain sequential algorithm
 * (the paper's own criterion, Section 5.2: accelerated and native chunks
 * are identical).
 *
 * Conventions for every entry point:
 *   - Data and output buffers are caller-owned DEVICE memory unless the name
 *     says host. Any alignment is accepted.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued on it; entry points that return a count synchronise it.
 *   - A handle owns device workspace and is not thread-safe: use one handle
 *     per host thread (or serialise calls). Workspace grows on demand
 *     outside the hot path; while a stream is being captured into a CUDA
 *     graph the workspace must already be large enough (else
 *     CDC_ERR_NOMEM).
 *   - Errors are returned, never printed; cdc_status_string() names them.
 *   - Parameter rules (CDC_ERR_INVALID otherwise): w >= 1, 1 <= min <= max,
 *     and for RAM / AE w < max. A NULL data pointer with len > 0, a NULL
 *     output pointer, an unknown algorithm or an unknown option is invalid.
 */
#ifndef CDC_H
#define CDC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CDC_API __attribute__((visibility("default")))
#else
#define CDC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDC_RAM = 0,     /* Rapid Asymmetric Maximum */
    CDC_AE = 1,      /* Asymmetric Extremum, maxima (AE-Max) */
    CDC_MAXP = 2,    /* local maximum over +-w */
    CDC_AE_MIN = 3   /* Asymmetric Extremum, minima (AE-Min) */
} cdc_alg;

typedef struct {
    uint32_t w;      /* window size in bytes */
    uint32_t min;    /* minimum chunk size in bytes */
    uint32_t max;    /* maximum chunk size in bytes */
} cdc_params;

typedef enum {
    CDC_OK = 0,
    CDC_ERR_INVALID = 1,   /* bad argument */
    CDC_ERR_CAPACITY = 2,  /* output too small; the count holds the size needed */
    CDC_ERR_CUDA = 3,      /* a CUDA call failed (no device, launch error, ...) */
    CDC_ERR_TIMEOUT = 4,   /* a bounded device-side wait ran out */
    CDC_ERR_NOMEM = 5,     /* workspace could not be allocated */
    CDC_ERR_INTERNAL = 6   /* a device-side consistency check failed */
} cdc_status;

typedef struct cdc_handle_s* cdc_handle;
typedef void* cdc_stream;  /* a cudaStream_t */

/* Create a handle on CUDA device `device` (which becomes current for the
 * calling thread). *out receives the handle; nothing is allocated on the
 * device until first use. */
CDC_API cdc_status cdc_create(cdc_handle* out, int device);

/* Release the handle and its device workspace. NULL is accepted. */
CDC_API cdc_status cdc_destroy(cdc_handle h);

/* Chunk one device buffer `data` of `len` bytes with algorithm `alg`.
 * out_bounds: device array receiving the chunk ends (uint64, offsets from
 * data). *n: on entry its capacity in elements, on return the number of
 * boundaries (also when CDC_ERR_CAPACITY is returned, in which case the
 * contents of out_bounds are unspecified). len == 0 gives *n = 0.
 * Synchronises `stream`. */
CDC_API cdc_status cdc_chunk(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                     uint64_t* out_bounds, size_t* n, cdc_stream stream);

/* As cdc_chunk, without synchronising: the boundary count (uint64) is
 * written to the device word *d_count when the work completes. A count
 * above `capacity` means the output was too small (contents unspecified);
 * device-side errors are reported by the next cdc_chunk / cdc_sync_status
 * call on the handle. Capturable into a CUDA graph once the workspace is
 * sized (call cdc_reserve first). */
CDC_API cdc_status cdc_chunk_async(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data,
                           size_t len, uint64_t* out_bounds, size_t capacity,
                           uint64_t* d_count, cdc_stream stream);

/* Chunk many files packed in one device arena in a single persistent
 * launch. File f is data[file_off[f], file_off[f+1]) and is chunked from its
 * own start. data_len: bytes of the arena (>= file_off[n_files]).
 * d_file_off: device array of n_files + 1 non-decreasing offsets.
 * d_bounds: device array receiving every file's boundaries, file after file,
 * each relative to its file's start. d_bounds_index: device array of
 * n_files + 1 entries; file f's boundaries are
 * d_bounds[d_bounds_index[f] .. d_bounds_index[f+1]). capacity: elements of
 * d_bounds. total: if not NULL, receives the total count and the stream is
 * synchronised; if NULL the call is asynchronous (the total is then
 * d_bounds_index[n_files]). */
CDC_API cdc_status cdc_chunk_batch(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data,
                           size_t data_len, const uint64_t* d_file_off, size_t n_files,
                           uint64_t* d_bounds, uint64_t* d_bounds_index, size_t capacity,
                           size_t* total, cdc_stream stream);

/* End-to-end call on HOST buffers: copies `host_data` to the device, chunks
 * it and copies the boundaries back into host_bounds (capacity *n; *n
 * receives the count). Page-locked host memory gives the fastest copies.
 * Synchronises `stream`. */
CDC_API cdc_status cdc_chunk_host(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* host_data,
                          size_t len, uint64_t* host_bounds, size_t* n, cdc_stream stream);

/* Make sure the workspace fits `len` bytes of data in up to `n_files` files
 * for algorithm `alg` and parameters p (so that later calls allocate
 * nothing, e.g. before graph capture). */
CDC_API cdc_status cdc_reserve(cdc_handle h, cdc_alg alg, cdc_params p, size_t len, size_t n_files);

/* Wait for the work on `stream` and report device-side errors of the
 * asynchronous calls made on the handle since the last check. */
CDC_API cdc_status cdc_sync_status(cdc_handle h, cdc_stream stream);

/* Tuning and test options (value semantics per option). */
typedef enum {
    CDC_OPT_SEGMENT = 0,      /* bytes per speculative segment; 0 = automatic */
    CDC_OPT_SPAN = 1,         /* bytes over which a segment's 128 speculative
                                 chains start; 0 = automatic */
    CDC_OPT_TIMEOUT_MS = 2,   /* bound on any device-side wait (default 2000) */
    CDC_OPT_FORCE_BYTES = 3,  /* 1 = skip the block summaries and scan raw
                                 bytes in the chain stage (testing) */
    CDC_OPT_DEBUG_HOLD_ITEM = 4, /* testing only: the segment with this index
                                 never publishes its state, so its successors
                                 time out (-1 = off, the default) */
    CDC_OPT_PROFILE = 5,      /* 1 = record CUDA events around the stages of
                                 every call (up to 1024 calls) for
                                 cdc_profile_collect; setting it clears them */
    CDC_OPT_STATS = 6,        /* 1 = the chain stage counts its work (chain
                                 steps, stitch walks, uncovered entries, ...)
                                 for cdc_stats; costs atomics, testing only */
    CDC_OPT_WARP_CHAINS = 7,  /* speculative chains of a segment are stepped one
                                 per thread while more than this many are
                                 alive, then one per warp (all 32 lanes share
                                 each step); 1..128, 0 = automatic (96) */
    CDC_OPT_STARTS = 8,       /* distinct speculative starts per segment, spread
                                 over its first `span` bytes; 1..128, 0 =
                                 automatic (span / 128, within 16..128;
                                 16 for MAXP) */
    CDC_OPT_PIPELINE = 9,     /* chain stage of cdc_chunk / cdc_chunk_async /
                                 cdc_chunk_host: 0 = automatic (the candidate
                                 graph for inputs up to 512 MiB, 768 MiB for
                                 AE, where it applies: RAM and AE-Max with
                                 w >= 64 and min <= w + 1, MAXP with
                                 63 <= w <= 16384; else speculation),
                                 1 = speculative segments always,
                                 2 = the candidate graph wherever it applies
                                 (AE-Min included) */
    CDC_OPT_GRAPH_SEGMENT = 10, /* bytes per segment of the candidate graph
                                 (a multiple of 4096; raised to max if below);
                                 0 = automatic */
    CDC_OPT_GRAPH_SLOTS = 11  /* candidate slots per graph segment (1..4096,
                                 rounded up to a multiple of 16; candidates
                                 beyond them are stepped, slower but exact);
                                 0 = automatic (segment / 32) */
} cdc_option;

CDC_API cdc_status cdc_set_option(cdc_handle h, cdc_option opt, int64_t value);
CDC_API cdc_status cdc_get_option(cdc_handle h, cdc_option opt, int64_t* value);

/* Autotuner for the segment size, the warp-chain threshold and the number
 * of speculative starts: runs the chunk path on the caller's input for each
 * pair of a small grid (segment bytes: automatic, 128 KiB, 256 KiB, 384 KiB,
 * 512 KiB, 1 MiB; warp chains: 32, 64, 96; automatic starts), then for 32, 64 and 128
 * starts at the best pair, twice each, timed with CUDA events on `stream`, and
 * keeps the fastest setting on the handle (CDC_OPT_SEGMENT,
 * CDC_OPT_WARP_CHAINS, CDC_OPT_STARTS, the last readable with
 * cdc_get_option), reported in *seg_out, *warp_chains_out and *best_ms (each
 * may be NULL). Every setting gives the
 * same boundaries, so tuning never changes results. d_file_off / n_files /
 * d_bounds_index as for cdc_chunk_batch (d_file_off NULL: one stream of len
 * bytes); d_bounds (capacity entries) is overwritten. Not during stream
 * capture (CDC_ERR_INVALID); synchronises `stream`. On an error the options
 * are left as they were. The paper has no counterpart. */
CDC_API cdc_status cdc_autotune(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                const uint64_t* d_file_off, size_t n_files, uint64_t* d_bounds,
                                uint64_t* d_bounds_index, size_t capacity, int64_t* seg_out,
                                int64_t* warp_chains_out, float* best_ms, cdc_stream stream);

/* Device time in milliseconds of the two stages of the last call on the
 * handle (block summaries; chain), measured with CUDA events on the call's
 * stream. Synchronises on those events. Either pointer may be NULL. */
CDC_API cdc_status cdc_last_timing(cdc_handle h, float* summary_ms, float* chain_ms);

/* Totals over the calls recorded since profiling was switched on or last
 * collected: number of calls, device milliseconds of the summary stage, of
 * the chain stage, and of the speculation kernel alone (the first kernel of
 * the chain stage; part of chain_ms), and kernels launched. Synchronises on
 * the recorded events and clears them. Any output pointer may be NULL. */
CDC_API cdc_status cdc_profile_collect(cdc_handle h, int* calls, double* summary_ms, double* chain_ms,
                                       double* spec_ms, int64_t* launches);

/* Counters of the last call made with CDC_OPT_STATS on (up to n of them,
 * in this order): segments, single-thread chain steps, whole-warp chain steps
 * in speculation, merged chains, stitch walks, stitch steps, uncovered table
 * entries, segments whose position hash filled, fallback walks in the
 * resolution, output steps, empty segments, chains handed to whole warps,
 * then clock cycles summed over segments (set-up, speculation, merge
 * resolution, stitching), per-thread rounds, the cycles of the rounds and of
 * the one-warp-per-chain phase, stitch walks of more than 64 steps,
 * (steps << 32 | segment) of the longest one, the output kernel's passes over
 * step logs, records it replayed, its cycles and the part of them spent in
 * its own chain steps (25 counters). When the call took the candidate graph
 * (cdc_last_stage 2) the counters are the graph's instead: segments,
 * candidates, F evaluated by stepping, the local kernel's cycles summed over
 * segments (staging, F, pointer jumping), jumping rounds, the longest segment,
 * the stepped F's cycles and the longest one, the candidate kernel's cycles
 * summed over chunks (staging, listing blocks, testing their bytes, writing),
 * blocks listed, the longest segment of each local-kernel phase, (cycles << 24
 * | segment) of the longest local segment and the longest candidate-kernel
 * chunk (20 counters).
 * Synchronises `stream`. */
CDC_API cdc_status cdc_stats(cdc_handle h, uint64_t* out, int n, cdc_stream stream);

/* Number of kernels the last call launched. */
CDC_API cdc_status cdc_last_launches(cdc_handle h, int* launches);

/* Chain stage the last call on the handle used (CDC_OPT_PIPELINE 0 chooses
 * per call): 1 = speculative segments, 2 = the candidate graph, 0 before the
 * first call. Host-side bookkeeping only; no synchronisation. */
CDC_API cdc_status cdc_last_stage(cdc_handle h, int* stage);

/* ---- chunking without any allocation --------------------------------------
 *
 * The paper has no counterpart: it is a property of this library's interface,
 * not of the chunking method.
 *
 * cdc_chunk_static does what cdc_chunk does, on the CURRENT device, without a
 * handle and without allocating anything: no cudaMalloc / cudaFree, no
 * allocating library routine, no pinned host memory. Its scratch (block
 * summaries, per-segment speculation state, position hashes and step logs,
 * control block) is one fixed
 * array of CDC_STATIC_SCRATCH_BYTES in the library's device image, so it
 * serves inputs of at most CDC_STATIC_MAX_LEN bytes.
 *
 * For callers that cannot allocate: code running under a memory cap that is
 * already fully claimed (for instance by a caching allocator that owns the
 * device's free memory), latency-sensitive paths where cudaMalloc / cudaFree
 * would synchronise the device and stall other streams, and callers that
 * cannot keep a handle's lifetime (create / destroy) around a call.
 *
 * Arguments and results are those of cdc_chunk (`*n`: in = capacity of
 * out_bounds, out = number of boundaries; CDC_ERR_CAPACITY with `*n` = the
 * number needed). The call synchronises `stream`.
 *   - len > CDC_STATIC_MAX_LEN returns CDC_ERR_INVALID and enqueues nothing.
 *   - data and out_bounds must be memory of the current device (or managed
 *     memory); host memory, pinned or not, and another device's memory
 *     return CDC_ERR_INVALID and enqueue nothing.
 *   - The first call on a device looks up the scratch array's device address
 *     (the CUDA runtime may load the library's device code at that moment,
 *     which claims the CDC_STATIC_SCRATCH_BYTES of device memory) and clears
 *     the parts that must start at zero: the control block and the segments'
 *     ready flags. Make that first call at start-up, before memory is fully
 *     claimed and before any stream capture starts. Every call also clears
 *     the control block's error word before it launches.
 *   - The call cannot be captured into a CUDA graph: it reads the boundary
 *     count back to the host and synchronises `stream`.
 *   - The address is cached per device for the life of the process. A
 *     device reset (cudaDeviceReset) while the library is loaded is not
 *     supported: later calls would use the stale address.
 *   - The scratch is shared by every caller on a device: calls that overlap
 *     in time (several host threads, or several streams) race on it and give
 *     wrong results. Serialise them.
 */
#define CDC_STATIC_MAX_LEN ((size_t)16 << 20)
#define CDC_STATIC_SCRATCH_BYTES ((size_t)21677312)

CDC_API cdc_status cdc_chunk_static(cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                    uint64_t* out_bounds, size_t* n, cdc_stream stream);

/* ---- the two processing patterns as standalone device operations -----------
 *
 * Extreme Byte Search (Section 3.1) and Range Scan (Section 3.2) over many
 * byte ranges of one device buffer at once. d_ranges holds 2n offsets
 * (start, end) into data, each range [start, end) clipped to len; results
 * are offsets into data. Asynchronous on `stream`; no handle needed.
 */
typedef enum { CDC_EBS_MAX = 0, CDC_EBS_MIN = 1 } cdc_ebs_op;
typedef enum { CDC_RS_GT = 0, CDC_RS_LT = 1, CDC_RS_GEQ = 2, CDC_RS_LEQ = 3, CDC_RS_EQ = 4 } cdc_rs_cmp;

/* d_value[i] = the maximum (CDC_EBS_MAX) or minimum byte of range i and, if
 * d_pos is not NULL, d_pos[i] = the offset of its first occurrence. An empty
 * range gives 0 (max) or 255 (min) and its start. */
CDC_API cdc_status cdc_ebs(cdc_ebs_op op, const uint8_t* data, size_t len, const uint64_t* d_ranges, size_t n,
                           uint8_t* d_value, uint64_t* d_pos, cdc_stream stream);

/* d_pos[i] = the first offset p in range i with cmp(data[p], d_thresholds[i])
 * (GT: >, LT: <, GEQ: >=, LEQ: <=, EQ: ==), or the range's end if none. */
CDC_API cdc_status cdc_rs(cdc_rs_cmp cmp, const uint8_t* data, size_t len, const uint64_t* d_ranges,
                          const uint8_t* d_thresholds, size_t n, uint64_t* d_pos, cdc_stream stream);

/* Bytes read by each of the two processing patterns while the chunks of a
 * buffer are found, as Section 3.3 composes the algorithms (the paper plots
 * these shares per algorithm and dataset). d_bounds: the n boundaries
 * cdc_chunk wrote for `data` with the same alg and p. d_out (device, 2
 * uint64) receives the bytes read by Extreme Byte Searches, then by Range
 * Scans. RAM: per chunk one search over its w-byte window (the rest, for a
 * tail of at most w bytes) and one GEQ scan from max(s + w, s + min - 1) to
 * the cut. AE-Max / AE-Min: per target (a byte beyond every earlier byte of
 * the chunk) one search over the w bytes after it, clipped at the chunk's
 * last byte, and GT / LT scans from target to target. MAXP: from
 * p = max(s + min - 1, w), a search over the left window [p - w, p) gives its
 * maximum and the last position m holding it; a GT scan from p, stopping at
 * m + w (where m leaves the window) or at the first byte above that maximum,
 * reads the bytes up to the one it stops at; a byte it stops at costs one
 * search over its right window, which decides whether the chunk ends after it
 * or the scan resumes one byte later. AE with min > w + 1 (where the window
 * end is not always a permitted cut), w = 0, min = 0 or min > max give
 * CDC_ERR_INVALID. Asynchronous on `stream`; no handle needed. */
CDC_API cdc_status cdc_byte_shares(cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                   const uint64_t* d_bounds, size_t n, uint64_t* d_out, cdc_stream stream);

/* 128-bit fingerprints of the chunks of a buffer, for deduplication
 * reports: chunk i is [d_bounds[i-1], d_bounds[i]) (d_bounds[-1] = 0; the
 * boundary list cdc_chunk writes, each <= len), its fingerprint d_fp[2i],
 * d_fp[2i+1]. A non-cryptographic mix of the chunk's bytes and length: equal
 * chunks give equal fingerprints, different chunks collide with negligible
 * probability. The paper has no counterpart (it fingerprints on the CPU with
 * xxHash3, Section 5). Asynchronous on `stream`. */
CDC_API cdc_status cdc_fingerprint(const uint8_t* data, size_t len, const uint64_t* d_bounds, size_t n,
                                   uint64_t* d_fp, cdc_stream stream);

/* Chunk-size distribution (the paper plots its CDF per algorithm, Section
 * 5.2): chunk i of the boundary list d_bounds (n entries, as cdc_chunk writes
 * them; chunk i is [d_bounds[i-1], d_bounds[i]), d_bounds[-1] = 0) is counted
 * in bin floor(size / bin_width), sizes of n_bins * bin_width bytes or more in
 * the last bin. d_hist: n_bins uint64 counters on the device, overwritten.
 * 1 <= n_bins <= 8192, bin_width >= 1 (else CDC_ERR_INVALID). Asynchronous on
 * `stream`; no handle needed. */
CDC_API cdc_status cdc_size_histogram(const uint64_t* d_bounds, size_t n, uint64_t bin_width, uint32_t n_bins,
                                      uint64_t* d_hist, cdc_stream stream);

/* ---- resumable chunking of a stream that arrives in pieces ----------------
 *
 * A feed chunks one stream that is handed over piece by piece (device
 * buffers of any size, including 0) and emits each chunk as soon as no later
 * byte can change it. Each algorithm works one chunk at a time (Section 3.3),
 * and the chunk that starts at s depends only on the bytes before s + H, with
 * H = max for RAM / AE (the forced cut, Section 2.1) and H = max + w for MAXP
 * (a target's right window, Section 2.1; MAXP also reads the w bytes before s,
 * which the feed keeps). So a push emits every chunk whose start s has
 * s + H <= bytes received, and the final push emits the rest, ending at the
 * stream's length. The emitted lists of all pushes, concatenated, equal
 * cdc_chunk of the whole stream.
 *
 * The feed keeps the bytes from the first unsettled start (less w for MAXP)
 * in a device staging buffer it owns (at most H + w bytes between pushes)
 * and copies each piece behind them; it runs the chain on the handle h, which
 * it borrows (h must outlive the feed; calls on h and on the feed must not
 * overlap). Staging grows with the largest piece (cudaMalloc outside any
 * capture); a feed cannot be captured into a CUDA graph.
 */
typedef struct cdc_feed_s* cdc_feed;

/* Create a feed for one stream on the current device, chunked with alg and p
 * (the parameter rules of cdc_chunk). Nothing is staged until the first push. */
CDC_API cdc_status cdc_feed_create(cdc_feed* out, cdc_handle h, cdc_alg alg, cdc_params p);

/* Append `len` bytes of device memory at `piece` (the stream's next bytes)
 * and write the newly settled boundaries to out_bounds (device, uint64,
 * offsets from the START OF THE STREAM, increasing). *n: on entry the
 * capacity of out_bounds in elements, on return the count written. final_piece
 * != 0 marks the end of the stream (the last boundary is then the total
 * length); a push after it is CDC_ERR_INVALID. On CDC_ERR_CAPACITY *n holds
 * the count needed, nothing is consumed and the piece stays staged: push
 * again with len 0 (and the same final_piece) and a larger buffer.
 * Synchronises `stream` once; `piece` may be reused when the call returns.
 * Consecutive pushes may use different streams (the feed orders its own
 * copies with an event). */
CDC_API cdc_status cdc_feed_push(cdc_feed f, const uint8_t* piece, size_t len, int final_piece,
                                 uint64_t* out_bounds, size_t* n, cdc_stream stream);

/* Bytes received so far and the stream offset where the next (unsettled)
 * chunk starts; either pointer may be NULL. */
CDC_API cdc_status cdc_feed_position(cdc_feed f, uint64_t* received, uint64_t* next_start);

/* Start a new stream on the same feed (same algorithm and parameters),
 * keeping its buffers. */
CDC_API cdc_status cdc_feed_reset(cdc_feed f);

/* Release the feed's staging buffers (not the handle). NULL is accepted. */
CDC_API cdc_status cdc_feed_destroy(cdc_feed f);

/* ---- serving: requests from host memory, continuous batching --------------
 *
 * The paper has no counterpart (it chunks one stream on a CPU). A server owns
 * `slots` execution slots on one device, each with its own stream, handle
 * (workspace kept on the device), arena and pinned staging, all allocated at
 * creation within `budget_bytes` (each slot's share holds its arena for
 * request bytes, a boundary buffer of arena/1024 + max_batch + 1 entries and
 * the library's workspace for a full arena). Requests become eligible at their
 * arrival time; whenever a slot is free, a worker thread packs the eligible
 * requests that share the oldest one's algorithm and parameters (oldest first,
 * up to max_batch requests and the slot's capacity) into one batched call:
 * one copy in per request, one cdc_chunk_batch, one copy of the boundaries
 * out. Requests arriving meanwhile join later batches; batches on different
 * slots overlap on the device. Results are those of cdc_chunk on each
 * request's bytes alone.
 */
typedef struct cdc_server_s* cdc_server;

typedef struct {
    uint64_t tag;        /* the caller's id from cdc_server_submit */
    uint64_t n_bounds;   /* boundaries of the request (copied out if they fit) */
    double t_arrive_ms;  /* arrival, submission, start of its batch and */
    double t_submit_ms;  /* completion, in ms on the server's clock */
    double t_start_ms;   /* (cdc_server_clock) */
    double t_done_ms;
    int32_t status;      /* cdc_status of the request */
    int32_t alg;
    uint32_t batch_size; /* requests in its batch */
    uint32_t pad;
} cdc_result;

/* budget_bytes >= 64 MiB; 1 <= slots <= 64; max_batch 0 = 4096. Allocates
 * everything up front (CDC_ERR_NOMEM if it does not fit). */
CDC_API cdc_status cdc_server_create(cdc_server* out, int device, size_t budget_bytes, int slots, size_t max_batch);

/* Queue a request: len bytes at host_data (pinned memory is fastest; it must
 * stay valid and unchanged until the request completes), boundaries into
 * host_bounds (capacity entries; CDC_ERR_CAPACITY in the result, with
 * n_bounds set, if they do not fit). It becomes eligible at arrive_ms on the
 * server's clock (earlier values, e.g. 0 or -1: now). Parameters as for
 * cdc_chunk with min >= 64; CDC_ERR_CAPACITY here if len exceeds a slot's
 * arena or len / min + 1 its boundary buffer. */
CDC_API cdc_status cdc_server_submit(cdc_server s, cdc_alg alg, cdc_params p, const uint8_t* host_data, size_t len,
                                     uint64_t* host_bounds, size_t capacity, uint64_t tag, double arrive_ms);

/* Up to max finished requests (waiting up to wait_ms for the first); *n is
 * the number returned. Returns a sticky error of the engine, else CDC_OK. */
CDC_API cdc_status cdc_server_poll(cdc_server s, cdc_result* out, int max, int* n, int wait_ms);

/* The server's clock: ms since cdc_server_create. */
CDC_API cdc_status cdc_server_clock(cdc_server s, double* now_ms);

/* Finishes the queued requests, then frees everything. */
CDC_API cdc_status cdc_server_destroy(cdc_server s);

CDC_API const char* cdc_status_string(cdc_status s);

#ifdef __cplusplus
}
#endif

#endif /* CDC_H */
