/*
 * bp128.h -- C ABI of the GB300 library for S4-BP128-D4 posting lists:
 * decoding and conjunctive intersection (Lemire, Boytsov and Kurz, "SIMD
 * Compression and the Intersection of Sorted Integers", arXiv 1401.6399).
 *
 * Problem statement (Section 1, Section 6): posting lists are sorted lists of
 * distinct 32-bit document identifiers, stored compressed; the library takes
 * compressed lists in and returns the decoded list, or the sorted
 * intersection of several lists.  All arithmetic is exact 32-bit integer.
 *
 * Conventions for every call
 *  - Host calls are synchronous and use caller-owned host buffers.
 *  - Device calls take device pointers and a CUDA stream (cudaStream_t passed
 *    as void*; NULL means the legacy default stream).  They only enqueue
 *    work: they allocate no memory, never synchronise the stream, and return
 *    once the kernels are queued.  The caller owns every buffer and must keep
 *    it alive until the stream reaches that point.
 *  - The return value reports argument errors and launch failures at once
 *    (BP_ERR_ARG, BP_ERR_CUDA).  Errors found in the data (a corrupt stream,
 *    a full output buffer, a wait that timed out) are written by the kernels
 *    to *d_status, a device uint32 that the caller sets to BP_OK before the
 *    first call and reads after synchronising; the first error recorded wins.
 *    Several calls may share one status word.
 *  - Scratch: calls that need temporary device memory take (d_scratch,
 *    scratch_bytes); the matching *_scratch_bytes() function gives the
 *    required size, and a smaller buffer returns BP_ERR_SCRATCH.  Scratch
 *    needs no initialisation and its contents are undefined afterwards.
 *  - Nothing here falls back to the CPU.
 */
#ifndef BP128_H
#define BP128_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BP_OK = 0,
  BP_ERR_ARG = 1,      /* invalid argument                                */
  BP_ERR_UNSORTED = 2, /* encoder input not strictly increasing          */
  BP_ERR_CORRUPT = 3,  /* malformed compressed stream                    */
  BP_ERR_CAPACITY = 4, /* output buffer too small                        */
  BP_ERR_CUDA = 5,     /* a CUDA launch or API call failed               */
  BP_ERR_TIMEOUT = 6,  /* a bounded device wait gave up                  */
  BP_ERR_SCRATCH = 7   /* scratch buffer too small                       */
} bp_status;

typedef enum {
  /* The paper's S4-BP128-D4 byte layout (Section 4.3): meta-blocks of 16
   * width bytes followed by 16 blocks of 128 integers, each block 4b words in
   * the 4-lane interleave of Fig. 2 holding D4 deltas (Section 5) carried
   * from block to block; leftover whole blocks each with their own width
   * byte; fewer than 128 final integers as varint (Section 4.1).  Our
   * reading of what the paper leaves open: a 16-byte header
   * {u32 n, u32 0, u32 tail_bytes, u32 0} and D1 gaps in the varint tail. */
  BP_LAYOUT_PAPER = 0,
  /* The GPU layout: same 128-integer blocks, one bit width per block and D4
   * deltas, but each block restarts D4 from its first value (a per-block
   * skip header), and a block's deltas are stored column-major -- the delta
   * of in-block position 4t+s at bit b*(32s+t) -- so that warp lane l
   * (column l/8, rows 4(l%8)..4(l%8)+3) reads one contiguous 4b-bit field.
   * Header (64 bytes, u32 little endian): magic 0x344C4742, layout 1, n,
   * nblocks, nsuper, payload_words, off_first, off_sbo, off_bw, off_payload,
   * total bytes (u64), zeros; then first[nblocks] u32 (x[128k]),
   * sbo[nsuper+1] u32 (payload word offset of every 32nd block),
   * bw[nblocks] u8 (bit widths), payload words; sections 16-byte aligned. */
  BP_LAYOUT_GPU = 1,
  /* A bitmap over the docID universe, for the long lists of a hybrid index
   * (the hyb+m2 framework the paper's query experiments use: lists whose
   * average gap is at most B are stored as bitmaps, the others compressed;
   * Section 7.7).  Header (16 bytes, u32 little endian): magic 0x314D5042,
   * layout 2, n, words; then `words` u32 (a multiple of 4): bit v%32 of
   * word v/32 is set iff v is in the list.  Only bp_query_batch reads it. */
  BP_LAYOUT_BITMAP = 2,
  /* S4-FastPFOR (Section 4.4, Fig. 3) in a GPU layout: GL's blocks (any
   * kind of differential coding, each restarting from its first value) and
   * pages of 32 blocks, every block bit packed at a width b' <= b chosen to
   * minimize 128 b' + c (b - b' + 8) (c: deltas >= 2^b', the exceptions).
   * Header (16 u32): magic 0x34504742, 3, n, nblocks, npages, payload
   * words, off_first, off_spo, off_meta, off_payload, total bytes (u64),
   * kind, 0, 0, 0; then first[nblocks] u32, spo[npages+1] u32 (payload
   * word offset of each page), meta[nblocks] 4 bytes {b', b - b', c, 0},
   * payload; sections 16-byte aligned.  Page p: the b' low bits of each of
   * its blocks (4 b' words, GL order), then the c position bytes of each
   * block (ascending, zero-padded to a word), then the b - b' high bits of
   * each exception in order (LSB first, zero-padded to a word), the page
   * zero-padded to 4 words.  Decoded by bp_decode, bp_decode_sum and
   * bp_decode_batch; not by the intersection calls. */
  BP_LAYOUT_PFOR = 3
} bp_layout;

/* Kind of differential coding of a stream (Section 5), stored in its
 * header (word 3 of the paper layout's, word 12 of the GPU layout's):
 *   D4  delta[i] = x[i] - x[i-4]                       (the default)
 *   DM  delta[4t+s] = x[4t+s] - x[4t-1]   (every 4-vector minus the last
 *                                          value of the previous one)
 *   D2  delta[i] = x[i] - x[i-2]
 *   D1  delta[i] = x[i] - x[i-1]
 * In the paper layout the values before the list are 0 and deltas run on
 * from block to block; in the GPU layout every block starts again from its
 * first value.  Decoding reads the kind from the header.  The fused
 * intersection paths (bp_intersect_pair with BP_MODE_FUSED or AUTO,
 * bp_intersect_pair_noalloc, bp_query_batch) take D4 streams only and record
 * BP_ERR_ARG for others; BP_MODE_UNFUSED and bp_query_one take every kind. */
typedef enum {
  BP_DELTA_D4 = 0,
  BP_DELTA_DM = 1,
  BP_DELTA_D2 = 2,
  BP_DELTA_D1 = 3
} bp_delta;

/* One list of a batch.  Filled by the caller except unit_base, which
 * bp_plan_lists() fills. */
typedef struct bp_list {
  uint64_t enc_offset; /* byte offset of the stream in the data buffer;
                          16-byte aligned                                   */
  uint64_t enc_bytes;  /* size of the stream in bytes                       */
  uint64_t out_offset; /* element offset of the decoded list in the output  */
  uint64_t unit_base;  /* first work unit of this list (bp_plan_lists)      */
  uint32_t n;          /* number of integers, equal to the stream header    */
  uint32_t layout;     /* bp_layout; all lists of one call share it         */
  uint64_t reserved;
} bp_list;

/* Intersection modes of bp_intersect_pair. */
typedef enum {
  BP_MODE_AUTO = 0,    /* fused for BP_LAYOUT_GPU, unfused for the paper layout */
  BP_MODE_UNFUSED = 1, /* decode both lists to scratch, intersect the arrays    */
  BP_MODE_FUSED = 2    /* BP_LAYOUT_GPU only: decode only candidate blocks      */
} bp_mode;

/* Tuning parameters (process-wide; bp_set_tuning installs the autotuner's
 * choice).  dense_blocks is the skew threshold between the two regimes of
 * Section 6: a 128-value chunk of the shorter list whose range covers at
 * most dense_blocks blocks of the longer list decodes them all and searches
 * them (similar lengths, the V1/V3 regime); a wider range decodes only the
 * blocks that some value falls in, found by binary search over the skip
 * headers (skewed lengths, the galloping regime).  query_chunk_blocks is the
 * number of blocks of a query's shortest list per work item in
 * bp_query_batch, query_warps the warps per CTA of its persistent kernel.
 * merge_span selects the merge regime for similar lengths: a run of the
 * shorter list whose value range covers at most merge_span blocks of the
 * longer list per block of its own is intersected by merging the decoded
 * runs (Section 6's merge, split over a warp's lanes by merge path) instead
 * of by searching; 0 turns the merge regime off.  In bp_query_batch it
 * applies to the first list a query's candidates meet.
 *
 * The last two fields bound and test the waits of the ordered output of
 * bp_intersect_pair (each CTA, in ticket order, waits for the output counts
 * of the CTAs before it).  lookback_spin_limit is the number of polls of
 * one predecessor's count before the wait gives up, records BP_ERR_TIMEOUT
 * in the status word and carries on (0: the default, 2^22 polls, seconds).
 * withhold_tile = k > 0 makes tile k - 1 of every later pair call publish
 * no count, so that the tiles after it exhaust their polls: it exists to
 * show that such a wait ends and is reported, and must stay 0 otherwise
 * (the output of a call made with it is wrong by design). */
typedef struct bp_tuning {
  uint32_t dense_blocks;        /* 1..8, default 4 */
  uint32_t query_chunk_blocks;  /* 1..8, default 1 */
  uint32_t query_warps;         /* 4 or 8, default 8 */
  uint32_t lookback_spin_limit; /* 0 (default 2^22) or 1..2^22 */
  uint32_t withhold_tile;       /* 0 (none), or 1 + the tile to withhold */
  uint32_t merge_span;          /* 0 (off, the default) or 1..64 */
  uint32_t reserved[2];
} bp_tuning;

/* Status text for a bp_status code (static string, never NULL). */
const char *bp_status_string(int status);

/* ---------------------------------------------------------------- host -- */

/* Upper bound of the encoded size of n integers in `layout`. */
size_t bp_encode_bound(size_t n, int layout);

/* Encode n strictly increasing uint32 (Section 3: sorted distinct docIDs)
 * into out[0..cap) in `layout`; *out_bytes receives the size.  Errors:
 * BP_ERR_UNSORTED, BP_ERR_CAPACITY (cap < bp_encode_bound), BP_ERR_ARG.
 * nthreads <= 1 encodes on the calling thread; more split the blocks over
 * that many host threads (the output is identical). */
int bp_encode(const uint32_t *in, size_t n, int layout, uint8_t *out,
              size_t cap, size_t *out_bytes, int nthreads);

/* bp_encode with the kind of differential coding `delta` (bp_delta);
 * bp_encode is this call with BP_DELTA_D4.  BP_ERR_ARG for an unknown kind.
 * delta may be or-ed with BP_ENCODE_ANY_ORDER: the input is then any
 * sequence of uint32 (deltas modulo 2^32; decoding returns it exactly, as
 * the codec's arithmetic is modular) instead of a strictly increasing
 * posting list.  Such streams are for decoding only: the intersection calls
 * assume sorted lists. */
#define BP_ENCODE_ANY_ORDER 0x100
int bp_encode_kind(const uint32_t *in, size_t n, int layout, int delta,
                   uint8_t *out, size_t cap, size_t *out_bytes, int nthreads);

/* Parse a stream header on the host: *n_out = number of integers,
 * *layout_out = its layout.  BP_ERR_CORRUPT if the header is invalid. */
int bp_stream_info(const uint8_t *enc, size_t enc_bytes, uint32_t *n_out,
                   int *layout_out);

/* The kind of differential coding (bp_delta) of a stream whose header
 * bp_stream_info accepts.  BP_ERR_CORRUPT otherwise. */
int bp_stream_kind(const uint8_t *enc, size_t enc_bytes, int *delta_out);

/* Index builder: encode `count` lists (list i = values[offs[i] ..
 * offs[i+1]), strictly increasing) in BP_LAYOUT_GPU back to back into out
 * (each stream 16-byte aligned, cap bytes; bp_index_bound gives enough) and
 * fill lists[i] (enc_offset, enc_bytes, out_offset = offs[i], n, layout,
 * unit_base as bp_plan_lists).  *out_bytes: bytes used.  Errors as
 * bp_encode.  nthreads host threads share the lists. */
size_t bp_index_bound(const uint64_t *offs, uint32_t count);
int bp_index_encode(const uint32_t *values, const uint64_t *offs,
                    uint32_t count, uint8_t *out, size_t cap, bp_list *lists,
                    size_t *out_bytes, int nthreads);

/* Hybrid index (hyb+m2): as bp_index_encode, except that every list whose
 * average gap is at most B (n * B >= universe) is stored as a
 * BP_LAYOUT_BITMAP of `universe` bits (every value must be below it).
 * B = 0 stores no bitmap.  lists[i].layout tells which form each list took. */
size_t bp_index_hybrid_bound(const uint64_t *offs, uint32_t count, uint32_t universe,
                             uint32_t B);
int bp_index_encode_hybrid(const uint32_t *values, const uint64_t *offs, uint32_t count,
                           uint32_t universe, uint32_t B, uint8_t *out, size_t cap,
                           bp_list *lists, size_t *out_bytes, int nthreads);

/* Fill lists[i].unit_base for a batch of `count` lists of one layout and
 * return the total number of work units (GL: groups of 32 blocks; PL: blocks
 * of 128 integers plus one unit for each list's tail). */
uint64_t bp_plan_lists(bp_list *lists, uint32_t count);

/* -------------------------------------------------------------- device -- */

/* Scratch needed by bp_decode / bp_decode_sum for a list of n integers
 * (0 for BP_LAYOUT_GPU; PL needs per-block offsets and scan state). */
size_t bp_decode_scratch_bytes(size_t n, int layout);

/* Decode one compressed list of n integers (Section 4.3 container;
 * Algorithm 1 unpacking with the D4 prefix of Section 5).  d_enc: device
 * stream of enc_bytes bytes, 16-byte aligned; n: its integer count (from
 * bp_encode or bp_stream_info), which the device checks against the stream
 * header (mismatch: BP_ERR_CORRUPT); d_out: out_cap >= n uint32 (else
 * BP_ERR_CAPACITY, returned at once).  A corrupt stream records
 * BP_ERR_CORRUPT in *d_status and leaves the output undefined.  Scratch:
 * bp_decode_scratch_bytes(n, layout); the call also enqueues a memset of
 * part of it. */
int bp_decode(const uint8_t *d_enc, size_t enc_bytes, int layout, size_t n,
              uint32_t *d_out, size_t out_cap, void *d_scratch,
              size_t scratch_bytes, uint32_t *d_status, void *stream);

/* As bp_decode, but instead of storing the list adds the exact sum of its
 * values (mod 2^64) to *d_sum (a device uint64 the caller zeroes). */
int bp_decode_sum(const uint8_t *d_enc, size_t enc_bytes, int layout,
                  size_t n, uint64_t *d_sum, void *d_scratch,
                  size_t scratch_bytes, uint32_t *d_status, void *stream);

/* Scratch needed by bp_decode_batch for these lists (host array). */
size_t bp_decode_batch_scratch_bytes(const bp_list *lists, uint32_t count);

/* Decode `count` lists of one layout in one pass.  d_data: device buffer the
 * streams live in; d_lists: device copy of the planned descriptors
 * (bp_plan_lists); total_units: its return value.  List i is written to
 * d_out[out_offset .. out_offset + n) (out_cap elements in total).  If
 * d_sums is not NULL the lists are summed instead of stored: d_sums[i] +=
 * sum of list i (device uint64, zeroed by the caller) and d_out is unused. */
int bp_decode_batch(const uint8_t *d_data, const bp_list *d_lists,
                    uint32_t count, uint64_t total_units, int layout,
                    uint32_t *d_out, uint64_t out_cap, uint64_t *d_sums,
                    void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                    void *stream);

/* Decode GPU-layout lists of any kind with the differential coding either
 * integrated into the unpacking (two_pass = 0: each unpacked 4-vector is
 * prefixed before it is stored, Algorithm 1) or applied as a separate pass
 * (two_pass = 1, the regular scheme Section 7.4 measures against, Figure 6a):
 * each block's deltas are stored to a buffer of 128 words of shared memory
 * per warp, read back and prefixed.  Both variants run one list-major
 * kernel of identical structure, so the difference between them is what
 * integration saves; the output equals bp_decode_batch's.  d_lists: device descriptors (out_offset, n,
 * enc_offset, enc_bytes; unit_base is not used); a list that is not a GL
 * stream records BP_ERR_CORRUPT, one that does not fit out_cap
 * BP_ERR_CAPACITY. */
int bp_decode_ablation(const uint8_t *d_data, const bp_list *d_lists,
                       uint32_t count, uint32_t *d_out, uint64_t out_cap,
                       uint32_t *d_status, int two_pass, void *stream);

/* bp_decode_batch from and to host memory, for callers that keep the
 * compressed lists on the host: enqueues on `stream` the copy of h_data
 * (data_bytes) to d_data and of h_lists (count planned descriptors) to
 * d_lists, a reset of *d_status, the decode, and the copies of the decoded
 * lists (sum of n over the lists, as uint32) to h_out and of the status to
 * *h_status.  When the lists are laid out in order (streams and outputs
 * ascending and disjoint, as bp_plan_lists plans them for packed buffers)
 * and there are at least two, the copies and the decode run as a pipeline
 * over groups of lists on the library's own streams, forked from `stream`
 * and joined back into it (later work on `stream` still runs after the
 * call); d_lists then holds per-group rebased descriptors afterwards.  Host
 * buffers should be pinned for the copies to be asynchronous; all buffers
 * belong to the caller and must stay alive until the stream has passed the
 * call.  Layout, scratch and errors as in bp_decode_batch (sums are not
 * offered here). */
int bp_decode_batch_host(const uint8_t *h_data, size_t data_bytes,
                         const bp_list *h_lists, uint32_t count,
                         uint64_t total_units, int layout, uint8_t *d_data,
                         bp_list *d_lists, uint32_t *d_out, uint64_t out_cap,
                         uint32_t *h_out, void *d_scratch, size_t scratch_bytes,
                         uint32_t *d_status, uint32_t *h_status, void *stream);

/* Current tuning parameters / install new ones (BP_ERR_ARG if out of
 * range).  Calls already enqueued keep the values they were launched with. */
int bp_get_tuning(bp_tuning *out);
int bp_set_tuning(const bp_tuning *in);

/* Scratch needed by bp_intersect_pair for lists of n_a and n_b integers. */
size_t bp_intersect_scratch_bytes(size_t n_a, size_t n_b, int layout, int mode);

/* Sorted intersection of two compressed lists of distinct sorted integers
 * (Section 6: the shorter list r is searched in the longer list f; the
 * result is the values of r found in f, ascending).  Streams as in
 * bp_decode (device, 16-byte aligned, n checked against the header).
 * Writes min(count, out_cap) values to d_out and the count to *d_count
 * (device uint32); count > out_cap records BP_ERR_CAPACITY (out_cap >=
 * min(n_a, n_b) always suffices).  layout: BP_LAYOUT_PAPER or
 * BP_LAYOUT_GPU (BP_ERR_ARG otherwise); mode: bp_mode; BP_MODE_FUSED needs
 * BP_LAYOUT_GPU (else BP_ERR_ARG).  Scratch: bp_intersect_scratch_bytes;
 * the call enqueues a memset of part of it. */
int bp_intersect_pair(const uint8_t *d_a, size_t a_bytes, size_t n_a,
                      const uint8_t *d_b, size_t b_bytes, size_t n_b,
                      int layout, int mode, uint32_t *d_out, size_t out_cap,
                      uint32_t *d_count, void *d_scratch, size_t scratch_bytes,
                      uint32_t *d_status, void *stream);

/* The paper has no counterpart to this call; it exists for the library's
 * users.  bp_intersect_pair for callers that cannot allocate device memory:
 * a plug-in that only works on the buffers its host framework hands it, a
 * server whose pool already holds all device memory, or latency-bound code
 * that must not call cudaMalloc (it can synchronise the device) has no way
 * to provide the scratch buffer bp_intersect_pair asks for.  This call
 * computes the same intersection of two BP_LAYOUT_GPU lists (arguments,
 * output and errors as in bp_intersect_pair with BP_MODE_FUSED) with a
 * simpler, fixed schedule -- one block of 128 values of the shorter list
 * per warp, no choice of run length, no shared-memory window carried from
 * run to run -- so its speed can differ from bp_intersect_pair's, most on
 * very skewed pairs.  It keeps its scratch in a 256 KiB array of device
 * memory that the library reserves on every GPU that loads it, for the life
 * of the process; it allocates nothing.  The shorter list may hold at most
 * BP_NOALLOC_MAX_SHORT_LIST integers (larger: BP_ERR_SCRATCH, nothing
 * enqueued).  The first call on a device looks up the array's device
 * address (a runtime call) and keeps it, so make that first call before any
 * stream capture, and do not use the call again on a device after
 * cudaDeviceReset (the kept address would be stale).  All calls share the
 * array and each clears the part it uses: calls whose work overlaps on the
 * GPU corrupt each other's results, so issue them in order on one stream. */
#define BP_NOALLOC_MAX_SHORT_LIST 33552384u
int bp_intersect_pair_noalloc(const uint8_t *d_a, size_t a_bytes, size_t n_a,
                              const uint8_t *d_b, size_t b_bytes, size_t n_b,
                              uint32_t *d_out, size_t out_cap,
                              uint32_t *d_count, uint32_t *d_status,
                              void *stream);

/* ---- conjunctive queries over a resident index -------------------------- *
 * The index is a device buffer d_data holding one GL stream per term
 * (16-byte aligned) -- or, in a hybrid index, a BP_LAYOUT_BITMAP stream for
 * the longest lists -- and a device array d_lists of n_terms descriptors
 * (enc_offset, enc_bytes, n, layout; the other fields are ignored).  A
 * query is a set of term ids; its answer is the sorted intersection of their
 * lists (Section 1 and Section 6: Set-vs-Set, from the shortest list; in a
 * hybrid index the compressed lists first, then one bit test per surviving
 * candidate for each bitmap, as in hyb+m2). */

/* Scratch needed by bp_query_batch; host copies of the index descriptors
 * and of the queries' terms, out_cap as passed to bp_query_batch. */
size_t bp_query_batch_scratch_bytes(const bp_list *h_lists, uint32_t n_terms,
                                    const uint32_t *h_terms,
                                    const uint64_t *h_term_off,
                                    uint32_t n_queries, uint64_t out_cap);

/* Answer n_queries queries in one pass: query q has the terms
 * d_terms[d_term_off[q] .. d_term_off[q+1]) (at most 64; device arrays,
 * total_terms = d_term_off[n_queries]).  The answers are written back to
 * back in query order to d_out (out_cap uint32 in total): query q's answer
 * starts at d_out_off[q] (device uint64, n_queries+1 entries) and has
 * d_counts[q] values (device uint32).  A total beyond out_cap, or beyond the
 * work items the scratch holds, records BP_ERR_CAPACITY / BP_ERR_SCRATCH;
 * counts and offsets stay exact.  An unknown term id records BP_ERR_ARG.
 * Every launch size depends only on n_queries and the buffers, so the call
 * can be captured in a CUDA graph and replayed with new terms in the same
 * device arrays. */
int bp_query_batch(const uint8_t *d_data, const bp_list *d_lists,
                   uint32_t n_terms, const uint32_t *d_terms,
                   const uint64_t *d_term_off, uint64_t total_terms,
                   uint32_t n_queries, uint32_t *d_out, uint64_t out_cap,
                   uint64_t *d_out_off, uint32_t *d_counts, void *d_scratch,
                   size_t scratch_bytes, uint32_t *d_status, void *stream);

/* Scratch needed by bp_query_one for the k terms h_terms. */
size_t bp_query_one_scratch_bytes(const bp_list *h_lists, uint32_t n_terms,
                                  const uint32_t *h_terms, uint32_t k);

/* One query, the plain way: every list of the query is decoded whole into
 * scratch, then the decoded arrays are intersected two at a time from the
 * shortest (decompress-then-intersect, Section 7.6 of the paper).  h_lists:
 * host copy of the descriptors; h_terms: k host term ids (GL lists only:
 * BP_ERR_ARG for a bitmap term).  Answer in d_out[0..count), count in
 * *d_count (device). */
int bp_query_one(const uint8_t *d_data, const bp_list *h_lists,
                 uint32_t n_terms, const uint32_t *h_terms, uint32_t k,
                 uint32_t *d_out, size_t out_cap, uint32_t *d_count,
                 void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                 void *stream);

/* ---- serving ------------------------------------------------------------- *
 * A serving engine over a resident index (not in the paper: its query
 * processing of Section 7.6, run continuously).  Queries are submitted from
 * any host thread; a dispatcher thread batches them continuously: whenever
 * one of `slots` batch slots is free it admits waiting queries in arrival
 * order as long as their scratch and answer capacity fit the slot's memory,
 * and launches them with bp_query_batch on the slot's stream, so new
 * requests join while earlier batches are still on the GPU and several
 * batches overlap on the device.  The kernels write a batch's answers to
 * the slot's device memory (slot_bytes holds them and the batch's scratch)
 * and its answer counts and offsets to the slot's pinned host memory, which
 * must be device-accessible (pinned memory on a unified-address system);
 * once the batch is done the engine copies exactly its answer values to the
 * pinned memory with one transfer.  The engine allocates no device or
 * pinned memory and creates only one event per slot. */
typedef struct bp_server bp_server;

typedef struct bp_server_config {
  uint32_t slots;             /* batches in flight (one stream each), 1..16 */
  uint32_t max_batch_queries; /* queries per batch                         */
  uint32_t max_terms;         /* terms per query, 1..64                    */
  uint32_t deliver_answers;   /* 1: bp_server_poll returns answer arrays    */
  uint64_t slot_bytes;        /* device bytes per slot (scratch + answers)  */
  uint64_t reserved[4];
} bp_server_config;

/* Times are steady-clock seconds.  arrival_s is when the query was due:
 * its scheduled arrival under bp_server_replay, else the moment
 * bp_server_submit was called; submit_s is when it entered the queue
 * (submit_s - arrival_s is the load generator's lag); done_s is when the
 * dispatcher saw its batch finish.  Latency = done_s - arrival_s. */
typedef struct bp_server_result {
  uint64_t tag;
  uint32_t count;          /* answer values                               */
  int32_t status;          /* BP_OK, or the error of the query's batch    */
  double arrival_s, submit_s, done_s;
  const uint32_t *answer;  /* deliver_answers = 1: valid until the next poll */
} bp_server_result;

/* One launched batch, for a timeline of the engine: the slot, its queries,
 * the earliest arrival among them, when admission started, when the
 * launches had been enqueued, when the dispatcher saw the batch finish,
 * and when its answers were handed over. */
typedef struct bp_server_batch {
  uint32_t slot, queries;
  uint64_t answer_values;
  double first_arrival_s, admit_s, launched_s, done_s, retired_s;
} bp_server_batch;

/* Device bytes (slots x slot_bytes) and pinned host bytes the engine needs. */
size_t bp_server_device_bytes(const bp_server_config *cfg);
size_t bp_server_host_bytes(const bp_server_config *cfg);

/* Start an engine.  d_data/d_lists: the index (as bp_query_batch); h_lists:
 * host copy of the descriptors; d_mem, h_pinned: caller buffers of the sizes
 * above; streams: cfg->slots CUDA streams.  NULL on error (*err set). */
bp_server *bp_server_create(const uint8_t *d_data, const bp_list *d_lists,
                            const bp_list *h_lists, uint32_t n_terms,
                            const bp_server_config *cfg, void *d_mem,
                            void *h_pinned, void *const *streams, int *err);

/* Queue one query of k terms under `tag` (thread-safe). */
int bp_server_submit(bp_server *s, uint64_t tag, const uint32_t *terms,
                     uint32_t k);

/* Open-loop load: submit query i (terms[term_off[i]..term_off[i+1])) at
 * arrival_s[i] seconds after the call starts, on the calling thread,
 * whatever the engine's progress.  Each query's arrival_s in its result is
 * that scheduled time, so a late submission counts in its latency. */
int bp_server_replay(bp_server *s, const uint64_t *tags, const uint32_t *terms,
                     const uint64_t *term_off, uint32_t n,
                     const double *arrival_s);

/* Move up to max finished queries to out; returns how many. */
uint32_t bp_server_poll(bp_server *s, bp_server_result *out, uint32_t max);

/* Wait until every submitted query has finished (BP_ERR_TIMEOUT after
 * timeout_s); returns the first error seen, else BP_OK. */
int bp_server_drain(bp_server *s, double timeout_s);

/* out = {submitted, completed, batches launched, rejected (too large for a
 * slot), most slots busy at once, queries waiting}. */
int bp_server_stats(bp_server *s, uint64_t out[6]);

/* Move up to max records of retired batches (oldest first) to out; returns
 * how many.  The engine keeps the records of the last 2^20 batches. */
uint32_t bp_server_batches(bp_server *s, bp_server_batch *out, uint32_t max);

/* Finish the queued and running queries, then stop the engine. */
void bp_server_destroy(bp_server *s);

#ifdef __cplusplus
}
#endif
#endif
