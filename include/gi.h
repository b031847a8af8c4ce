/*
 * gi.h -- C ABI of a static GPU index over (key, rowID) pairs, stored in sorted,
 * Eytzinger (EBS) or k-ary Eytzinger (EKS) order, for NVIDIA GB300 (sm_103a).
 *
 * Method: Henneberg & Schuhknecht, "Bigger Is Not Better: The Fastest Static GPU
 * Index Is Also Lightweight!" (arXiv 2506.01576).
 *   Problem statement (point and range lookups) ........ Section 1
 *   Sorted array + binary search (BS) .................. Section 3
 *   Eytzinger order, EBS lookup ........................ Section 3, Figs 5-6
 *   One-read-one-write permutation into that order ..... Section 4 (p(t), p'(t))
 *   Range lookups over Eytzinger order ................. Section 5
 *   k-ary Eytzinger order and EKS lookup ............... Section 6 (6.1, 6.2)
 *   Cache pinning of top levels, static scheduling ..... Sections 7.2, 7.3
 *   Coalescing micro-benchmark ......................... Section 5.1, Fig 9
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers.  Every data pointer may be DEVICE memory (e.g. a torch CUDA
 *    tensor's data_ptr) or HOST memory (pinned or pageable).  Device pointers are
 *    used in place and the call is asynchronous on the index's stream.  When any
 *    input or output of a call is host memory, the library stages it through
 *    device buffers it owns (pipelined in chunks on internal streams) and the call
 *    returns only after the host outputs are written.  Device pointers must belong
 *    to the current device.
 *  - Ownership.  gi_build copies what it needs: the caller keeps keys/rowids.
 *    Outputs are always caller-allocated.  The index owns its device arrays and
 *    internal scratch; gi_destroy frees them.
 *  - Keys are unsigned 32- or 64-bit integers (GI_KEY_U32 / GI_KEY_U64, OR-ed
 *    into `layout`); probes and range bounds have the index's key width.
 *  - rowIDs are uint32; the value GI_MISS is reserved: it is what a point lookup
 *    that finds nothing reports, and gi_build rejects it as an input rowID.
 *  - Duplicate keys are allowed.  Ties keep input order (a stable sort): a point
 *    lookup returns the rowID of the first entry in that order (lower bound), a
 *    range lookup returns all of them in (key, input position) order.
 *  - Return codes: GI_OK or a GI_ERR_* code; gi_last_error() then holds a
 *    message (thread-local, valid until the next call on the same thread).
 *    Errors found on the device (a bounded wait that gave up) are latched in the
 *    index and reported by gi_sync or by the next call that synchronises.
 */
#ifndef GI_H_
#define GI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gi_index gi_index;

/* Layout (low byte of `layout`). */
#define GI_SORTED         0 /* ascending order; textbook binary search (Section 3)   */
#define GI_EYTZINGER      1 /* Eytzinger order, 1-based, empty slot 0 (Sections 3-4) */
#define GI_EYTZINGER_KARY 2 /* k-ary Eytzinger order, k-1 keys per node (Section 6)  */
/* Key width, OR-ed into `layout`. */
#define GI_KEY_U32 0x000
#define GI_KEY_U64 0x100
/* Build flags, OR-ed into `layout` of gi_build (at most one).  Both give the same
 * index; they choose how the pairs are sorted.
 *   default          u64 keys with at least five non-trivial digits (bytes that
 *                    differ between keys) and 2^18 <= n <= 2^28 + 2^27 (about), and
 *                    u32 keys with four non-trivial digits and 2^23 <= n <= that
 *                    bound, take the hybrid sort: a stable scatter on the 8 bits just below the
 *                    highest bit in which two keys differ, then one on up to 8
 *                    further bits (as many as split the largest bucket into pieces
 *                    of about 2048 pairs), then every resulting bucket sorted in
 *                    one CTA's shared memory and written straight into the layout.
 *                    Smaller or narrower inputs, and inputs whose buckets come out
 *                    larger than 5120 pairs, take the plain LSD sort.
 *   GI_BUILD_LSD     always the plain 8-bit LSD radix passes (then the permutation).
 *   GI_BUILD_HYBRID  the hybrid sort whenever it can run (at least two non-trivial
 *                    digits, n < 2^32, buckets of at most 5120 pairs), whatever n
 *                    and the key width; else the LSD sort. */
#define GI_BUILD_LSD 0x10000
#define GI_BUILD_HYBRID 0x20000

/* Return codes. */
#define GI_OK          0
#define GI_ERR_INVALID 1 /* bad argument (null/misaligned pointer, bad layout/k, reserved rowID) */
#define GI_ERR_NOMEM   2 /* device or pinned allocation failed                          */
#define GI_ERR_CUDA    3 /* a CUDA runtime call failed                                  */
#define GI_ERR_TIMEOUT 4 /* a bounded device-side wait gave up; results are not valid  */
#define GI_ERR_CAPACITY 5 /* a served range result is larger than the room given for it */

#define GI_MISS 0xFFFFFFFFu

/*
 * gi_build -- build an index over n (key, rowID) pairs.                (Sections 3, 4, 6.1)
 *   keys    n keys of the width given in `layout` (device or host memory).
 *   rowids  n uint32 rowIDs; rowids[j] belongs to keys[j]; none may equal GI_MISS.
 *   n       number of pairs; 0 is valid (every lookup misses, every range is empty).
 *   layout  GI_SORTED | GI_EYTZINGER | GI_EYTZINGER_KARY, OR-ed with GI_KEY_U32/U64.
 *   k       fan-out for GI_EYTZINGER_KARY, 2 <= k <= 33 (nodes of k-1 keys); the
 *           paper prefers k-1 a power of two (Section 6.1).  Ignored otherwise.
 *   out     receives the new index.
 * The pairs are key-value radix sorted (stable; see GI_BUILD_LSD) and, for the Eytzinger layouts,
 * moved into place by the closed-form permutation of Sections 4 and 6.1.  Runs on
 * the thread's default gi stream (gi_set_stream(NULL, s)); returns after the index
 * is complete.  The index stores exactly n keys and n rowIDs (plus the empty slot
 * 0 of GI_EYTZINGER, Section 3).
 * Errors: GI_ERR_INVALID (bad layout/k/pointer, a rowID equal to GI_MISS),
 * GI_ERR_NOMEM, GI_ERR_CUDA, GI_ERR_TIMEOUT.  On error *out is set to NULL.
 */
int gi_build(const void* keys, const uint32_t* rowids, uint64_t n, int layout, uint32_t k,
             gi_index** out);

/*
 * gi_point_lookup -- m point lookups.                           (Sections 1, 3, 6.2)
 *   queries     m probes of the index's key width.
 *   out_rowids  m uint32: the rowID of the first entry whose key equals
 *               queries[i], or GI_MISS.  Written in probe order.
 * SORTED: textbook lower_bound; EYTZINGER: branch-free descent; EYTZINGER_KARY:
 * one node per level, read by one thread (the default wherever that kernel is
 * compiled: k in {3, 4, 5, 8, 9, 16, 17}), with vector loads where the node is
 * whole 16- or 32-byte vectors, or by a group of lanes (GI_OPT_GROUP) that sums
 * its per-lane pivot counts; the child is s*k + (c+1)*(k-1) for c pivots below
 * the probe.
 * Errors: GI_ERR_INVALID (null index/pointer), GI_ERR_CUDA, GI_ERR_NOMEM (staging).
 */
int gi_point_lookup(const gi_index* index, const void* queries, uint64_t m,
                    uint32_t* out_rowids);

/*
 * gi_range_lookup -- m inclusive range lookups [lo[i], hi[i]] as CSR.    (Sections 1, 5)
 *   lo, hi       m bounds each, index key width; lo[i] > hi[i] is an empty range.
 *   out_offsets  m+1 uint64: out_offsets[i] is where range i's rows start,
 *                out_offsets[m] is the total row count.
 *   out_rowids   NULL, or room for out_offsets[m] uint32 rowIDs.  Range i's rows
 *                are in ascending (key, input position) order.
 * Two-call protocol: call with out_rowids == NULL to get the offsets (and the
 * total), allocate, call again with the same inputs and out_rowids set.  When
 * every pointer is device memory and the second call passes the same lo, hi, m
 * and out_offsets as the first, with no other range lookup on this index in
 * between, it reuses the first call's counts and runs only the fill pass: the
 * caller must not change lo, hi or out_offsets between the two calls.
 * Errors: GI_ERR_INVALID, GI_ERR_CUDA, GI_ERR_NOMEM (scratch or staging).
 */
int gi_range_lookup(const gi_index* index, const void* lo, const void* hi, uint64_t m,
                    uint64_t* out_offsets, uint32_t* out_rowids);

/* gi_destroy -- free the index and everything it owns (waits for its stream). NULL is a no-op. */
void gi_destroy(gi_index* index);

/*
 * gi_set_stream -- run the index's work on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  With index == NULL, sets the calling thread's default
 * stream for later gi_build calls; a built index starts on that stream.
 */
int gi_set_stream(gi_index* index, void* stream);

/* gi_sync -- wait for the index's stream; report a latched device-side error. */
int gi_sync(gi_index* index);

/* gi_last_error -- message of the last failing call on this thread ("" if none). */
const char* gi_last_error(void);

/* gi_footprint_bytes -- device bytes the index keeps: n*(key+4), + one key for GI_EYTZINGER. */
uint64_t gi_footprint_bytes(const gi_index* index);

/* Description of a built index.  `keys`/`rowids` are the index's own device arrays
 * (read-only views, valid until gi_destroy): slot t of the layout is keys[t] and
 * rowids[t], except GI_EYTZINGER where slot t (0-based) is keys[t+1], rowids[t]. */
typedef struct gi_info {
  uint64_t n;
  int32_t layout;        /* GI_SORTED / GI_EYTZINGER / GI_EYTZINGER_KARY */
  uint32_t k;            /* fan-out: 2 for GI_EYTZINGER, k for KARY, 0 for SORTED */
  uint32_t key_bytes;    /* 4 or 8 */
  uint32_t unique;       /* 1 if no two keys are equal */
  uint32_t levels;       /* tree levels (SORTED: ceil(log2(n+1))) */
  uint32_t reserved;
  const void* keys;
  const uint32_t* rowids;
  uint64_t footprint_bytes;
} gi_info;
int gi_get_info(const gi_index* index, gi_info* out);

/*
 * gi_copy_layout -- copy the index's arrays in layout order: keys_out[t] and
 * rowids_out[t] for slot t = 0..n-1 (for GI_EYTZINGER the 0-based slots, i.e.
 * without the empty slot 0).  Either output may be NULL; each may be device or
 * host memory.  Returns after the copy is complete.  Lets a caller inspect or
 * save the built order (Sections 3, 4, 6.1).
 */
int gi_copy_layout(const gi_index* index, void* keys_out, uint32_t* rowids_out);

/*
 * Tuning knobs (Sections 7.2, 7.3 and the EKS group size of Section 6.2).  A value
 * of -1 restores the automatic choice.  Values outside the supported set return
 * GI_ERR_INVALID.
 *   GI_OPT_GROUP        lanes per lookup for EYTZINGER_KARY (1 = one thread per
 *                       lookup, "EKS (single)"; up to 32; must be supported for k).
 *   GI_OPT_PER_THREAD   independent lookups interleaved per thread/group: 1, 2, 4.
 *   GI_OPT_SMEM_LEVELS  top tree levels pinned in shared memory (0 = none).
 *   GI_OPT_BLOCK        threads per block: 64, 128, 256, 512.
 *   GI_OPT_BLOCKS_PER_SM  0 = one thread (group) per work item; >0 = persistent grid
 *                       of that many blocks per SM with a static schedule.
 *   GI_OPT_PREFETCH     EYTZINGER prefetch distance in levels: 0, 2, 3, 4.
 *   GI_OPT_EARLY_EXIT   stop a point lookup at an equal pivot: 0 or 1 (only honoured
 *                       when the keys are unique, by the kernel for k values that
 *                       are not compiled in; the others resolve equality at the end).
 *   GI_OPT_HOT_LEVELS   EYTZINGER_KARY: top levels read with an L2 evict-last hint;
 *                       deeper levels, rowIDs, probes and results use evict-first
 *                       (0 = every level streamed).  Default: the levels whose keys
 *                       fit in 5/8 of L2.  (The levels whose keys fit in 128 KB are
 *                       also the only ones allocated in L1.)
 *   GI_OPT_RANGE_FILL   Eytzinger layouts: 1 writes a range's rows level by level,
 *                       one contiguous slot run per level, a warp taking runs of
 *                       >= 32 slots (Sections 5, 5.1); 0 (default) maps every rank
 *                       to its slot one at a time.  Same output either way.
 *   GI_OPT_REORDER      point lookups: 1 sorts each CTA's tile of 2048 probes in
 *                       shared memory before the descent and restores probe order
 *                       before the store (local lookup reordering, Section 7.4);
 *                       sorted, Eytzinger and k in {3, 5, 9, 17}.  Default 0.
 */
#define GI_OPT_GROUP         1
#define GI_OPT_PER_THREAD    2
#define GI_OPT_SMEM_LEVELS   3
#define GI_OPT_BLOCK         4
#define GI_OPT_BLOCKS_PER_SM 5
#define GI_OPT_PREFETCH      6
#define GI_OPT_EARLY_EXIT    7
#define GI_OPT_HOT_LEVELS    8
#define GI_OPT_RANGE_FILL    9
#define GI_OPT_REORDER       10
int gi_set_option(gi_index* index, int option, int64_t value);
int gi_get_option(const gi_index* index, int option, int64_t* value);

/*
 * Autotuner.  The paper picks block size, lookups per thread, limited concurrency,
 * pinned levels, prefetch distance, lane-group size and lookup reordering by sweeps
 * per figure (Sections 7.2-7.4, 8.2-8.4); this runs such a sweep on the caller's own
 * index and probes.
 *
 * gi_tune -- times point lookups of the DEVICE probes queries[0..m) under candidate
 *   values of the knobs that apply to the index's layout (GI_OPT_GROUP, PER_THREAD,
 *   BLOCK, BLOCKS_PER_SM, SMEM_LEVELS alone and paired with a persistent grid,
 *   PREFETCH, HOT_LEVELS, EARLY_EXIT, REORDER) by coordinate descent: from the
 *   index's current settings, each knob in turn takes its fastest candidate with the
 *   others held; the sweep repeats until a pass changes nothing (at most 3 passes).
 *   A change is kept only if it is at least 1% faster.  Each timing is one untimed
 *   run and `reps` runs timed with CUDA events on the index's stream, the best kept
 *   (reps = 0: 5).  The knobs change the schedule only, never a lookup's result.
 *   flags: GI_TUNE_APPLY sets the chosen values on the index (otherwise its settings
 *   are restored); GI_TUNE_RECORD stores them in a process-wide table keyed by (key
 *   width, layout, k, floor(log2 n)), from which every index of that class takes
 *   the knobs it leaves automatic (-1).
 *   out (may be NULL): the values on entry and the chosen values, indexed by
 *   GI_OPT_* (-1 where the knob does not apply), and their times.
 *   Allocates m uint32 of device scratch for the call.  Synchronous.
 *   Errors: GI_ERR_INVALID (NULL index, m == 0, host probes, unknown flags),
 *   GI_ERR_NOMEM, GI_ERR_CUDA, GI_ERR_TIMEOUT.  On error the settings are restored.
 * gi_tune_table_get -- the table's entry for (layout | key width, k, n):
 *   options[o], o = 1..10, or -1 where nothing is recorded; *found = 1 if the class
 *   has an entry.  options: 11 int64.
 * gi_tune_table_clear -- empties the table.
 */
#define GI_TUNE_APPLY  1
#define GI_TUNE_RECORD 2
typedef struct gi_tune_result {
  int64_t start_options[11]; /* [GI_OPT_*] on entry; [0] unused (-1)          */
  int64_t options[11];       /* [GI_OPT_*] chosen                             */
  double start_ms;           /* best time of the settings on entry            */
  double best_ms;            /* best time of the chosen settings              */
  uint32_t trials;           /* settings timed                                */
  uint32_t passes;           /* coordinate-descent passes                     */
} gi_tune_result;
int gi_tune(gi_index* index, const void* queries, uint64_t m, uint32_t reps, int flags,
            gi_tune_result* out);
int gi_tune_table_get(int layout, uint32_t k, uint64_t n, int64_t* options, int* found);
void gi_tune_table_clear(void);

/*
 * gi_build_tuned -- picks the layout and k as well (the paper's composite strategy,
 *   Section 9, measured instead of assumed).  Builds the pairs as GI_SORTED,
 *   GI_EYTZINGER and GI_EYTZINGER_KARY with k = 3, 5, 9, 17 in turn (arguments as
 *   gi_build; key_flags = the key width and build flags, no layout), tunes each with
 *   gi_tune on the DEVICE probes queries[0..m) and keeps the index whose best time
 *   is shortest; the others are destroyed as soon as they lose, so at most two
 *   indexes exist at a time.  flags: GI_TUNE_APPLY leaves the winner's knobs set
 *   (otherwise automatic); GI_TUNE_RECORD records its knobs as gi_tune does and its
 *   (layout, k) under (key width, floor(log2 n)) for gi_tune_table_layout.
 *   result (may be NULL): the winner's gi_tune result; gi_get_info gives its layout.
 *   Synchronous.  Errors: as gi_build and gi_tune; *out is NULL on error.
 * gi_tune_table_layout -- the recorded (layout, k) for (key width, n): *found = 1 if
 *   the size class has one (else *layout = -1, *k = 0).
 */
int gi_build_tuned(const void* keys, const uint32_t* rowids, uint64_t n, int key_flags,
                   const void* queries, uint64_t m, uint32_t reps, int flags, gi_index** out,
                   gi_tune_result* result);
int gi_tune_table_layout(int key_flags, uint64_t n, int* layout, uint32_t* k, int* found);

/*
 * gi_probe_random_sectors -- roofline probe: `loads` loads of `chunk_bytes`
 * (16, 32, 64, 128 or 256) contiguous bytes each from uniformly random
 * chunk-aligned offsets of the device buffer `buf` (`bytes` long, 256-byte
 * aligned), many in flight per warp.  With buf much larger than L2 it measures
 * the random-access throughput of HBM.  The XOR of everything loaded goes to
 * *sink (device).  Asynchronous on `stream`.                     (Section 5.1)
 */
int gi_probe_random_sectors(const void* buf, uint64_t bytes, uint32_t chunk_bytes,
                            uint64_t loads, uint64_t seed, uint64_t* sink, void* stream);

/*
 * gi_coalescing_probe -- the micro-benchmark of Section 5.1 / Fig 9: `threads`
 * threads in groups of `group` neighbours; for `steps` steps each group draws a
 * random position p in the uint32 array `buf` (`entries` long) and thread i of the
 * group loads entry p+i.  The XOR of the loads goes to *sink.  Asynchronous.
 */
int gi_coalescing_probe(const uint32_t* buf, uint64_t entries, uint32_t threads,
                        uint32_t group, uint32_t steps, uint64_t seed, uint64_t* sink,
                        void* stream);

/*
 * Batched form: B independent indexes of uneven size, built and probed together.
 * The paper evaluates one index at a time; this form serves many small indexes
 * (e.g. one per partition of a join) with one launch per phase instead of one per
 * index.  Index b holds pairs key_offsets[b] .. key_offsets[b+1]-1 of the
 * concatenated key/rowID arrays.  Layouts: GI_EYTZINGER_KARY with k in
 * {2, 3, 5, 9, 17}, or GI_SORTED, for every index; or a fan-out per index
 * (gi_batch_set_fanouts below); either key width.
 *
 * gi_batch_create -- sizes and allocates all device memory of the batch from the
 *   HOST array key_offsets[B+1] (key_offsets[0] = 0, non-decreasing, each index
 *   below 2^31 keys) and uploads the tile tables.  Synchronous.
 * gi_batch_build -- segmented radix sort of all pairs (no pair leaves its index)
 *   and the per-index closed-form permutation (Sections 4, 6.1).  keys/rowids:
 *   DEVICE memory.  Asynchronous on the batch's stream, no allocation and no host
 *   synchronisation, so it can be captured in a CUDA graph.  Errors found on the
 *   device (reserved rowID, a bounded wait that gave up) come back from gi_batch_sync,
 *   which waits for the batch's stream and reports each such status once (the
 *   status is cleared when it is returned).
 * gi_batch_point_lookup -- one persistent launch over (index, chunk of probes).
 *   queries: DEVICE, m probes; index b's probes are
 *   queries[query_offsets[b] .. query_offsets[b+1]); query_offsets: DEVICE array of
 *   B+1 uint64 with query_offsets[B] = m; out_rowids: DEVICE, m uint32 (rowID or
 *   GI_MISS).  Each CTA pins the top levels of the index it serves in shared memory
 *   (a bulk asynchronous copy; whole small indexes), up to a per-CTA budget.
 *   Asynchronous, no allocation, capturable.
 * gi_batch_copy_index -- copy index b's arrays in layout order (device or host).
 * gi_batch_set_option -- GI_BATCH_OPT_CHUNK (probes per work item, default 2048),
 *   GI_BATCH_OPT_BLOCKS_PER_SM (default 8), GI_BATCH_OPT_SMEM_BUDGET (bytes of
 *   pinned levels per CTA, 0..40960, default 0: no pinning).  The defaults are
 *   gi_batch_tune's choice on 4096 indexes of 2^8..2^20 u64 keys.
 */
typedef struct gi_batch gi_batch;
#define GI_BATCH_OPT_CHUNK         1
#define GI_BATCH_OPT_BLOCKS_PER_SM 2
#define GI_BATCH_OPT_SMEM_BUDGET   3
int gi_batch_create(const uint64_t* key_offsets, uint32_t B, int layout, uint32_t k,
                    gi_batch** out);
int gi_batch_set_stream(gi_batch* batch, void* stream);
int gi_batch_build(gi_batch* batch, const void* keys, const uint32_t* rowids);
int gi_batch_point_lookup(gi_batch* batch, const void* queries, const uint64_t* query_offsets,
                          uint64_t m, uint32_t* out_rowids);
int gi_batch_sync(gi_batch* batch);
int gi_batch_copy_index(const gi_batch* batch, uint32_t i, void* keys_out, uint32_t* rowids_out);
int gi_batch_set_option(gi_batch* batch, int option, int64_t value);
uint64_t gi_batch_footprint_bytes(const gi_batch* batch);
/*
 * gi_batch_tune -- the autotuner for the batched lookup: times
 *   gi_batch_point_lookup(batch, queries, query_offsets, m, .) (arguments as there,
 *   DEVICE memory) under GI_BATCH_OPT_CHUNK, GI_BATCH_OPT_BLOCKS_PER_SM and
 *   GI_BATCH_OPT_SMEM_BUDGET candidates by the coordinate descent of gi_tune, and
 *   leaves the fastest values set on the batch.  out (may be NULL): values on entry
 *   and chosen, indexed by GI_BATCH_OPT_*.  Allocates m uint32 of device scratch.
 *   Synchronous; the batch must be built.  Errors: as gi_batch_point_lookup and
 *   gi_batch_sync; on error the values on entry are restored.
 */
int gi_batch_tune(gi_batch* batch, const void* queries, const uint64_t* query_offsets, uint64_t m,
                  uint32_t reps, gi_tune_result* out);
void gi_batch_destroy(gi_batch* batch);

/*
 * Per-index fan-out.  The paper's composite strategy (Section 9: Eytzinger order
 * while the index fits in L2, k-ary above) is a choice per index size; a batch of
 * indexes of uneven size makes it per index.  Each index of a batch is laid out
 * with its own fan-out k_i: 0 (sorted order, binary search), 2 (Eytzinger order,
 * stored 0-based as the k-ary layout with k = 2), 3, 5, 9 or 17.  The build writes
 * every index in its own order and the lookup's work items dispatch on it; build
 * and lookup stay one launch sequence, free of allocation and host round trips
 * (capturable).
 * gi_batch_set_fanouts -- ks: B host fan-outs, or NULL for the automatic choice
 *   per size class floor(log2 n_i): the one gi_batch_tune_fanouts recorded for the
 *   batch's key width, else k = 3 up to 32 KB of keys and k = 5 above (measured on
 *   a batch of 2^8..2^20 u64 keys per index).  Takes effect at the next
 *   gi_batch_build (the indexes must be built again).  Synchronous (waits for the
 *   batch's stream); call it outside stream capture.
 *   Errors: GI_ERR_INVALID (a fan-out outside the set), GI_ERR_CUDA.
 * gi_batch_get_fanouts -- the B fan-outs in use into ks_out (host).
 * gi_batch_tune_fanouts -- the autotuner for the fan-outs: gathers the probes of
 *   each size class, builds the batch with every candidate fan-out (2, 3, 5, 9, 17)
 *   in turn and times each class's lookups alone (best of `reps`, 0: 5), then picks
 *   per class the fastest.  keys/rowids/queries/query_offsets as in gi_batch_build
 *   and gi_batch_point_lookup (DEVICE memory).  flags: GI_TUNE_APPLY leaves the
 *   chosen fan-outs set, otherwise those on entry; GI_TUNE_RECORD stores the
 *   per-class choice for the automatic choice of later batches with this key
 *   width.  Either way the batch is left built.  ks_out (may be NULL): the chosen
 *   B fan-outs; class_ms (may be NULL): 64 x 5 doubles, the best time of size class
 *   c under candidate j at [c * 5 + j] (-1 where the class has no probes).
 *   Allocates scratch for the call; synchronous.
 * gi_batch_fanout_table_clear -- forget every recorded per-class choice.
 */
int gi_batch_set_fanouts(gi_batch* batch, const uint32_t* ks);
int gi_batch_get_fanouts(const gi_batch* batch, uint32_t* ks_out);
int gi_batch_tune_fanouts(gi_batch* batch, const void* keys, const uint32_t* rowids,
                          const void* queries, const uint64_t* query_offsets, uint64_t m,
                          uint32_t reps, int flags, uint32_t* ks_out, double* class_ms);
void gi_batch_fanout_table_clear(void);

/*
 * Serving form: resident indexes answer a stream of requests with continuous
 * batching.  The paper measures batches of lookups; this form serves requests
 * that arrive at any time from many client threads.
 *
 * gi_server_create -- serve `count` built indexes (same key width, layout and k;
 *   GI_SORTED or GI_EYTZINGER_KARY with k in {3, 5, 9, 17}).  `arena_bytes` of
 *   device memory hold the admitted requests' inputs and results: a request is
 *   admitted, first-in first-out, only when its bytes fit (admission by free
 *   device memory).  Up to `max_inflight` batches run at once, each on its own
 *   stream.  Starts one server thread.  The indexes must outlive the server.
 * gi_server_submit -- queue a request (thread-safe, returns at once with a
 *   ticket).  All buffers are HOST memory: page-locked buffers of requests of
 *   more than 2048 probes or ranges are copied by the copy engine straight from
 *   and to them; the others are gathered on the host into one staging copy per
 *   batch (point results scattered back likewise):
 *     GI_REQ_POINT: keys[m] probes -> out_rowids[m] (rowID or GI_MISS);
 *     GI_REQ_RANGE: keys[m] lower and hi[m] upper bounds (inclusive) ->
 *       out_offsets[m+1] and, when it fits, out_rowids[rows_capacity] in
 *       ascending key order.
 *   A request whose inputs and results exceed the whole arena is refused
 *   (GI_ERR_NOMEM).  Requests that arrive while batches run join the next batch.
 * gi_server_wait -- block until the ticket's request completes; returns its
 *   status.  Ranges whose rows exceed rows_capacity return GI_ERR_CAPACITY with
 *   out_offsets filled (out_offsets[m] is the row count).  Also reports the
 *   submit and completion times (steady clock, ns) for latency figures.
 * gi_server_stats -- batches launched, requests submitted, probes admitted.
 * gi_server_destroy -- finish queued requests, stop the thread, free the server.
 */
typedef struct gi_server gi_server;
#define GI_REQ_POINT 0
#define GI_REQ_RANGE 1
typedef struct gi_request {
  uint32_t index;          /* which served index */
  uint32_t kind;           /* GI_REQ_POINT or GI_REQ_RANGE */
  uint64_t m;              /* probes or ranges, >= 1 */
  const void* keys;        /* probes, or lower bounds */
  const void* hi;          /* upper bounds (ranges) */
  uint32_t* out_rowids;    /* point results, or range rows */
  uint64_t* out_offsets;   /* range CSR offsets, m+1 */
  uint64_t rows_capacity;  /* room in out_rowids for range rows */
} gi_request;
int gi_server_create(gi_index* const* indexes, uint32_t count, uint64_t arena_bytes,
                     uint32_t max_inflight, gi_server** out);
int gi_server_submit(gi_server* server, const gi_request* request, uint64_t* ticket);
int gi_server_wait(gi_server* server, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns);
int gi_server_stats(const gi_server* server, uint64_t* batches, uint64_t* requests,
                    uint64_t* probes);
void gi_server_destroy(gi_server* server);

/*
 * Load generators for the serving form (open loop: arrivals do not wait for
 * completions), so that latency is measured without an interpreter's jitter.
 *   reqs[i] is submitted at arrival_ns[i] nanoseconds (>= 0; any order) after a
 *   common start time set a few milliseconds after the call begins.
 *   latency_ns[i]: completion time minus that scheduled arrival (queueing and
 *   service together), or -1 if the request was not accepted; status[i] (may be
 *   NULL): its return code (GI_ERR_CAPACITY for range rows beyond rows_capacity).
 *   wall_s (may be NULL): seconds from the start time to the last completion.
 *   Returns GI_OK, or the first failure other than GI_ERR_CAPACITY.
 * gi_server_replay -- `threads` native threads (1..64) submit to the server,
 *   request i by thread i mod threads; this thread collects the completions.
 *   Latencies come from the server's completion times (gi_server_wait).
 * gi_replay_serial -- the baseline without the server: one thread takes the
 *   requests in index order, each at its arrival time or as soon as the previous
 *   one is done, through gi_point_lookup / gi_range_lookup on indexes[reqs[i].index]
 *   with the request's host buffers (ranges by the two-call protocol: offsets,
 *   then rows if they fit rows_capacity).
 */
int gi_server_replay(gi_server* server, const gi_request* reqs, const int64_t* arrival_ns,
                     uint64_t count, uint32_t threads, int64_t* latency_ns, int* status,
                     double* wall_s);
int gi_replay_serial(gi_index* const* indexes, uint32_t nindexes, const gi_request* reqs,
                     const int64_t* arrival_ns, uint64_t count, int64_t* latency_ns, int* status,
                     double* wall_s);

/*
 * gi_range_lookup_noalloc -- gi_range_lookup for callers that must not allocate.
 * The paper has no counterpart: this entry point exists for users whose device
 * memory is owned by someone else (a query engine or framework that hands the
 * whole GPU to its own pool allocator) or who cannot afford an allocation call
 * in the middle of a query (cudaMalloc/cudaFree can block or synchronise the
 * device).  It computes exactly what gi_range_lookup computes, but its scratch
 * (the lower rank of every range and the scan's block sums) lives in one
 * fixed-size array inside the library, so it calls no allocator at all.
 *   m            at most GI_NOALLOC_MAX_RANGES ranges; more returns GI_ERR_INVALID.
 *   lo, hi, out_offsets, out_rowids
 *                as in gi_range_lookup, but all must be DEVICE memory (staging
 *                host memory would need an allocation): host pointers return
 *                GI_ERR_INVALID.  out_rowids may be NULL (offsets only).
 * The array is a static device variable of GI_NOALLOC_SCRATCH_BYTES bytes that
 * every GPU which loads this library holds until the process exits.  The first
 * call on a device looks up the array's device address on that device (a
 * cudaGetSymbolAddress call, made with the index's device current); make that
 * first call before any stream capture.  Every call on a device shares the one
 * array and leaves its contents behind (nothing in it needs to start zeroed):
 * calls whose GPU work overlaps -- on different streams, or from different
 * threads -- race on it and must be serialised by the caller.  Asynchronous on
 * the index's stream, like gi_range_lookup with device pointers.
 */
#define GI_NOALLOC_MAX_RANGES (1u << 20)
#define GI_NOALLOC_SCRATCH_BYTES ((8u << 20) + 8192u)
int gi_range_lookup_noalloc(const gi_index* index, const void* lo, const void* hi, uint64_t m,
                            uint64_t* out_offsets, uint32_t* out_rowids);

/* Number of kernels this library has launched in the process so far. */
uint64_t gi_launch_count(void);

/*
 * gi_debug_fail_alloc -- test hook for out-of-memory handling without exhausting a
 *   shared GPU: after `after` more successful device allocations made through the
 *   library's index paths (build buffers, sort scratch, range scratch, host-memory
 *   staging), the next one reports cudaErrorMemoryAllocation without allocating, and
 *   the hook disarms.  The failing call returns GI_ERR_NOMEM having freed what it had
 *   allocated; the library stays usable.  after < 0 disarms.  Process-wide.
 */
void gi_debug_fail_alloc(int64_t after);

#ifdef __cplusplus
}
#endif
#endif /* GI_H_ */
