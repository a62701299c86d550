/*
 * ipmerge — GB300 (sm_103a) parallel in-place merge.
 *
 * C ABI of the data-parallel hot path of B. Bramas, Q. Bramas, "On the improvement of
 * the in-place merge algorithm parallelization" (arXiv 2005.12648):
 *
 *   1. split      exact stable merge-path split points (the optimal split of Sec. 3.1)
 *                 on the diagonals d_k = floor(k*n/P), k = 0..P, n = len_a + len_b;
 *   2. rearrange  the sRecPar division stage (Alg. 3): level by level, the two middle
 *                 blocks of every pair are exchanged in place (the partition exchange of
 *                 Sec. 3.4), giving A_0 B_0 A_1 B_1 ... A_{P-1} B_{P-1}; or the same
 *                 layout by one permutation along its cycles (sOptMov, Alg. 2);
 *   3. merge      every pair (A_k, B_k) is merged stably in place (the per-thread merge
 *                 of Alg. 2/3, here one CTA per pair, staged in shared memory).
 *
 * Conventions for every entry point:
 *   - Device pointers are plain CUDA device addresses, owned by the caller.  The
 *     library never allocates or frees device memory; every call that needs scratch
 *     takes a caller-owned workspace sized by the matching *_workspace_bytes query.
 *   - Lengths and offsets count elements, not bytes.
 *   - Merge calls must not run concurrently with each other on different streams: their
 *     persistent kernels size their grids to the whole GPU and their group barriers need
 *     their own CTAs resident (order such calls with events; copies may overlap them).
 *   - Keys are compared with the key type's own "<=": signed for IPM_INT32 /
 *     IPM_INT64, unsigned for IPM_UINT32 / IPM_UINT64, IEEE for IPM_FLOAT32 (NaN keys
 *     are not allowed;
 *     -0.0 and +0.0 compare equal and keep their input order).
 *   - The merge is stable: equal keys keep their input order, every A element before
 *     every equal B element.  Keys (and payloads) are only moved, never computed, so
 *     the result is bit-exact.
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream), except
 *     the ipm_read_* queries and ipm_rearrange_permute, which synchronise the stream,
 *     and ipm_timing_read, which waits for the recorded events.
 *     Argument errors detectable on the host return immediately and launch nothing.  Errors
 *     found on the device (a bounded wait that expired) are recorded in the status
 *     word at the start of the workspace, read with ipm_read_device_status.
 *   - Preconditions that are not checked: both runs are sorted under the comparison
 *     above, the buffer holds len_a + len_b elements, and no other work touches the
 *     buffer or the workspace while the call runs on the stream.
 */
#ifndef IPMERGE_H
#define IPMERGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The same type as cudaStream_t. */
typedef struct CUstream_st *ipm_stream_t;

typedef enum {
    IPM_OK = 0,
    IPM_ERR_INVALID_ARG = 1,       /* NULL pointer, size overflow, bad option */
    IPM_ERR_UNSUPPORTED_DTYPE = 2, /* dtype not in ipm_dtype / not allowed here */
    IPM_ERR_ALIGNMENT = 3,         /* pointer not aligned to its element size */
    IPM_ERR_WORKSPACE = 4,         /* workspace NULL or smaller than required */
    IPM_ERR_CUDA = 5,              /* a CUDA runtime call or launch failed */
    IPM_ERR_TIMEOUT = 6,           /* a bounded device-side wait expired */
    IPM_ERR_DEVICE = 7             /* the device found an inconsistent state; or (no-alloc
                                      merge) the buffer or stream is not on the current
                                      device */
} ipm_status;

typedef enum {
    IPM_INT32 = 0,
    IPM_UINT32 = 1,
    IPM_UINT64 = 2,
    IPM_FLOAT32 = 3,
    IPM_INT64 = 4
} ipm_dtype;

/* Human-readable name of a status code (static string). */
const char *ipm_status_string(ipm_status s);

/* Library version as major*10000 + minor*100 + patch. */
int ipm_version(void);

/*
 * Number of pairs P = 2^log2_pairs the plain merge uses for n = len_a + len_b keys of
 * this dtype (the smallest power of two whose pairs all fit one CTA's shared-memory
 * tile), and that tile's capacity in elements.  with_values is the payload width:
 * 0 keys only, 1 or 4 a 4-byte payload, 8 an 8-byte payload (other values:
 * IPM_ERR_UNSUPPORTED_DTYPE).  Either output pointer may be NULL.
 */
ipm_status ipm_merge_plan(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                          int with_values, uint32_t *log2_pairs, uint64_t *tile_capacity);

/*
 * Workspace bytes for ipm_merge_inplace / _kv with this size, dtype, payload width
 * (with_values as for ipm_merge_plan) and pair count (log2_pairs = 0 picks the
 * automatic count of ipm_merge_plan).  The size is O(P):
 * the split table, the per-level exchange plans and a 256-byte status block.
 */
ipm_status ipm_merge_workspace_bytes(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                                     int with_values, uint32_t log2_pairs, size_t *bytes);

/*
 * Stable in-place merge of the two sorted runs A = d_buf[0, len_a) and
 * B = d_buf[len_a, len_a + len_b) into one sorted run d_buf[0, len_a + len_b)
 * (Sec. 1 problem statement; division stage Alg. 3; exchange Sec. 3.4).
 *   d_buf      device pointer to len_a + len_b keys of key_dtype, aligned to the key
 *              size; overwritten with the merged run.
 *   log2_pairs 0 = automatic; otherwise P = 2^log2_pairs pairs (every pair must fit
 *              the tile capacity, else IPM_ERR_INVALID_ARG).
 *   d_ws       workspace of at least ipm_merge_workspace_bytes(...) bytes, 256-byte
 *              aligned, used for the duration of the call on `stream`.
 * If A is empty, B is empty, or A[last] <= B[0] (the early exit of Alg. 2/3), the
 * buffer is left as it is.
 */
ipm_status ipm_merge_inplace(void *d_buf, uint64_t len_a, uint64_t len_b,
                             ipm_dtype key_dtype, uint32_t log2_pairs, void *d_ws,
                             size_t ws_bytes, ipm_stream_t stream);

/*
 * Key-value form of ipm_merge_inplace: the payload d_vals[t] moves with the key
 * d_keys[t] (structure of arrays).  Payloads are never compared; val_dtype only gives
 * their width: a 4-byte type (IPM_UINT32, IPM_INT32, IPM_FLOAT32) or an 8-byte type
 * (IPM_UINT64, IPM_INT64; any 8-byte record can be passed as IPM_UINT64).  d_vals is
 * aligned to that width.  The workspace comes from ipm_merge_workspace_bytes with
 * with_values = the payload width.  Key-value tiles hold fewer elements (the
 * shared-memory tile is shared by keys and payloads), so more pairs are used.
 */
ipm_status ipm_merge_inplace_kv(void *d_keys, void *d_vals, uint64_t len_a,
                                uint64_t len_b, ipm_dtype key_dtype, ipm_dtype val_dtype,
                                uint32_t log2_pairs, void *d_ws, size_t ws_bytes,
                                ipm_stream_t stream);

/*
 * Step 1 alone: the exact stable split on every diagonal d_k = floor(k*n/P),
 * k = 0..P (P = num_pairs >= 1, n = len_a + len_b, num_pairs * n < 2^64).
 * d_split_a[k] receives i_k, the number of A elements among the first d_k keys of the
 * stable merge; the B count is d_k - i_k.  d_split_a holds num_pairs + 1 uint64.
 * This is the "optimal" split of Sec. 3.1 / Fig. 5, evaluated by a warp-cooperative
 * binary search on each diagonal.  The input buffer is only read.
 */
ipm_status ipm_merge_splits(const void *d_buf, uint64_t len_a, uint64_t len_b,
                            ipm_dtype key_dtype, uint64_t num_pairs, uint64_t *d_split_a,
                            ipm_stream_t stream);

/*
 * The division of Alg. 3 (sRecPar, Sec. 3.3) to 2^depth pairs without moving data,
 * for the balance comparison of Sec. 4 between FindMedian (Alg. 1, Sec. 3.1) and the
 * optimal split.  Level by level (depth levels), every region
 * A[d_ia[k0], d_ia[k1]) | B[d_jb[k0], d_jb[k1]) is cut at its pivot (pA, pB):
 *   IPM_SPLIT_EXACT       the exact stable split at the region's half diagonal
 *                         floor(c/2) (the optimal balance);
 *   IPM_SPLIT_FINDMEDIAN  FindMedian, read as: both corner cases first (A before B:
 *                         (|A|, 0); A after B: (0, |B|)); the midpoints recomputed at the
 *                         top of each iteration and returned when their keys are equal;
 *                         the midpoints of the final intervals when one empties.
 * A region with an empty side is not divided (Alg. 3 stops there): it stays whole in
 * its left child and the right child is empty.  d_ia and d_jb (device, caller-owned)
 * receive 2^depth + 1 boundaries each: pair k is A[d_ia[k], d_ia[k+1]) with
 * B[d_jb[k], d_jb[k+1]).  d_buf = A|B is only read.  depth <= 24.  One launch per
 * level, asynchronous on `stream`.  Errors: IPM_ERR_INVALID_ARG (NULL pointers, depth,
 * split_kind), IPM_ERR_UNSUPPORTED_DTYPE, IPM_ERR_ALIGNMENT (d_buf not aligned to the
 * key size, d_ia / d_jb not 8-byte aligned), IPM_ERR_CUDA.
 */
#define IPM_SPLIT_EXACT 0u
#define IPM_SPLIT_FINDMEDIAN 1u
ipm_status ipm_division_splits(const void *d_buf, uint64_t len_a, uint64_t len_b,
                               ipm_dtype key_dtype, uint32_t depth, uint32_t split_kind,
                               uint64_t *d_ia, uint64_t *d_jb, ipm_stream_t stream);

/*
 * Step 2 alone: the division stage of Alg. 3 applied to d_buf from a split table made
 * by ipm_merge_splits with P = 2^log2_pairs.  Afterwards pair k occupies
 * d_buf[d_k, d_{k+1}) as A[i_k, i_{k+1}) followed by B[j_k, j_{k+1}).  d_vals may be
 * NULL (keys only) or a uint32 payload array moved with the keys.  The workspace is
 * the one of ipm_merge_workspace_bytes for the same arguments; the split table is
 * read from d_split_a (not from the workspace).
 */
ipm_status ipm_merge_rearrange(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                               ipm_dtype key_dtype, const uint64_t *d_split_a,
                               uint32_t log2_pairs, void *d_ws, size_t ws_bytes,
                               ipm_stream_t stream);

/*
 * Step 2 by one permutation (sOptMov, Alg. 2, Sec. 3.2): the same layout as
 * ipm_merge_rearrange (pair k at d_buf[d_k, d_{k+1}) as A[i_k, i_{k+1}) followed by
 * B[j_k, j_{k+1}), d_k = floor(k*n/2^log2_pairs), j_k = d_k - i_k), reached by moving
 * every element once along the cycles of that permutation instead of level by level.
 * d_split_a (device, 2^log2_pairs + 1 uint64, read only) is any table with i_0 = 0,
 * i_P = len_a and, for every k, i_k <= i_{k+1}, i_{k+1} - i_k <= d_{k+1} - d_k,
 * i_k <= d_k and d_{k+1} - i_{k+1} <= len_b (ipm_merge_splits makes one).  The paper's
 * in-value marker of moved elements is replaced by a bitmap of n bits in the workspace,
 * so keys of every type keep their full range.  with_values is the payload width as in
 * ipm_merge_plan (0: d_vals must be NULL; 1 or 4: uint32; 8: uint64), moved with the
 * keys.  The workspace (ipm_rearrange_permute_workspace_bytes for the same sizes, type
 * and payload; 256-byte aligned) holds the bitmap and the elements saved per round,
 * about n/8 + (n/31) * (key + payload + 8) bytes.  The call blocks the host thread: it
 * runs rounds on `stream` and reads the uncovered count back after each (at most 32
 * rounds).  Errors: IPM_ERR_INVALID_ARG (NULL pointers, d_vals not matching
 * with_values, log2_pairs > 22, len_a or len_b > 2^40, or a table that is not of the
 * form above: detected on the device before any element moves), IPM_ERR_ALIGNMENT
 * (d_buf / d_vals not aligned to their element size, d_split_a not 8-byte aligned,
 * d_ws not 256-byte aligned), IPM_ERR_WORKSPACE, IPM_ERR_UNSUPPORTED_DTYPE,
 * IPM_ERR_CUDA, IPM_ERR_DEVICE (an internal consistency check failed).
 */
ipm_status ipm_rearrange_permute_workspace_bytes(uint64_t len_a, uint64_t len_b,
                                                 ipm_dtype key_dtype, int with_values,
                                                 size_t *bytes);
ipm_status ipm_rearrange_permute(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                                 ipm_dtype key_dtype, int with_values,
                                 const uint64_t *d_split_a, uint32_t log2_pairs, void *d_ws,
                                 size_t ws_bytes, ipm_stream_t stream);

/*
 * Step 3 alone: merge every pair of an arranged buffer (the layout step 2 produces)
 * in place, one CTA per pair through shared memory.  d_split_a is the P+1 split table
 * (P = 2^log2_pairs); every pair must fit the tile capacity.  d_vals as above.
 */
ipm_status ipm_merge_pairs(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                           ipm_dtype key_dtype, const uint64_t *d_split_a,
                           uint32_t log2_pairs, ipm_stream_t stream);

/*
 * Partition exchange alone (Sec. 3.4): d_ptr[0, len_x + len_y) = [X | Y] becomes
 * [Y | X] in place.  elem_bytes is 4 or 8 (the bytes are moved, never compared).
 * Executed as linear shifting: LS block swaps while both the size difference and the
 * smaller block are larger than the on-chip stash, then the remaining LS steps in
 * closed form in one pass (every element read and written once).  The workspace size
 * comes from ipm_rotate_workspace_bytes for the same sizes.
 */
ipm_status ipm_rotate_workspace_bytes(uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                                      size_t *bytes);
ipm_status ipm_rotate(void *d_ptr, uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                      void *d_ws, size_t ws_bytes, ipm_stream_t stream);

/*
 * The same exchange by circular shifting (Sec. 3.4, with the cycle count of its proof
 * of correctness: gcd(len_x, len_y) cycles): every position x takes the element at
 * (x + len_x) mod n, followed cycle by cycle; cycles longer than a worker's share are
 * cut into segments that run concurrently (a first launch saves each segment's first
 * value).  Every element is read once and written once; accesses coalesce only when
 * the cycle count is >= 32, so this is the comparison point for ipm_rotate, not the
 * path the merge uses.  elem_bytes is 4 or 8.  The workspace (status block + at most
 * 2^19 saved elements, <= 4 MiB + 256 B) comes from ipm_rotate_cs_workspace_bytes for
 * the same sizes; d_ptr must be elem_bytes-aligned, d_ws 256-byte aligned.  Errors:
 * IPM_ERR_INVALID_ARG (NULL pointer, a length above 2^40), IPM_ERR_UNSUPPORTED_DTYPE
 * (elem_bytes), IPM_ERR_WORKSPACE, IPM_ERR_ALIGNMENT, IPM_ERR_CUDA (launch failure).
 * len_x = 0 or len_y = 0 returns IPM_OK without touching the device.
 */
ipm_status ipm_rotate_cs_workspace_bytes(uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                                         size_t *bytes);
ipm_status ipm_rotate_cs(void *d_ptr, uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                         void *d_ws, size_t ws_bytes, ipm_stream_t stream);

/*
 * Algorithmic bytes the exchange levels of the last merge (or rotate) that used this
 * workspace moved (the levels that ran as exchanges; fused bottom levels move their
 * data in the pair merge instead): 2 bytes-per-element for every element of a
 * one-pass exchange, 4 per swapped pair of an LS block swap.  Synchronises `stream`.
 */
ipm_status ipm_read_exchange_bytes(const void *d_ws, ipm_stream_t stream, uint64_t *out);

/*
 * How many of the last levels of the division stage the merge entry points fuse with
 * the pair merge (process-wide, default 10: as many as the engine can, 8 or 9 on a
 * 152-SM GB300).  With F fused levels the exchange levels
 * stop F levels short, and each group of 2^F consecutive pairs is finished by 2^F CTAs
 * together: the group's region holds exactly those pairs' A and B slices, so each CTA
 * stages its pair's two slices, the group synchronises once the whole group has been
 * read, and each pair is merged on chip and written to its final place.  The fused path
 * uses half-size tiles (two CTAs per SM) and splits one level deeper.  The result is
 * identical for every F; F trades exchange passes over the buffer for group size.
 * 0 <= levels <= 10 (the device may lower it: a group needs at most the resident CTAs,
 * a thread-block cluster at most 16), else IPM_ERR_INVALID_ARG.  Not thread-safe
 * against concurrent merge calls.
 *
 * ipm_set_fused_engine selects how a group synchronises: 0 = one thread-block cluster
 * per group (cluster barrier; F <= 4), 1 = CTAs taken from a ticket in order and a
 * group barrier in global memory, 2 = two pairs per CTA, the first merged pair parked
 * in tensor memory (TMEM), each pair written once the pairs that read its destination
 * have their slices on chip (a per-pair count in global memory instead of the whole
 * group), which fuses one level more (the default, for every key type with or without
 * payload).
 * ipm_merge_fused_plan reports what a merge will use.
 */
/*
 * The fused engine (0, 1, 2 as above; 0xFFFFFFFF when no level is fused) and the number
 * of fused levels ipm_merge_inplace / _kv would use for these sizes, key type and payload
 * width (with_values as for ipm_merge_plan) under the current settings and device.
 * Either output may be NULL.  Host only (queries the device's occupancy once).
 */
ipm_status ipm_merge_fused_plan(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                                int with_values, uint32_t *engine, uint32_t *levels);
ipm_status ipm_set_fused_levels(uint32_t levels);
ipm_status ipm_get_fused_levels(uint32_t *levels);
ipm_status ipm_set_fused_engine(uint32_t engine);

/*
 * Executor of the exchange levels (process-wide): 0 = every thread of a CTA takes
 * every role in turn (claim, decode, stage, wait, store); 1 = warp-specialized (one
 * producer warp claims, decodes and stages items while 15 consumer warps store the
 * previous one; the default).  Both produce the same result; else
 * IPM_ERR_INVALID_ARG.
 */
ipm_status ipm_set_exchange_engine(uint32_t engine);

/*
 * Limit, in nanoseconds of GPU wall time, of the waits in which a CTA of a merge call
 * waits for another CTA's progress: the "reads done" flags and step joins of the
 * exchange levels (Sec. 3.4 executed by many CTAs) and the group barrier of the fused
 * bottom levels.  Process-wide, read when a merge call (ipm_merge_inplace, _kv,
 * _learned, _noalloc) is issued; 0 restores the default of 2 s; at most 2 s, else
 * IPM_ERR_INVALID_ARG.  When such a wait runs out, the kernel records IPM_ERR_TIMEOUT in
 * the call's status word (ipm_read_device_status) and leaves without finishing its
 * work, the call's later kernels skip theirs, and the buffer's contents are
 * unspecified; the device stays usable.  Waits for a CTA's own bulk copies
 * always keep the 2 s limit, so no copy into a CTA's shared memory is in flight when it
 * leaves.  A short limit exists to test this path; normal use keeps the default.
 * ipm_get_wait_limit_ns reports the limit in effect.
 */
ipm_status ipm_set_wait_limit_ns(uint64_t ns);
ipm_status ipm_get_wait_limit_ns(uint64_t *ns);

/*
 * Batched segmented merge: many independent in-place merges in one call.
 * Segment t of the table is the problem of Sec. 1 on its own slice of the buffer:
 * A = d_buf[offset, offset + len_a) and B = d_buf[offset + len_a, offset + len_a +
 * len_b), both sorted, merged stably in place.  Offsets and lengths count elements.
 */
typedef struct {
    uint64_t offset;
    uint64_t len_a;
    uint64_t len_b;
} ipm_segment;

/*
 * Launch options of ipm_merge_batched (a NULL options pointer = all zero):
 *   tile         0 = library default (2), 1 = wide tile (the plain merge's tile, one
 *                CTA per SM), 2 = narrow tile (half of it, two CTAs per SM),
 *                3 = quarter tile (four CTAs per SM);
 *   ctas_per_sm  0 = as many as fit, else at most this many resident CTAs per SM;
 *   order        0 = work queue in segment-size order, largest first; 1 = table order;
 *   form         0 = library default (1), 1 = three launches (queue preparation by one
 *                CTA, then the exchange levels of every long segment, then the pair
 *                merges), 2 = one launch (a memset node clears the call's counters, then
 *                one persistent kernel prepares the queue with many CTAs and does each
 *                segment whole: early exit, splits, exchange levels, pair merges).
 * Every option changes only the speed, never the result.
 */
typedef struct {
    uint32_t tile;
    uint32_t ctas_per_sm;
    uint32_t order;
    uint32_t form;
} ipm_batched_options;

/*
 * Workspace bytes of ipm_merge_batched for a buffer of buf_len elements, a table of
 * nseg segments, this dtype, payload choice and options: O(nseg + buf_len / tile) (the
 * queue and the split tables of the segments longer than one tile).
 */
ipm_status ipm_merge_batched_workspace_bytes(uint64_t buf_len, uint32_t nseg,
                                            ipm_dtype key_dtype, int with_values,
                                            const ipm_batched_options *opt, size_t *bytes);

/*
 * Longest segment (len_a + len_b, elements) ipm_merge_batched accepts for this dtype,
 * payload choice and options: 512 tiles of the chosen tile size.  Longer segments are skipped on the device
 * (status IPM_ERR_INVALID_ARG); merge them with ipm_merge_inplace instead.
 */
ipm_status ipm_merge_batched_max_segment(ipm_dtype key_dtype, int with_values,
                                         const ipm_batched_options *opt, uint64_t *elems);

/*
 * Merge every segment of d_segs (nseg entries, device memory) in place.
 *   d_buf     device keys, buf_len elements, aligned to the key size.
 *   d_vals    NULL, or a uint32 payload array of buf_len elements moved with the keys
 *             (val_dtype IPM_UINT32; ignored when d_vals is NULL).
 *   d_segs    device array of nseg ipm_segment, 8-byte aligned; the segments must not
 *             overlap (overlapping segments give an unspecified result, but every
 *             access stays inside [0, buf_len)).
 *   d_ws      workspace of ipm_merge_batched_workspace_bytes(buf_len, nseg, ...) bytes
 *             (same dtype, payload choice and options), 256-byte aligned.
 * Every segment is handled by one CTA at a time: the early exit of Alg. 2/3, then (when
 * it is longer than one tile) its exact splits and its sRecPar exchange levels
 * (Alg. 3, Sec. 3.4) in a first persistent launch, and its pair merges in a second;
 * a segment that fits one tile is merged directly.  CTAs take segments from atomic
 * work queues.  A segment that leaves the buffer or is longer than
 * ipm_merge_batched_max_segment is left untouched and the device status becomes
 * IPM_ERR_INVALID_ARG (ipm_read_device_status).  The call launches three kernels
 * (queue preparation, levels, merge), or in the one-launch form a memset node and one
 * kernel; it performs no host synchronisation and no allocation, so it can be captured
 * in a CUDA graph.
 */
ipm_status ipm_merge_batched(void *d_buf, void *d_vals, uint64_t buf_len,
                             const ipm_segment *d_segs, uint32_t nseg, ipm_dtype key_dtype,
                             ipm_dtype val_dtype, const ipm_batched_options *opt,
                             void *d_ws, size_t ws_bytes, ipm_stream_t stream);

/*
 * Autotuner of ipm_merge_batched.  The paper has no counterpart: every option set gives
 * the same result, and the tuner picks the fastest for a given segment table.  It times
 * each candidate (both launch forms; the three merge tiles, which also fix the pair
 * count P = 2^G of every segment longer than one tile; full and reduced resident CTAs
 * per SM; both queue orders; IPM_TUNE_MAX_CANDIDATES at most) and the defaults, each as
 * the median of
 * `reps` runs (1 <= reps <= 100) after one warm-up run, with CUDA events on `stream`.
 * Every run first restores d_scratch (and d_scratch_vals) from d_buf (and d_vals), so
 * the caller's input is only read; the scratch buffers hold buf_len elements each and
 * end up merged.  d_ws holds ipm_merge_batched_tune_workspace_bytes(...) bytes.
 *
 * Cache: the choice is stored under a signature of the workload (key type, payload
 * width, and floor(log2) of the segment count, of the total length, of the longest and
 * of the median segment; ipm_batched_tune_signature computes it from a host copy of the
 * table) in a text file: cache_path, or when cache_path is NULL the file named by the
 * environment variable IPM_TUNE_CACHE, or no cache when neither is set (an empty string
 * disables it too).  A signature found there is returned without timing anything
 * (from_cache = 1; with h_segs given, without any CUDA call).  h_segs is an optional host
 * copy of the table; when NULL the table is copied from d_segs.  The call synchronises
 * `stream` and blocks the host thread while it times.  Errors: IPM_ERR_INVALID_ARG (NULL
 * out, reps, a scratch pointer missing, or no option set that merges every segment),
 * IPM_ERR_UNSUPPORTED_DTYPE (payloads other than IPM_UINT32), IPM_ERR_WORKSPACE, and the
 * errors of ipm_merge_batched.
 */
#define IPM_TUNE_MAX_CANDIDATES 32
typedef struct {
    ipm_batched_options options;
    float ms;       /* median time of the candidate */
    uint32_t pad;
} ipm_batched_tune_entry;

typedef struct {
    ipm_batched_options best;  /* the fastest option set (from the cache: the stored one) */
    float best_ms;             /* its median time (from the cache: the stored time) */
    float default_ms;          /* the defaults' median time; negative when not timed or
                                  when the defaults refuse a segment of the table */
    uint32_t candidates;       /* option sets timed (0 when the cache answered) */
    uint32_t from_cache;       /* 1: read from the cache file, nothing timed */
    uint64_t signature;        /* the workload's cache key */
    ipm_batched_tune_entry table[IPM_TUNE_MAX_CANDIDATES];  /* every timed candidate */
} ipm_batched_tune_result;

ipm_status ipm_merge_batched_tune_workspace_bytes(uint64_t buf_len, uint32_t nseg,
                                                  ipm_dtype key_dtype, int with_values,
                                                  size_t *bytes);
ipm_status ipm_batched_tune_signature(const ipm_segment *h_segs, uint32_t nseg,
                                      ipm_dtype key_dtype, int with_values, uint64_t *out);
ipm_status ipm_merge_batched_tune(const void *d_buf, const void *d_vals, uint64_t buf_len,
                                  const ipm_segment *d_segs, const ipm_segment *h_segs,
                                  uint32_t nseg, ipm_dtype key_dtype, ipm_dtype val_dtype,
                                  void *d_scratch, void *d_scratch_vals, void *d_ws,
                                  size_t ws_bytes, uint32_t reps, const char *cache_path,
                                  ipm_batched_tune_result *out, ipm_stream_t stream);

/*
 * Algorithmic bytes the pair merges of the last batched call that used this workspace
 * moved: 2 bytes-per-element for every element of a segment that was merged (segments
 * that took the early exit move nothing).  Synchronises `stream`.
 */
ipm_status ipm_read_merge_bytes(const void *d_ws, ipm_stream_t stream, uint64_t *out);

/*
 * Learned split proposer.  The paper has no counterpart: it extends the split step
 * (Sec. 3.1), whose cost is the chain of dependent probes of each diagonal's search.
 * A small model predicts the split of a diagonal from its position; a warp then
 * corrects the proposal to the exact split with one round of exponentially spaced
 * probes around it (galloping) followed by the bracket search of ipm_merge_splits, so
 * the result is always the exact split, only the number of dependent probe rounds
 * changes.
 *
 * Model: y(x) = b2 + sum_h w2[h] * tanh(w1[h] * x + b1[h]), h < 32, FP32, with input
 * x = d / n (the diagonal's relative position) and target y = i / len_a (the split's
 * relative position in A); the proposal for diagonal d is round(y * len_a) clamped to
 * the diagonal's range.  The struct lives in DEVICE memory, owned by the caller.
 */
#define IPM_SPLIT_MODEL_HIDDEN 32
typedef struct {
    float w1[IPM_SPLIT_MODEL_HIDDEN];
    float b1[IPM_SPLIT_MODEL_HIDDEN];
    float w2[IPM_SPLIT_MODEL_HIDDEN];
    float b2;
    float loss;      /* mean squared error on the training samples after training */
    uint32_t steps;  /* Adam steps taken by the last ipm_split_model_train */
    uint32_t reserved;
} ipm_split_model;

/* Adam hyper-parameters of ipm_split_model_train (Kingma & Ba). */
typedef struct {
    uint32_t steps;  /* full-batch Adam steps */
    float lr;        /* learning rate */
    float beta1, beta2, eps;
} ipm_split_train_options;

/* Device counters of a learned (or plain) split pass, accumulated by ipm_merge_splits_learned. */
typedef struct {
    uint64_t diagonals;    /* diagonals searched */
    uint64_t rounds;       /* dependent probe rounds, summed over diagonals */
    uint64_t probes;       /* predicate evaluations, summed over diagonals */
    uint64_t abs_err_sum;  /* sum of |proposal - exact split| (0 without a model) */
    uint64_t abs_err_max;  /* max of |proposal - exact split| */
} ipm_split_stats;

/* Workspace bytes of ipm_split_model_train for nsamples training diagonals. */
ipm_status ipm_split_model_train_workspace_bytes(uint32_t nsamples, size_t *bytes);

/*
 * Train d_model in place on the runs A = d_buf[0, len_a), B = d_buf[len_a, len_a +
 * len_b): the exact split of each of the nsamples diagonals d_diags[s] (uint64, device,
 * 0 <= d <= len_a + len_b) is computed on the device (as ipm_merge_splits does) and
 * becomes the target t_s = i_s / len_a for the input x_s = d_s / n; then opt->steps
 * full-batch Adam steps minimise the mean squared error, starting from the parameters
 * d_model holds on entry (Adam moments start at zero).  One CTA runs every step, so the
 * call is a fixed number of launches.  len_a >= 1, 1 <= nsamples <= 2^20.
 */
ipm_status ipm_split_model_train(const void *d_buf, uint64_t len_a, uint64_t len_b,
                                 ipm_dtype key_dtype, const uint64_t *d_diags,
                                 uint32_t nsamples, const ipm_split_train_options *opt,
                                 ipm_split_model *d_model, void *d_ws, size_t ws_bytes,
                                 ipm_stream_t stream);

/*
 * The model's FP32 forward pass (d_y[s] = y(d_x[s])) and its mean-squared-error loss
 * and gradient on (d_x, d_t): d_grad receives the 97 gradient entries in the order
 * w1, b1, w2, b2, then the loss (98 floats).  These are the device functions the
 * training uses, exposed for checking.  All arrays are device float arrays of n.
 */
ipm_status ipm_split_model_forward(const ipm_split_model *d_model, const float *d_x,
                                   uint32_t n, float *d_y, ipm_stream_t stream);
ipm_status ipm_split_model_loss_grad(const ipm_split_model *d_model, const float *d_x,
                                     const float *d_t, uint32_t n, float *d_grad,
                                     ipm_stream_t stream);

/*
 * ipm_merge_splits with proposals: the same exact splits d_split_a[k] on the diagonals
 * d_k = floor(k*n/P), k = 0..P, found by galloping from the model's proposal.
 * d_model may be NULL (no proposal: the plain bracket search, for comparison).
 * d_stats (nullable, device, zeroed by the caller) accumulates the probe counts.
 */
ipm_status ipm_merge_splits_learned(const void *d_buf, uint64_t len_a, uint64_t len_b,
                                    ipm_dtype key_dtype, uint64_t num_pairs,
                                    const ipm_split_model *d_model, uint64_t *d_split_a,
                                    ipm_split_stats *d_stats, ipm_stream_t stream);

/*
 * ipm_merge_inplace with the split step of ipm_merge_splits_learned (same workspace,
 * same result, bit for bit).
 */
ipm_status ipm_merge_inplace_learned(void *d_buf, uint64_t len_a, uint64_t len_b,
                                     ipm_dtype key_dtype, uint32_t log2_pairs,
                                     const ipm_split_model *d_model, void *d_ws,
                                     size_t ws_bytes, ipm_stream_t stream);

/*
 * ipm_merge_inplace for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the same merge.
 * Some callers cannot call cudaMalloc (another framework holds nearly all device
 * memory in its own pool; a latency-critical path cannot afford an allocation and the
 * synchronisation of a later cudaFree; a plain C caller has no allocator to borrow).
 * This entry point takes no workspace: its scratch is an 8 MiB array compiled into the
 * library, which every GPU that loads the library keeps until the process exits.
 *   - Limit: at most 2^15 pairs, i.e. len_a + len_b <= 2^15 * tile capacity
 *     (~1.1e9 4-byte keys, ~5.5e8 8-byte keys).  Larger inputs return
 *     IPM_ERR_INVALID_ARG before anything is launched.  Keys only (no payload).
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   - The first call on each device looks up the array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - Every call shares the one array.  The merge re-initialises what must start at
 *     zero on every call, but calls that overlap on the GPU (e.g. on two streams
 *     without ordering between them) race on it: order them.
 * Same arguments, result and asynchrony as ipm_merge_inplace otherwise.
 */
ipm_status ipm_merge_inplace_noalloc(void *d_buf, uint64_t len_a, uint64_t len_b,
                                     ipm_dtype key_dtype, ipm_stream_t stream);

/*
 * Device rule and status of ipm_merge_inplace_noalloc.  The array exists once per
 * device, so the call needs d_buf to be memory of the CURRENT device and `stream` a
 * stream of that device (NULL: the current device's legacy stream); otherwise it returns
 * IPM_ERR_DEVICE and launches nothing (a host pointer gives the same answer).
 * ipm_read_noalloc_status reads the device status word (IPM_OK, IPM_ERR_TIMEOUT or
 * IPM_ERR_DEVICE) that the last no-alloc call on the current device left in the array;
 * it synchronises `stream`.  Before the first no-alloc call on a device it reads IPM_OK.
 */
ipm_status ipm_read_noalloc_status(ipm_stream_t stream, ipm_status *out);

/*
 * Optional per-phase timing (for benchmarks).  When enabled on a host thread, the
 * merge entry points called from that thread record a CUDA event pair on their stream
 * around each launch group: phase 0 = early exit + split, 1 = exchange plan,
 * 2 = exchange levels (one launch per level), 3 = pair merge, 4 = batched merge
 * (queue order + persistent kernel), 5 = split-model training, 6 = learned splits.
 * ipm_timing_read waits for the recorded events, adds their elapsed times and
 * kernel-launch counts into *out and forgets them.  Timing adds two event records per
 * group and changes no kernel.
 */
#define IPM_TIMING_PHASES 8
typedef struct {
    double ms[IPM_TIMING_PHASES];
    uint32_t launches[IPM_TIMING_PHASES];
} ipm_timing;

ipm_status ipm_timing_enable(int enable);
ipm_status ipm_timing_read(ipm_timing *out);

/*
 * Read the device status word that the last call using this workspace left (IPM_OK,
 * IPM_ERR_TIMEOUT or IPM_ERR_DEVICE).  Synchronises `stream`.
 */
ipm_status ipm_read_device_status(const void *d_ws, ipm_stream_t stream, ipm_status *out);

#ifdef __cplusplus
}
#endif

#endif /* IPMERGE_H */
