/*
 * pkd.h -- C ABI of the GB300 (sm_103a) Pkd-tree library, libpkd.so.
 *
 * The Pkd-tree is the parallel kd-tree of "Parallel kd-tree with Batch
 * Updates" (Men, Shen, Gu, Sun, SIGMOD 2025).  Every step of these calls runs
 * in the library's own CUDA kernels; the host only sequences launches.
 *
 * Conventions for every entry point:
 *  - Points have d int32 coordinates in [0, 2^30) stored point-major
 *    (coords[i*d + j]) and a uint32 id that names the point: the ids stored
 *    in a tree are distinct, and 0xFFFFFFFF is never an id.  Builds, inserts
 *    and queries reject coordinates outside that range with PKD_EINVAL.
 *  - Point, query and result buffers are DEVICE pointers owned by the
 *    caller, except in pkd_export (host buffers).  The library copies what it
 *    keeps; input buffers may be reused once the call has returned.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Builds
 *    and batch updates return after their work on `stream` has completed
 *    (they report device-side failures).  A build's sieve rounds are decided
 *    on the device: the rounds, the skeleton levels within them and the
 *    exact levels run from one CUDA graph launch whose conditional nodes
 *    test counts the kernels leave in device memory, so the host does not
 *    wait between rounds (option "graph_rounds").  The rebuilds inside a
 *    batch update run the same way; the update's own routing rounds read
 *    their counts on the host.  Queries are asynchronous: their outputs are
 *    valid once `stream` has been synchronised.
 *  - A pkd_tree is not thread-safe: one call at a time per tree, except
 *    that queries on an unchanging tree may overlap.
 *  - Return value 0 (PKD_OK) or one of the error codes below; device-side
 *    failures (a bound exceeded, a wait that ran out) are reported by the
 *    call that detects them, and leave the tree unusable: free it.
 */
#ifndef PKD_H
#define PKD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PKD_OK 0
#define PKD_EINVAL 1    /* bad parameter, size or coordinate */
#define PKD_ENOMEM 2    /* device memory exhausted; the tree is unchanged */
#define PKD_ECUDA 3     /* a CUDA runtime call failed */
#define PKD_ETIMEOUT 4  /* a bounded device-side wait ran out */
#define PKD_EINTERNAL 5 /* a device-side consistency check failed */

typedef struct pkd_tree pkd_tree;

/* Parameters (Sec. 5 "Parameter Choosing" of the paper uses lambda = 6,
 * phi = 32, sigma = 32, alpha = 0.3).
 *   d           dimensions, 1..8
 *   phi         leaf wrap: a subproblem of at most phi points is a leaf (>= 1)
 *   lambda      skeleton levels built per sieve round, 1..10 (Alg. 1)
 *   sigma_log2  rate mode: each point is sampled with probability
 *               2^-sigma_log2 (0..30; 0 samples every point)
 *   sigma_os    a skeleton node is split only when it holds at least
 *               2*sigma_os samples (the oversampling of Lemma 3.1), >= 1
 *   count_mode  1: instead of a fixed rate, sample about 2^lambda*sigma_os
 *               points per subproblem as Alg. 1 does
 *   alpha       weight-balance parameter alpha_num/alpha_den in [0, 1/2]
 *               (Sec. 2), alpha_den <= 2^20
 *   seed        salt of the sampling hash
 * The tree is a deterministic function of (points, ids, parameters). */
typedef struct {
  int d;
  int phi;
  int lambda;
  int sigma_log2;
  int sigma_os;
  int count_mode;
  int alpha_num;
  int alpha_den;
  uint64_t seed;
} pkd_params;

/* Build a Pkd-tree over n points (Alg. 1: sample, lambda-level skeleton,
 * sieve into 2^lambda buckets, recurse; leaves of at most phi points).
 *   coords  device, [n][d] int32
 *   ids     device, [n] uint32, or NULL for ids 0..n-1.  Ids name the
 *           points: they must be distinct and not 0xFFFFFFFF (the k-NN
 *           padding value).  The tree keeps an id table (id -> coordinates)
 *           for deletes by id and for the id checks of inserts.
 *   n       number of points, < 2^31 (0 gives an empty tree); the tree
 *           holds fewer than 2^31 points after any insert (node slots are
 *           32-bit: two per arena position, plus skeleton nodes)
 *   out     receives the new tree (owns all device memory it allocates)
 * Errors: PKD_EINVAL (parameters, n, coordinates, a repeated or reserved
 * id), PKD_ENOMEM, PKD_ECUDA. */
int pkd_build(const int32_t* coords, const uint32_t* ids, uint64_t n, const pkd_params* params,
              void* stream, pkd_tree** out);

/* BatchInsert (Alg. 2): sieve the batch through the existing skeletons,
 * update subtree sizes top-down, rebuild with Build every subtree that would
 * leave the alpha balance and every leaf that receives points.
 *   coords  device, [m][d] int32;  ids  device, [m] uint32 (required)
 * The whole batch is rejected with PKD_EINVAL, and the tree is unchanged,
 * when an id is 0xFFFFFFFF, names a point stored in the tree, or appears
 * twice in the batch.  An id deleted earlier may be inserted again.
 * Errors: PKD_EINVAL (tree unchanged), PKD_ENOMEM (see below),
 * PKD_ECUDA / PKD_ETIMEOUT / PKD_EINTERNAL (tree unusable). */
int pkd_batch_insert(pkd_tree* tree, const int32_t* coords, const uint32_t* ids, uint64_t m,
                     void* stream);

/* BatchDelete (Sec. 4.2, two rounds) of the points named by ids: each id is
 * looked up in the tree's id table for its coordinates, the found points are
 * sieved to the leaves and removed, then the tree is rebalanced top-down
 * with the exact new sizes (subtrees that leave the alpha balance are
 * rebuilt).  Ids that name no stored point (never inserted, or deleted
 * already) and repeats within the batch are skipped, as round 1 of Sec. 4.2
 * discards points that are not in the tree; they are not errors.
 *   ids        device, [m] uint32
 *   n_deleted  host, optional: number of points removed
 * Errors as for pkd_batch_insert. */
int pkd_batch_delete(pkd_tree* tree, const uint32_t* ids, uint64_t m, uint64_t* n_deleted, void* stream);

/* k nearest neighbours (Sec. 5 "Queries": depth-first search, near child
 * first, far child pruned by the distance to its subspace).  For query i,
 * out_ids[i*k .. i*k+k) and out_d2[...] receive the k smallest
 * (squared Euclidean distance, id) pairs in lexicographic order; slots past
 * the tree size hold id 0xFFFFFFFF and distance INT64_MAX.
 *   queries  device, [q][d] int32 in [0, 2^30);  k  in 1..128
 *   out_ids  device, [q][k] uint32;  out_d2  device, [q][k] int64 */
int pkd_knn(const pkd_tree* tree, const int32_t* queries, uint64_t q, int k, uint32_t* out_ids,
            int64_t* out_d2, void* stream);

/* k-NN ids that allocate nothing (the paper has no counterpart): the same
 * search and the same out_ids as pkd_knn, for callers that may not allocate
 * device memory during the call (a server that has given its spare memory
 * to its trees and may not let a pool grow mid-request, or one that wants no
 * allocator or mapping work in a query's latency).  The coordinate-check
 * flag and the k distances per query live in one fixed scratch array
 * compiled into the library (one per device), so
 *   - q * k must not exceed PKD_NOALLOC_MAX_PAIRS (8 MiB of distances);
 *     larger batches return PKD_EINVAL with a message on stderr (split
 *     them, or use pkd_knn);
 *   - the call must run on the tree's device (the current device);
 *   - calls whose device work overlaps (other streams, other host threads)
 *     race on the scratch; calls one after another on one stream do not;
 *   - the first call on a device is its set-up: it resolves the scratch
 *     address and runs every search kernel variant (all d, both k ranges)
 *     once on an empty query set, so that the kernels are loaded and the
 *     driver's local-memory reservation is sized for the largest of them
 *     (about 10 KB per resident thread at d = 8, k > 16); make that call
 *     before any region in which the caller may not allocate.  Later calls
 *     allocate nothing on the host or the device.
 * The call synchronises `stream` once (after the coordinate check) and
 * returns with the search queued on it; out_ids is valid once `stream` has
 * been synchronised.
 *   queries  device, [q][d] int32 in [0, 2^30);  k  in 1..128
 *   out_ids  device, [q][k] uint32 (as pkd_knn)
 * Errors: PKD_EINVAL (k, q * k, coordinates, wrong device), PKD_ECUDA,
 * PKD_EINTERNAL (also for a tree of height 126 or more, whose search stacks
 * would need scratch memory: pkd_knn serves those). */
#define PKD_NOALLOC_MAX_PAIRS (1u << 20)
int pkd_knn_ids_noalloc(const pkd_tree* tree, const int32_t* queries, uint64_t q, int k,
                        uint32_t* out_ids, void* stream);

/* Search depth (pkd_knn, pkd_range_count, pkd_range_report): each query's
 * depth-first stack holds up to height + 1 entries.  Below height 126 they
 * live in registers and local memory; a deeper tree (possible only after
 * long runs of one-sided updates with alpha near 1/2, where no interior node
 * is rebuilt) is searched with stacks in a scratch buffer of the library's
 * pool, at most 1 GiB, a chunk of queries at a time. */

/* Range count (Sec. 5): for each closed box lo[i][j] <= x_j <= hi[i][j],
 * the number of stored points inside; a subtree whose subspace lies inside
 * the box adds its stored size.
 *   lo, hi  device, [q][d] int32;  out_counts  device, [q] uint64 */
int pkd_range_count(const pkd_tree* tree, const int32_t* lo, const int32_t* hi, uint64_t q,
                    uint64_t* out_counts, void* stream);

/* Range report (Sec. 5, the reporting form of the range query): the ids of
 * the stored points inside each closed box lo[i][j] <= x_j <= hi[i][j].
 *   lo, hi    device, [q][d] int32
 *   offsets   device, [q + 1] uint64: box i's ids are
 *             ids[offsets[i] .. offsets[i+1]) (depth-first leaf order)
 *   ids       device, [ids_cap] uint32
 *   total     host: the number of ids (offsets[q])
 * The call counts, scans and synchronises `stream` once; when *total
 * exceeds ids_cap it returns PKD_EINVAL with offsets and *total filled and
 * no ids written (call again with a large enough buffer).  The ids are
 * valid once `stream` has been synchronised. */
int pkd_range_report(const pkd_tree* tree, const int32_t* lo, const int32_t* hi, uint64_t q, uint64_t* offsets,
                     uint32_t* ids, uint64_t ids_cap, uint64_t* total, void* stream);

/* Stored bounding boxes: the paper's Pkd-bb variant (Sec. 6, the study of
 * bounding boxes).  With enable = 1 every node keeps the tight box of the
 * points in its subtree (8d bytes per node slot, computed bottom-up now and
 * again after every batch update), and pkd_knn, pkd_range_count and
 * pkd_range_report prune with those boxes instead of the subspace implied by
 * the splitters above a node (the Pkd form, the default).  The answers are
 * identical; only the search differs.  enable = 0 frees the boxes.
 * Synchronises `stream`.  Errors: PKD_EINVAL, PKD_ENOMEM (boxes off), PKD_ECUDA. */
int pkd_set_bounding_boxes(pkd_tree* tree, int enable, void* stream);

/* The stored boxes in the pre-order of pkd_export, into HOST buffers
 * lo[n_nodes][d], hi[n_nodes][d] (n_nodes as pkd_export reports it); an
 * empty subtree has lo = INT32_MAX and hi = INT32_MIN.  PKD_EINVAL when
 * the boxes are off or n_nodes differs.  Synchronises the device. */
int pkd_export_boxes(const pkd_tree* tree, int32_t* lo, int32_t* hi, uint64_t n_nodes);

/* Canonical form of the tree into HOST buffers (for parity checks and
 * checkpoints): nodes in pre-order, interior nodes as (dim, split, size),
 * leaves as (0xFF, 0, point count); leaves in in-order with their ids sorted
 * ascending, leaf k owning leaf_ids[leaf_offsets[k] .. leaf_offsets[k+1]).
 * Any NULL buffer is skipped, so a first call with NULL buffers returns
 * *n_nodes and *n_leaves for sizing (leaf_ids needs pkd_size() entries,
 * leaf_offsets n_leaves + 1).  Synchronises the device. */
int pkd_export(const pkd_tree* tree, uint8_t* dims, int32_t* splits, uint64_t* sizes,
               uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves);

/* Number of stored points. */
uint64_t pkd_size(const pkd_tree* tree);

/* Longest root-to-leaf path (edges) into *height.  Synchronises the device. */
int pkd_height(const pkd_tree* tree, int* height);

/* Free the tree and all device memory it owns (NULL is a no-op).  Returns
 * without waiting: the memory is released on the legacy default stream
 * after the work every earlier call queued on the tree (each call records
 * an event on its stream when it returns), so a query still running on
 * another stream finishes on the tree it was given.  After a
 * pkd_knn_ids_noalloc call on a stream no other call on this tree used (it
 * may not create an event), the free waits for the whole device instead.
 * pkd_forest_free behaves the same. */
void pkd_free(pkd_tree* tree);

/* Batched build of independent trees ("forest"): one pass over n_trees
 * point sets, each built exactly as pkd_build would build it alone (Alg. 1
 * per tree: its own root at depth 0, its own samples), with the sieve
 * rounds and base cases of all trees sharing the same launches.  The paper
 * builds one tree per call; batching many trees is this library's
 * extension.
 *   coords   device, [n][d] int32, the trees' points one after another
 *   ids      device, [n] uint32, or NULL for ids 0..n-1 (positions in coords)
 *   offsets  HOST, [n_trees + 1] uint64: tree i owns points
 *            offsets[i] .. offsets[i+1]; offsets[0] = 0, non-decreasing,
 *            n = offsets[n_trees] < 2^31 (empty trees are allowed)
 *   n_trees  1 .. 2^24 - 1
 * Errors: PKD_EINVAL (parameters, offsets, coordinates), PKD_ENOMEM,
 * PKD_ECUDA.  A forest is read-only: its trees take exports and k-NN queries
 * (same semantics as pkd_export / pkd_knn). */
typedef struct pkd_forest pkd_forest;
int pkd_build_forest(const int32_t* coords, const uint32_t* ids, const uint64_t* offsets, uint32_t n_trees,
                     const pkd_params* params, void* stream, pkd_forest** out);
uint32_t pkd_forest_trees(const pkd_forest* forest);
uint64_t pkd_forest_size(const pkd_forest* forest, uint32_t tree);
int pkd_forest_export(const pkd_forest* forest, uint32_t tree, uint8_t* dims, int32_t* splits, uint64_t* sizes,
                      uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves);
int pkd_forest_knn(const pkd_forest* forest, uint32_t tree, const int32_t* queries, uint64_t q, int k,
                   uint32_t* out_ids, int64_t* out_d2, void* stream);
void pkd_forest_free(pkd_forest* forest);

/* Device memory on the current device as the library sees it (HOST
 * outputs, each optional): the driver's free bytes, the bytes the library's
 * stream-ordered pool holds and of those the bytes in use (blocks kept in
 * the library's large-block cache for reuse count as in use), the cached
 * bytes, and `available` = free + the pool's unused bytes + the cache, the
 * memory a new request can draw on.  A server admits requests by it. */
int pkd_mem_info(uint64_t* device_free, uint64_t* pool_reserved, uint64_t* pool_used, uint64_t* cached,
                 uint64_t* available);

/* Human-readable text for an error code. */
const char* pkd_strerror(int code);

/* Tuning knobs (testing and autotuning; results never depend on them):
 *   "base_cap"   largest subproblem finished in one CTA's shared memory
 *                (0 = derived from d and the shared-memory size)
 *   "skel_cap"   largest sample handled by one CTA when building a skeleton
 *   "tile"       points per tile of the sieve kernels (256..4096, a power of
 *                two; default 2048)
 *   "sieve_kernel" sieve count/scatter: 0 persistent CTAs streaming tiles
 *                through shared memory with bulk copies, the count recording
 *                every point's bucket for the scatter when there are at most
 *                256 buckets (default); 2 the same kernels with the scatter
 *                walking the skeleton again; 1 one CTA per tile
 *   "base_kernel" shared-memory base case: 0 sorts each subproblem once per
 *                dimension and splits by lookups (default), 1 selects every
 *                splitter by a radix select
 *   "graph_rounds" 1 (default): a build's rounds run from one CUDA graph whose
 *                WHILE / IF nodes test device-side counts, and its base cases
 *                are persistent launches over device-side lists; 0: the same
 *                kernels with the host reading the counts after every step
 *                (one stream synchronisation per round and skeleton level)
 *   "front_cap"  > 0: first capacity (entries) of the lists with which an
 *                update flattens the subtrees it rebuilds (testing; 0, the
 *                default, sizes them by the points of those subtrees).  A
 *                list that overflows makes the update redo the flatten with
 *                room for every node of the tree, before any visible change.
 * Returns PKD_EINVAL for an unknown name or an out-of-range value. */
int pkd_set_option(const char* name, int64_t value);

/* Per-kernel timing with CUDA events on the launching stream (off by
 * default).  pkd_kernel_stats fills, for kernel family `name`, the number
 * of timed launches, their summed duration in ms and the points (items)
 * they processed; pkd_kernel_timing(1) enables and clears the counters.
 * The name "launches" reports, in *launches, every kernel launch the
 * library made since the last pkd_kernel_timing call (timed or not).
 * Families: "validate", "sample", "count" and "scatter" (sieve rounds of a
 * build), "count_route" and "scatter_route" (sieve rounds that route an
 * update batch; items = batch points they move), "smem_build" (shared-memory
 * base case, one CTA per subproblem), "smem_warp" (one warp per subproblem),
 * "knn", "range_count", "range_report", "id_claim" and "id_take" (the id
 * table's fill at an insert (a build fills it beside its base cases,
 * untimed) and its lookups at a delete; items = ids),
 * "graph_record" (host time to record a build's graph; items = graphs
 * recorded).  Counts without a time: "rebuilt_insert" and "rebuilt_delete"
 * (points in the subtrees an update rebuilt, one entry per call),
 * "delete_gather" (ids a delete found and looked up), "scratch_zeroed"
 * (a tree's first delete took a released tree's per-node delete scratch,
 * which every delete leaves all zero, from the block cache without clearing
 * it; items = bytes), "front_retries" (updates whose flatten lists
 * overflowed and were redone larger).  The name
 * "allocations" reports, in *launches, every device or pinned-host allocation
 * the library made since it was loaded; "graph_builds" the builds (and update
 * rebuilds) whose rounds ran from one graph launch.  With graph rounds,
 * "launches" counts each recorded kernel node once, although a node in a
 * loop body runs once per iteration. */
int pkd_kernel_timing(int enable);
int pkd_kernel_stats(const char* name, uint64_t* launches, double* total_ms, uint64_t* items);

#ifdef __cplusplus
}
#endif
#endif /* PKD_H */
