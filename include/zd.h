/*
 * zd.h -- C ABI of the zd-tree k-NN library (libzd) for one GB300 (sm_103a).
 *
 * The library implements the data-parallel path of the zd-tree of
 * Blelloch & Dobson, "Parallel Nearest Neighbors in Low Dimensions with Batch
 * Updates": Morton encoding, a radix sort by Morton key, the canonical pruned
 * zd-tree (Algorithm 1 with the empty-cut pruning of Sec. 2.1), exact k-NN
 * search (Algorithms 2 and 3), batch insert and delete (Sec. 2
 * "Batch-dynamic updates", Algorithm 4), plus a backward pass for a sum of
 * k-NN distances and a batched multi-cloud form.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *   are host pointers.  The caller owns every buffer it passes; the library
 *   never frees or keeps a caller buffer beyond the call.
 * - `stream` is a cudaStream_t passed as void*.  All work is enqueued on it;
 *   no entry point synchronizes the host unless its comment says so
 *   ("syncs").  Entry points that do not sync may be captured in a CUDA graph.
 * - Points are row-major [n, dim] arrays of int32 (ZD_COORD_I32) or float32
 *   (ZD_COORD_F32).
 * - Errors: arguments that can be checked on the host return a status at
 *   once.  Data-dependent errors (a coordinate out of range, an unknown
 *   delete id, a device-side wait that timed out) are recorded in a
 *   device-wide status word; zd_check() reads and clears it.
 * - The library owns the memory of a tree.  It allocates through the
 *   zd_allocator given to zd_build (stream-ordered); a NULL allocator means
 *   the library's own stream-ordered pool on the current device
 *   (cudaMallocFromPoolAsync / cudaFreeAsync on the call's stream), which
 *   keeps up to ZD_POOL_KEEP_BYTES of freed memory reserved for reuse across
 *   synchronizations instead of returning it to the driver at each one.
 * - Ids are int32.  zd_build gives point i the id i; inserts hand out new
 *   ids in order; deleted ids are never reused.
 * - A `const zd_tree*` may be searched from several streams at once (the
 *   paper's queries run concurrently on a shared tree, Sec. 1); updates need
 *   exclusive access.  A search launches persistent kernels (as many blocks
 *   as fit on the device) whose warps take work from per-SM queues that the
 *   call allocates for itself; no warp waits for another, so concurrent
 *   searches stay correct while they share the SMs.
 */
#ifndef ZD_H
#define ZD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum zd_status {
    ZD_OK = 0,
    ZD_ERR_INVALID_ARG = 1,  /* bad argument (host-checked) */
    ZD_ERR_RANGE = 2,        /* a shifted integer coordinate outside [0, 2^coord_bits),
                                or a float one non-finite or above 1e18 in magnitude */
    ZD_ERR_OOM = 3,          /* the allocator returned NULL */
    ZD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    ZD_ERR_NOT_FOUND = 5,    /* delete of an id that is not live */
    ZD_ERR_DUPLICATE_ID = 6, /* the same id twice in one delete batch */
    ZD_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    ZD_ERR_UNIMPLEMENTED = 8,/* a parameter combination not built (e.g. k > ZD_MAX_K) */
    ZD_ERR_CAPACITY = 9,     /* beyond a size limit: an insert past the tree's
                                capacity, or more than ZD_MAX_KEYS keys (or
                                ZD_NOALLOC_MAX_KEYS for the no-allocation sort) */
    ZD_ERR_INTERNAL = 10     /* a kernel's index check failed (recorded only by
                                a library built with -DZD_DEBUG; the access was
                                skipped): a bug in the library */
} zd_status;

enum { ZD_COORD_I32 = 0, ZD_COORD_F32 = 1 };

/* Search modes of Sec. 2: leaf-based (all points, Algorithm 3 from each
 * point's own leaf), bit-based (external queries: descend by Morton bits to a
 * leaf, then Algorithm 3) and root-based (external queries: Algorithm 2 from
 * the root). */
enum { ZD_SEARCH_LEAF = 0, ZD_SEARCH_BIT = 1, ZD_SEARCH_ROOT = 2 };

/* Optional thread mapping of a search, OR-ed into the mode of zd_knn /
 * zd_knn_batched.  ZD_KNN_THREAD_PER_QUERY: one thread runs one query's
 * traversal.  ZD_KNN_WARP_GROUP (leaf- and bit-based modes, and external
 * queries of a forest): one warp runs one shared traversal for 32 queries
 * that are consecutive in Morton order, each lane keeping its own k best.
 * Both return the same exact neighbours.  Default (neither flag): warp groups
 * for all points and for external queries at least a quarter as many as the
 * tree's points when k >= 3 (k >= 16 for integer trees with B > 24), one
 * thread per query otherwise. */
enum { ZD_KNN_THREAD_PER_QUERY = 0x100, ZD_KNN_WARP_GROUP = 0x200 };

/* OR-ed into ZD_SEARCH_BIT or ZD_SEARCH_ROOT with d_queries NULL: the k-NN
 * graph of the tree's own points (each excluding itself), every query started
 * the bit-based or root-based way -- the paper's three ways of computing the
 * k-NN graph (Sec. 2, Sec. 5).  The answer is the same for all three; these
 * starts always run one thread (or, for k > 32, one warp) per query. */
enum { ZD_KNN_ALL_POINTS = 0x400 };

/* Largest k of one search.  Up to 32 neighbours a query's list lives in one
 * thread's registers (both mappings above), up to 40 under warp groups; for
 * larger k (and for 32 < k <= 40 without warp groups) one warp serves one
 * query with the list spread over its lanes. */
#define ZD_MAX_K 128

/* Most keys one radix sort handles: the points of a tree (its capacity
 * included) or of a forest, the external queries of one zd_knn /
 * zd_knn_batched call, the keys of one zd_morton_sort and the (query,
 * neighbour) pairs of one zd_knn_dist_backward.  The sort's look-back words
 * carry a digit's running count in 30 bits.  Larger sizes return
 * ZD_ERR_CAPACITY before any work is enqueued. */
#define ZD_MAX_KEYS 1073741823 /* 2^30 - 1 */

/* Freed memory the default allocator's pool keeps reserved per device (8 GiB;
 * beyond that it is returned to the driver at synchronization points). */
#define ZD_POOL_KEEP_BYTES 8589934592ull

typedef struct zd_params {
    int32_t dim;        /* 2 or 3 */
    int32_t leaf_size;  /* L >= 1: a leaf holds at most L points unless all
                           its keys are equal (Alg. 1, sizeCutoff = L + 1) */
    int32_t coord_bits; /* B: integer coordinates + shift lie in [0, 2^B);
                           dim * B <= 64.  Float trees quantize onto this grid. */
    int32_t coord_type; /* ZD_COORD_I32 or ZD_COORD_F32 */
    uint32_t shift[3];  /* per-coordinate shift added before encoding (Sec. 2
                           "Construction"); integer trees only */
    int64_t capacity;   /* most live points the tree may ever hold (for
                           inserts); 0 means n */
} zd_params;

typedef struct zd_allocator {
    /* Stream-ordered allocation of `bytes`; return NULL on failure. */
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    /* Release a block returned by alloc (same size), ordered on `stream`. */
    void (*release)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} zd_allocator;

typedef struct zd_tree zd_tree;

typedef struct zd_tree_info {
    int64_t n;          /* live points */
    int64_t capacity;   /* most live points */
    int64_t next_id;    /* the id the next insert hands out */
    int64_t n_leaves;   /* leaves of the canonical tree */
    int64_t n_internal; /* internal nodes (= n_leaves - 1) */
    int32_t dim, leaf_size, coord_bits, coord_type;
    int64_t n_clouds;   /* 1, or the cloud count of a batched tree */
} zd_tree_info;

/* Message for a status code (static storage). */
const char *zd_status_string(int status);

/* Syncs `stream`, then returns and clears the device-wide status word: the
 * first data-dependent error recorded since the last zd_check, or ZD_OK. */
int zd_check(void *stream);

/* Failure-detection check (no counterpart in the paper).  Launches one warp
 * that waits on a device flag that nothing ever sets, through the same
 * bounded wait that guards every device-side wait of the library (the radix
 * sort's look-back).  The wait gives up after timeout_ms (1..2000) and
 * records ZD_ERR_TIMEOUT, so a following zd_check returns ZD_ERR_TIMEOUT and
 * the context stays usable.  Nothing faults or hangs. */
int zd_selftest_wait_timeout(int timeout_ms, void *stream);

/* ---------------------------------------------------------------- steps -- */

/* Morton keys (Sec. 1.1 "Morton ordering"; shift of Sec. 2 "Construction").
 * d_pts: int32 [n, dim]; d_keys: uint64 [n] out.  Key bit d*b + (d-1-j) is
 * bit b of coordinate j + shift[j]: at every bit level the first coordinate is
 * the most significant.  A coordinate with c + shift outside [0, 2^B) records
 * ZD_ERR_RANGE and gets key 0.  Integer points only. */
int zd_morton_encode(const zd_params *p, const int32_t *d_pts, int64_t n, uint64_t *d_keys,
                     void *stream);

/* Stable sort by key (Sec. 2 "Construction": the points are sorted by Morton
 * order; Sec. 2.2 / Theorem 1: a radix sort).  d_keys_in [n] is read only;
 * d_keys_out [n] gets the keys ascending and d_perm_out [n] the input
 * position of each output (equal keys keep input order).  key_bits (1..64)
 * bounds the significant low bits; digits above it are not sorted.  Scratch
 * comes from `alloc` (NULL: cudaMallocAsync).  n > ZD_MAX_KEYS returns
 * ZD_ERR_CAPACITY. */
int zd_morton_sort(const uint64_t *d_keys_in, int64_t n, int key_bits, uint64_t *d_keys_out,
                   int32_t *d_perm_out, const zd_allocator *alloc, void *stream);

/* zd_morton_sort without allocating: the paper has no counterpart.  It is
 * for callers that may not allocate device memory on their call path -- a
 * plug-in running inside a host framework that has reserved the GPU's memory
 * for its own pool, or a latency-critical loop that must not pay for (or be
 * serialized by) an allocation.  Same arguments and result as zd_morton_sort,
 * but all scratch lives in one static device array of this library
 * (about 26 MB for ZD_NOALLOC_MAX_KEYS keys), which every GPU that loads
 * the library holds until the process exits; nothing is allocated or freed.
 * n > ZD_NOALLOC_MAX_KEYS returns ZD_ERR_CAPACITY with no work enqueued.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  Every call shares
 * the one array: calls whose work overlaps on the GPU (for example on two
 * streams) race and corrupt each other; order them on one stream. */
#define ZD_NOALLOC_MAX_KEYS (1 << 20)
int zd_morton_sort_noalloc(const uint64_t *d_keys_in, int64_t n, int key_bits, uint64_t *d_keys_out,
                           int32_t *d_perm_out, void *stream);

/* ----------------------------------------------------------------- tree -- */

/* Build the canonical pruned zd-tree of n points (Sec. 2 "Construction",
 * Algorithm 1, Sec. 2.1): encode, sort, split every node on the highest bit
 * where its keys differ, leaves of at most L points, a tight bounding box per
 * node.  Float points (ZD_COORD_F32) are quantized for the keys only:
 * q = floor((x - lo_j) * s), s = (2^B - 1) / (largest extent), clamped; the
 * boxes and the search use the float values, which must be finite and at
 * most 1e18 in magnitude (else ZD_ERR_RANGE is recorded; the same holds for
 * float queries).  Integer coordinates outside the shifted universe record
 * ZD_ERR_RANGE too.  The point data is copied; the
 * caller may free d_pts after the call's work is done.  *out receives the
 * handle (free with zd_free).  n or capacity above ZD_MAX_KEYS returns
 * ZD_ERR_CAPACITY. */
int zd_build(const zd_params *p, const zd_allocator *alloc, const void *d_pts, int64_t n,
             void *stream, zd_tree **out);

/* Release a tree's memory (ordered on `stream`) and the handle. */
int zd_free(zd_tree *t, void *stream);

/* Sizes of a tree.  Syncs `stream` (the leaf count lives on the device). */
int zd_tree_info_get(const zd_tree *t, zd_tree_info *out, void *stream);

/* Copy the tree out, for inspection and checks.  Device outputs, any may be
 * NULL: d_ids [n] and d_keys [n] in sorted order; per leaf j (n_leaves):
 * d_leaf_lo [n_leaves + 1] start positions; per internal node i (n_internal):
 * d_node_lo, d_node_hi (range of sorted positions), d_node_bit (split bit),
 * d_node_left, d_node_right (child: >= 0 internal node, < 0 leaf ~c),
 * d_node_parent (-1 at the root); d_leaf_parent [n_leaves]; boxes as
 * [count, dim] int32 (integer trees) or float32 (float trees):
 * d_node_box_lo/hi and d_leaf_box_lo/hi.  The root is internal node 0 when
 * n_internal > 0, else leaf 0. */
int zd_export_tree(const zd_tree *t, int32_t *d_ids, uint64_t *d_keys, int32_t *d_leaf_lo,
                   int32_t *d_node_lo, int32_t *d_node_hi, int32_t *d_node_bit,
                   int32_t *d_node_left, int32_t *d_node_right, int32_t *d_node_parent,
                   int32_t *d_leaf_parent, void *d_node_box_lo, void *d_node_box_hi,
                   void *d_leaf_box_lo, void *d_leaf_box_hi, void *stream);

/* Exact k-NN (Algorithms 2 and 3).  Neighbours are ranked by (squared
 * distance, id): int64 exact for integer trees, fp64 evaluated as
 * ((dx*dx + dy*dy) + dz*dz) without contraction for float trees.
 *   mode ZD_SEARCH_LEAF (or ZD_SEARCH_BIT / ZD_SEARCH_ROOT | ZD_KNN_ALL_POINTS):
 *     d_queries must be NULL; every live point is a query and excludes itself
 *     (by id); row r of the outputs is the point with id r, so the outputs
 *     need next_id rows (rows of deleted ids are left untouched).
 *   mode ZD_SEARCH_BIT / ZD_SEARCH_ROOT: d_queries [m, dim] (the tree's
 *     coordinate type) are external queries; row r is query r.  The queries
 *     are sorted by Morton key first (Sec. 3.1), so bit-based queries must
 *     lie in the tree's key range (else ZD_ERR_RANGE is recorded).
 * d_idx [rows, k] gets ids (-1 where fewer than k candidates exist); d_dist
 * [rows, k] (may be NULL) gets int64 squared distances (integer trees,
 * INT64_MAX padding) or float32 Euclidean distances computed in fp32 (float
 * trees, +inf padding).  1 <= k <= ZD_MAX_K (larger k: ZD_ERR_UNIMPLEMENTED). */
int zd_knn(const zd_tree *t, const void *d_queries, int64_t m, int k, int mode, int32_t *d_idx,
           void *d_dist, void *stream);

/* Largest batch that zd_insert_batch / zd_delete_batch apply point by point
 * on the device (below). */
#define ZD_SMALL_BATCH 16

/* Batch insert (Sec. 2 "Batch-dynamic updates", Algorithm 4): the tree
 * afterwards equals the canonical tree of the new point set.  d_pts [b, dim]
 * in the tree's coordinate type (integer trees only); d_new_ids [b] (may be
 * NULL) receives the ids given to the batch, in batch order.  Returns
 * ZD_ERR_CAPACITY if n + b exceeds the capacity.
 * - b > ZD_SMALL_BATCH: encode and sort the batch, merge it into the sorted
 *   points and re-derive the tree; validates by syncing `stream` before it
 *   commits (a coordinate out of range returns ZD_ERR_RANGE, nothing changed).
 * - b <= ZD_SMALL_BATCH: one device thread inserts the points one by one into
 *   the tree's pointer form (descent by key bits, a new node where a key leaves
 *   a node's prefix, a leaf split past L): O(depth) work per point and no
 *   sync.  A coordinate out of range records ZD_ERR_RANGE for zd_check and the
 *   batch changes nothing (its ids are used up).  The first such batch after a
 *   build or a larger batch copies the tree into the pointer form and syncs
 *   once.  The searches read a flat layout of the tree: until it is
 *   re-derived, external queries with k <= 32 that are fewer than a quarter
 *   of the points search the pointer form directly (one thread per query,
 *   the same exact answers); any other search, an export, zd_tree_info_get
 *   or a larger batch re-derives the flat layout first (O(n) work, syncs
 *   once).  While small batches are pending the tree must not be searched
 *   from another stream. */
int zd_insert_batch(zd_tree *t, const void *d_pts, int64_t b, int32_t *d_new_ids, void *stream);

/* Batch delete by id (Sec. 2: "deletions use an almost identical algorithm"):
 * the tree afterwards equals the canonical tree of the remaining points.
 * d_ids [b] must be distinct live ids; otherwise nothing is deleted and the
 * status is ZD_ERR_NOT_FOUND or ZD_ERR_DUPLICATE_ID (returned for
 * b > ZD_SMALL_BATCH, which syncs `stream`; recorded for zd_check for smaller
 * batches, which do not sync and are applied point by point like small
 * inserts: a leaf that empties is spliced out, a subtree that drops to L points
 * becomes one leaf). */
int zd_delete_batch(zd_tree *t, const int32_t *d_ids, int64_t b, void *stream);

/* ------------------------------------------------------------- backward -- */

/* Gradient of loss = sum_{p,i,j} gout * || q_{p,i} - ref_{p, idx(p,i,j)} ||
 * over `batch` independent problems (no paper counterpart: an extension).
 * d_q [batch, m, dim], d_ref [batch, r, dim] float32; d_idx [batch, m, k]
 * ids local to each problem (< 0 entries are skipped); d_gout: one float32
 * (gout_per_pair = 0) or [batch, m, k] weights (gout_per_pair = 1).
 * Distances are recomputed in fp32 from the coordinates; a zero distance
 * contributes nothing.  d_gq [batch, m, dim] and d_gref [batch, r, dim] are
 * overwritten.  The reference gradient is a deterministic sum (no atomics). */
int zd_knn_dist_backward(const float *d_q, const float *d_ref, const int32_t *d_idx,
                         int64_t batch, int64_t m, int64_t r, int dim, int k,
                         const float *d_gout, int gout_per_pair, float *d_gq, float *d_gref,
                         void *stream);

/* -------------------------------------------------------------- batched -- */

/* Build one forest of n_clouds independent canonical trees in one pass:
 * d_pts holds the clouds back to back, cloud c at rows [h_offsets[c],
 * h_offsets[c+1]) (h_offsets: host int64 [n_clouds + 1]; d_offsets: the same
 * on the device).  Keys carry the cloud id above the Morton bits, so one
 * sort orders every cloud and each cloud's subtree is its own canonical tree;
 * coord_bits is lowered to fit dim * B + ceil(log2(n_clouds)) <= 64.  Float
 * clouds are quantized per cloud.  Ids are local to each cloud. */
int zd_build_batched(const zd_params *p, const zd_allocator *alloc, const void *d_pts,
                     const int64_t *h_offsets, const int64_t *d_offsets, int64_t n_clouds,
                     void *stream, zd_tree **out);

/* k-NN in every cloud of a batched tree, searches never leaving their cloud.
 * d_queries NULL: all points of every cloud (row = global row of the point in
 * the build input, ids local); else external queries [m, dim] with
 * d_query_offsets [n_clouds + 1] (device) assigning rows to clouds, searched
 * root-based within their cloud.  mode_flags: 0 or one ZD_KNN_* mapping flag.
 * Outputs as zd_knn. */
int zd_knn_batched(const zd_tree *t, const void *d_queries, const int64_t *d_query_offsets,
                   int64_t m, int k, int mode_flags, int32_t *d_idx, void *d_dist, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ZD_H */
