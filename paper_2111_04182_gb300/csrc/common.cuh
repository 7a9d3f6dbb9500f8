// common.cuh -- internal declarations shared by the libzd translation units.
//
// Device layout of a tree (all arrays owned by the tree, sized by capacity):
//   keys[n]      uint64 Morton keys in sorted order (cloud id above the Morton
//                bits for a batched forest)
//   pts[n]       int4 (x, y, z, id) in sorted order; float trees keep the
//                float bit patterns in x, y, z.  One 16-byte load per point.
//   leaf_of[n]   index of the leaf holding each sorted position
//   leaf_lo[]    leaf j holds sorted positions [leaf_lo[j], leaf_lo[j+1])
//   internal node i (0 <= i < n_leaves - 1; node 0 is the root):
//     ichild[i]  int2 (left, right): >= 0 internal node, < 0 leaf ~c
//     iparent[i], ibit[i] (split bit), ibox[2i], ibox[2i+1] (lo, hi corners)
//   leaf j: lparent[j], lbox[2j], lbox[2j+1]
//   meta[0]      n_leaves (device-resident so that a build needs no host sync)
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "../../include/zd.h"

namespace zdk {

// Host: an NVTX range over a scope, so a profiler's timeline shows every
// entry point and its phases (encode, sort, gather, topology, search, ...).
// With no tool attached a range costs one call.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

typedef unsigned long long u64;
typedef unsigned int u32;

// ------------------------------------------------------------------ status
// Device-wide status word: the first data-dependent error wins.
__device__ __forceinline__ void set_status(u32 *status, int code)
{
    atomicCAS(status, 0u, (u32)code);
}

// Host: address of this device's status word (looked up once per device).
u32 *status_word();

// Exact float copy of an integer point: the shifted coordinates (c + shift
// lies in [0, 2^B), B <= 24), id bits kept in w.
__device__ __forceinline__ float4 shifted_float4(int4 p, uint3 sh)
{
    return make_float4((float)((unsigned)p.x + sh.x), (float)((unsigned)p.y + sh.y),
                       (float)((unsigned)p.z + sh.z), __int_as_float(p.w));
}

// Host: this device's number of SMs (looked up once per device).
int sm_count();

// Debug builds (compiled with -DZD_DEBUG) check the index arithmetic of the
// kernels before the accesses it guards: a failed check records
// ZD_ERR_INTERNAL in the status word and evaluates to false, and the caller
// skips the access (never a trap, so the context stays usable).  In normal
// builds the check is the constant true and costs nothing.
#ifdef ZD_DEBUG
#define ZD_DCHECK(cond, status) ((cond) ? true : (::zdk::set_status((status), ZD_ERR_INTERNAL), false))
#else
#define ZD_DCHECK(cond, status) true
#endif

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every device-side wait of the library goes through this: poll *p until a
// bit of `mask` is set, backing off with __nanosleep, and give up after
// timeout_ns of wall time or max_polls polls.  Returns false on giving up;
// the caller then records ZD_ERR_TIMEOUT and carries on so the kernel ends
// and the context stays usable.
__device__ __forceinline__ bool wait_for_flag(const volatile u32 *p, u32 mask, unsigned long long timeout_ns,
                                              int max_polls, u32 &w)
{
    w = *p;
    if (w & mask) return true;
    const unsigned long long t0 = globaltimer();
    int polls = 0;
    while (!((w = *p) & mask)) {
        ++polls;
        if (polls > 32) __nanosleep(64);
        if (polls >= max_polls || ((polls & 1023) == 0 && globaltimer() - t0 > timeout_ns)) return false;
    }
    return true;
}

// ----------------------------------------------------------------- memory
struct Mem {
    const zd_allocator *a;
    cudaStream_t s;
    bool failed = false;
    void *get(size_t bytes);
    void put(void *p, size_t bytes);
};

// A scratch block returned to the allocator when it goes out of scope.
template <typename T>
struct Scratch {
    Mem *m = nullptr;
    T *p = nullptr;
    size_t bytes = 0;
    Scratch() {}
    Scratch(Mem &mem, size_t count) : m(&mem), bytes(count * sizeof(T) + 16)
    {
        p = (T *)mem.get(bytes);
    }
    ~Scratch()
    {
        if (p) m->put(p, bytes);
    }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
};

// ------------------------------------------------------------- tree view
struct TreeView {
    int n;
    int dim;
    int coord_bits;
    int cloud_bit;       // 64 for a single tree; dim*B for a batched forest
    const u64 *keys;
    const int4 *pts;
    const int *leaf_of;
    const int *leaf_lo;
    const int *meta;
    const int2 *ichild;
    const int *iparent;
    const int *ibit;
    const int2 *irange;   // sorted-position range [x, y) of internal nodes
    const int4 *ibox;
    const int *lparent;
    const int4 *lbox;
    const int64_t *cloud_off; // batched: device offsets [n_clouds + 1], else nullptr
    // exact float copies of integer points / boxes (coordinate window <= 2^24), or null
    const float4 *fpts;
    const float4 *fibox;
    const float4 *flbox;
};

struct zd_tree_impl;

// --------------------------------------------------------------- sorting
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;

// Encode integer points to Morton keys and (optionally) accumulate the digit
// histograms of all passes (hist may be null).  With seg_off (device offsets
// [n_seg + 1]) the segment (cloud) id of every row is placed at cloud_shift.
int launch_encode_i32(const int32_t *pts, int64_t n, int dim, int coord_bits, const uint32_t *shift,
                      const int64_t *seg_off, int64_t n_seg, int cloud_shift, u64 *keys, u32 *hist,
                      int npasses, cudaStream_t s);

// Float points: per-segment quantization frames (lo_x, lo_y, lo_z, scale),
// frame: device double [n_seg * 4]; mm: device int scratch [n_seg * 6].
int launch_float_frames(const float *pts, int64_t n, int dim, int coord_bits,
                        const int64_t *seg_off, int64_t n_seg, int64_t max_seg, double *frame,
                        int *mm, cudaStream_t s);
int launch_encode_f32(const float *pts, int64_t n, int dim, int coord_bits, const double *frame,
                      const int64_t *seg_off, int64_t n_seg, int cloud_shift, u64 *keys, u32 *hist,
                      int npasses, cudaStream_t s);

// Stable LSD radix sort of keys_in (read only) into keys_out / perm_out.
// hist: device [MAX_PASSES * RADIX] digit histograms of keys_in (already
// accumulated), or null to have the sort compute them.
int radix_sort(const u64 *keys_in, int64_t n, int key_bits, u64 *keys_out, int32_t *perm_out,
               u32 *hist, Mem &mem);

// ------------------------------------------------------------------ build
// Gather sorted points: pts_out[i] = (coords of row perm[i], id), with
// id = base_id + perm[i], or perm[i] - cloud_off[key >> cloud_bit] when
// cloud_off is given.  Float points travel as their bit patterns.  With
// fpts_out (integer points), the exact float copy of the coordinates plus
// fshift is written as well.
int launch_gather(const void *pts_in, int dim, int64_t n, const int32_t *perm,
                  const u64 *sorted_keys, int cloud_bit, const int64_t *cloud_off, int32_t base_id,
                  int4 *pts_out, cudaStream_t s, float4 *fpts_out = nullptr, uint3 fshift = {0, 0, 0});

struct TopoBuffers {
    int *leaf_of;
    int *leaf_lo;
    int *meta;
    int2 *ichild;
    int *iparent;
    int *ibit;
    int2 *irange;
    int4 *ibox;
    int *lparent;
    int4 *lbox;
    int *counter; // scratch [n] for the bottom-up box pass
    // integer trees with B <= 24: float copies of the SHIFTED coordinates
    // (c + shift lies in [0, 2^B), so they are exact; differences of shifted
    // coordinates are the coordinate differences), or null
    float4 *fpts, *fibox, *flbox;
    uint3 fshift;
};

// From sorted keys and points, build leaves, internal nodes and boxes.
// Boundaries whose highest differing key bit is >= force_bit (the cloud id
// bits of a forest; 64 for one tree) always separate leaves, so every
// cloud's subtree is that cloud's own canonical tree.
// Write the float copy of sorted integer points (shifted_float4).
int launch_fpts(const int4 *pts, int64_t n, float4 *fpts, uint3 shift, cudaStream_t s);

// fpts_ready: b.fpts was already written (by the gather or an update).
int build_topology(const u64 *keys, const int4 *pts, int64_t n, int leaf_size, int dim,
                   int is_float, int force_bit, const TopoBuffers &b, Mem &mem, bool fpts_ready = false);

// Forests: group_start[g] = first sorted position of the g-th 32-point group,
// groups laid out cloud by cloud so that none crosses a cloud boundary.
// gpre: device scratch [n_clouds + 1] owned by the caller; gpre[n_clouds]
// receives the number of groups (n_groups only bounds the launch).
int launch_group_starts(const int64_t *cloud_off, int64_t n_clouds, int64_t n_groups, int *group_start,
                        int64_t *gpre, cudaStream_t s);

// -------------------------------------------------------------------- knn
constexpr int KNN_MAX_K_THREAD = 32; // largest k of the one-thread-per-query mapping
constexpr int KNN_MAX_K_GROUP = 40;  // largest k of the warp-group mapping

struct KnnArgs {
    TreeView t;
    int k;
    int mode;              // ZD_SEARCH_*: how a query finds its start
    int allpts;            // queries are the tree's own points (self excluded)
    int is_float;
    // external queries, already in Morton order
    const int4 *q;         // (x, y, z, row) in tree coordinates (float bits for float trees)
    const u64 *qkey;       // Morton keys of the sorted queries (bit mode; cloud in batched root mode)
    int64_t m;
    int32_t *out_idx;
    void *out_dist;
    uint3 shift;             // the tree's coordinate shift (Morton cells)
    // warp-group mapping (integer coordinates)
    int idb;                 // id bits of the packed (d^2, id) keys
    const int *group_start;  // first sorted position of every group (forests), or null
    int64_t n_groups;        // groups launched (an upper bound when group_count is set)
    const int64_t *group_count; // device: groups that exist, or null
    const int64_t *q_off;    // forests, external queries: device query offsets [n_clouds + 1]
    int *fix_list;           // queries whose packed k-th distance saturated
    int *fix_count;
    // warp groups: one counter per chunk of the SM-affine group feed (zeroed
    // by the launcher), n_chunks of them, or null for one group per warp
    int *chunk_ctr;
    int n_chunks;
    int64_t chunk_len; // groups per chunk (the launcher sets it)
    // exact kernel restricted to listed sorted positions (fallback), or null
    const int *sel;
    const int *sel_count;
};
int launch_knn_i32(const KnnArgs &a, cudaStream_t s);
int launch_knn_group_i32(const KnnArgs &a, cudaStream_t s); // + exact fallback
int launch_knn_f32(const KnnArgs &a, cudaStream_t s);
int launch_knn_group_f32(const KnnArgs &a, cudaStream_t s);
// Large k (above the thread / group limits, up to ZD_MAX_K): one warp per
// query, any mode, integer or float.
int launch_knn_wide(const KnnArgs &a, cudaStream_t s);

// ---------------------------------------------------------- small updates
// (local.cu) The tree in pointer form, updated point by point by one device
// thread without a host round trip; re-derived into the flat layout before
// the next search.  The pools hold LOCAL_BUDGET point updates between two
// copies from the flat tree; LOCAL_GROW_RESERVE slab entries serve leaves of
// equal keys that outgrow their slab.
constexpr int LOCAL_BUDGET = 1 << 16;
constexpr int64_t LOCAL_GROW_RESERVE = 1 << 20;
struct LocalForm;
// Updates the pointer form could not apply (out of slab room), in order,
// for replay through the flat update path.
struct LocalLog {
    int64_t n = 0;
    std::vector<int> op, id, xyz; // op: 1 insert, 2 delete
};
// Copy the flat tree into a fresh pointer form for ids < id_slots (reads the
// leaf count back: syncs once).
int local_convert(LocalForm **lf, const TreeView &v, int64_t n, int L, int64_t id_slots, Mem &mem);
int64_t local_id_slots(const LocalForm *lf);
// One launch of one thread each; no sync.  Invalid batches record a status
// and change nothing.
int local_insert(LocalForm *lf, const int32_t *d_pts, int64_t b, int dim, int B, const uint32_t *shift,
                 int32_t first_id, int32_t *d_new_ids, u32 *live, cudaStream_t s);
int local_delete(LocalForm *lf, const int32_t *d_ids, int64_t b, u32 *live, int64_t id_cap, cudaStream_t s);
// The pointer form's points in (key, id) order into keys_out / pts_out (syncs
// to read the point count), and the log of updates it could not apply.
int local_flatten(LocalForm *lf, u64 *keys_out, int4 *pts_out, int64_t *n_out, LocalLog *log, Mem &mem);
void local_release(LocalForm *lf, Mem &mem);
// External k-NN queries (already in Morton order, row in w) on the pointer
// form, one thread per query, k <= LOCAL_MAX_K: what a search of a tree whose
// flat arrays lag behind uses when its queries are sparse (no re-derivation).
constexpr int LOCAL_MAX_K = 32;
int local_knn(LocalForm *lf, int dim, const int4 *q4, const u64 *qkeys, int64_t m, int k, int mode,
              int32_t *d_idx, void *d_dist, cudaStream_t s);

// --------------------------------------------------------------- backward
int launch_backward(const float *q, const float *ref, const int32_t *idx, int64_t batch, int64_t m,
                    int64_t r, int dim, int k, const float *gout, int gout_per, float *gq,
                    float *gref, Mem &mem);

} // namespace zdk

// Host-side errors from the CUDA runtime become ZD_ERR_CUDA.
#define ZD_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return ZD_ERR_CUDA;                                         \
    } while (0)

#define ZD_TRY(call)                                                                       \
    do {                                                                                   \
        int r_ = (call);                                                                   \
        if (r_ != ZD_OK) return r_;                                                        \
    } while (0)

static inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}
