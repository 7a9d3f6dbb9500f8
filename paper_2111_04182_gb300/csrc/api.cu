// api.cu -- the C ABI of libzd (declared in include/zd.h): argument checks,
// tree lifetime and memory, and the sequencing of the kernels of each step.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"

using namespace zdk;

// ------------------------------------------------------------ status word
static __device__ u32 g_status;

namespace zdk {
u32 *status_word()
{
    // per-device cache of the symbol's device address; atomic entries, so two
    // host threads making their first call at once store the same value
    static std::atomic<u32 *> addr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    u32 *a = addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        a = (u32 *)p;
        addr[dev].store(a, std::memory_order_release);
    }
    return a;
}

int sm_count()
{
    static std::atomic<int> cnt[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int v = cnt[dev].load(std::memory_order_acquire);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
        cnt[dev].store(v, std::memory_order_release);
    }
    return v;
}

// The default allocator's per-device memory pool.  The device's default
// stream-ordered pool returns freed memory to the driver at every
// synchronization (release threshold 0), so a caller that synchronizes between
// two builds would pay to map the tree's memory again on the second one
// (measured: build of 10^7 points 3.6 ms instead of 1.4 ms).  This pool keeps
// up to ZD_POOL_KEEP_BYTES reserved across synchronizations.
static cudaMemPool_t default_pool()
{
    static std::atomic<cudaMemPool_t> pools[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    cudaMemPool_t p = pools[dev].load(std::memory_order_acquire);
    if (p) return p;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t np = nullptr;
    if (cudaMemPoolCreate(&np, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = ZD_POOL_KEEP_BYTES;
    if (cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    cudaMemPool_t expected = nullptr;
    if (pools[dev].compare_exchange_strong(expected, np)) return np;
    cudaMemPoolDestroy(np); // another thread made this device's pool first
    return expected;
}

void *Mem::get(size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (a && a->alloc) {
        p = a->alloc(bytes, (void *)s, a->ctx);
    } else {
        cudaMemPool_t pool = default_pool();
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (!p) failed = true;
    return p;
}

void Mem::put(void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (a && a->release) a->release(p, bytes, (void *)s, a->ctx);
    else cudaFreeAsync(p, s);
}
} // namespace zdk

// ------------------------------------------------------------------- tree
struct Block {
    void *p;
    size_t bytes;
};

struct zd_tree {
    zd_params p;
    zd_allocator alloc;
    bool has_alloc;
    int64_t n, cap, next_id, n_clouds;
    int B;         // coordinate bits of the keys
    int key_bits;  // significant key bits (Morton + cloud id)
    int cloud_bit; // 64 for a single tree, dim * B for a forest
    int is_float;
    // device arrays
    u64 *keys, *keys2;
    int4 *pts, *pts2;
    int *leaf_of, *leaf_lo, *meta;
    int2 *ichild;
    int *iparent, *ibit;
    int2 *irange;
    int4 *ibox;
    int *lparent;
    int4 *lbox;
    int *counter;
    float4 *fpts, *fibox, *flbox; // integer trees with B <= 24: exact float copies
    double *frame;      // float trees: [n_clouds * 4]
    int64_t *cloud_off; // forests: [n_clouds + 1]
    u32 *alive;         // dynamic trees: live bits [0, W), marked bits [W, 2W), W = id_words
    int64_t id_cap;     // ids the bitmaps cover (a multiple of 32)
    int64_t id_words;
    int64_t max_cloud;  // largest cloud (forests): bounds the local ids
    int *group_start;   // forests: first sorted position of every 32-point group
    int64_t n_groups;
    Block blocks[32];
    int nblocks;
    // small update batches (local.cu): the pointer form, whether the flat
    // arrays lag behind it, whether it lags behind the flat arrays, and the
    // point updates it has taken since it was copied from them.  While the
    // flat arrays lag, n is an upper bound (a rejected batch is not known
    // until the flat arrays are re-derived).
    LocalForm *local;
    bool flat_stale, local_stale;
    int64_t local_ops;
};

// The flat arrays that every search reads lag behind the pointer form after
// small update batches; a search, export, info or large batch re-derives
// them first (defined with the updates below).
static int ensure_flat(zd_tree *t, cudaStream_t s);

static Mem mem_of(const zd_tree *t, cudaStream_t s)
{
    Mem m;
    m.a = t->has_alloc ? &t->alloc : nullptr;
    m.s = s;
    return m;
}

template <typename T>
static bool tree_alloc(zd_tree *t, Mem &m, T **out, size_t count)
{
    size_t bytes = count * sizeof(T) + 16;
    void *p = m.get(bytes);
    *out = (T *)p;
    if (!p) return false;
    t->blocks[t->nblocks++] = Block{p, bytes};
    return true;
}

static void tree_release(zd_tree *t, cudaStream_t s)
{
    Mem m = mem_of(t, s);
    for (int i = 0; i < t->nblocks; ++i) m.put(t->blocks[i].p, t->blocks[i].bytes);
    t->nblocks = 0;
    local_release(t->local, m);
    t->local = nullptr;
}

static TreeView view_of(const zd_tree *t)
{
    TreeView v;
    v.n = (int)t->n;
    v.dim = t->p.dim;
    v.coord_bits = t->B;
    v.cloud_bit = t->cloud_bit;
    v.keys = t->keys;
    v.pts = t->pts;
    v.leaf_of = t->leaf_of;
    v.leaf_lo = t->leaf_lo;
    v.meta = t->meta;
    v.ichild = t->ichild;
    v.iparent = t->iparent;
    v.ibit = t->ibit;
    v.irange = t->irange;
    v.ibox = t->ibox;
    v.lparent = t->lparent;
    v.lbox = t->lbox;
    v.cloud_off = t->cloud_off;
    v.fpts = t->fpts;
    v.fibox = t->fibox;
    v.flbox = t->flbox;
    return v;
}

static TopoBuffers topo_of(zd_tree *t)
{
    TopoBuffers b;
    b.leaf_of = t->leaf_of;
    b.leaf_lo = t->leaf_lo;
    b.meta = t->meta;
    b.ichild = t->ichild;
    b.iparent = t->iparent;
    b.ibit = t->ibit;
    b.irange = t->irange;
    b.ibox = t->ibox;
    b.lparent = t->lparent;
    b.lbox = t->lbox;
    b.counter = t->counter;
    b.fpts = t->fpts;
    b.fibox = t->fibox;
    b.flbox = t->flbox;
    b.fshift = make_uint3(t->p.shift[0], t->p.shift[1], t->p.shift[2]);
    return b;
}

static int check_params(const zd_params *p)
{
    if (!p) return ZD_ERR_INVALID_ARG;
    if (p->dim != 2 && p->dim != 3) return ZD_ERR_INVALID_ARG;
    if (p->leaf_size < 1 || p->leaf_size > 256) return ZD_ERR_INVALID_ARG;
    if (p->coord_type != ZD_COORD_I32 && p->coord_type != ZD_COORD_F32) return ZD_ERR_INVALID_ARG;
    // coordinate differences must fit int32: B <= 31 (2D), 21 (3D)
    const int bmax = p->dim == 3 ? 21 : 31;
    if (p->coord_bits < 1 || p->coord_bits > bmax) return ZD_ERR_INVALID_ARG;
    if (p->capacity < 0) return ZD_ERR_INVALID_ARG;
    return ZD_OK;
}

static int ceil_log2(int64_t x)
{
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Allocate every device array of a tree for `cap` points and `n_clouds`.
static int tree_arrays(zd_tree *t, Mem &m, bool dynamic)
{
    const size_t cap = (size_t)std::max<int64_t>(t->cap, 1);
    bool ok = tree_alloc(t, m, &t->keys, cap) && tree_alloc(t, m, &t->pts, cap) &&
              tree_alloc(t, m, &t->leaf_of, cap) && tree_alloc(t, m, &t->leaf_lo, cap + 2) &&
              tree_alloc(t, m, &t->meta, 4) && tree_alloc(t, m, &t->ichild, cap) &&
              tree_alloc(t, m, &t->iparent, cap) && tree_alloc(t, m, &t->ibit, cap) &&
              tree_alloc(t, m, &t->irange, cap) && tree_alloc(t, m, &t->ibox, 2 * cap) &&
              tree_alloc(t, m, &t->lparent, cap + 1) && tree_alloc(t, m, &t->lbox, 2 * cap + 2) &&
              tree_alloc(t, m, &t->counter, cap);
    if (ok && t->is_float) ok = tree_alloc(t, m, &t->frame, 4 * (size_t)t->n_clouds);
    if (ok && !t->is_float && t->B <= 24)
        ok = tree_alloc(t, m, &t->fpts, cap) && tree_alloc(t, m, &t->fibox, 2 * cap) &&
             tree_alloc(t, m, &t->flbox, 2 * cap + 2);
    if (ok && dynamic) {
        ok = tree_alloc(t, m, &t->keys2, cap) && tree_alloc(t, m, &t->pts2, cap);
    }
    return ok ? ZD_OK : ZD_ERR_OOM;
}

static zd_tree *tree_new(const zd_params *p, const zd_allocator *alloc)
{
    zd_tree *t = (zd_tree *)calloc(1, sizeof(zd_tree));
    if (!t) return nullptr;
    t->p = *p;
    if (alloc) {
        t->alloc = *alloc;
        t->has_alloc = true;
    }
    t->is_float = p->coord_type == ZD_COORD_F32;
    t->local = nullptr;
    t->flat_stale = false;
    t->local_stale = true;
    t->local_ops = 0;
    return t;
}

// encode -> sort -> gather -> topology, shared by every build.
static int build_core(zd_tree *t, const void *d_pts, const int64_t *seg_off, int64_t n_seg,
                      int64_t max_seg, cudaStream_t s)
{
    Mem m = mem_of(t, s);
    const int64_t n = t->n;
    const int dim = t->p.dim;
    const int npasses = (t->key_bits + RADIX_BITS - 1) / RADIX_BITS;
    Scratch<u64> raw(m, n > 0 ? n : 1);
    Scratch<int32_t> perm(m, n > 0 ? n : 1);
    Scratch<u32> hist(m, MAX_PASSES * RADIX);
    Scratch<int> mm(m, (size_t)6 * std::max<int64_t>(n_seg, 1));
    if (!raw.p || !perm.p || !hist.p || !mm.p) return ZD_ERR_OOM;
    ZD_CUDA(cudaMemsetAsync(hist.p, 0, MAX_PASSES * RADIX * sizeof(u32), s));
    const int cloud_shift = seg_off ? t->cloud_bit : 0;
    {
        NvtxScope r("encode");
        if (t->is_float) {
            ZD_TRY(launch_float_frames((const float *)d_pts, n, dim, t->B, seg_off, n_seg, max_seg,
                                       t->frame, mm.p, s));
            ZD_TRY(launch_encode_f32((const float *)d_pts, n, dim, t->B, t->frame, seg_off, n_seg,
                                     cloud_shift, raw.p, hist.p, npasses, s));
        } else {
            ZD_TRY(launch_encode_i32((const int32_t *)d_pts, n, dim, t->B, t->p.shift, seg_off, n_seg,
                                     cloud_shift, raw.p, hist.p, npasses, s));
        }
    }
    {
        NvtxScope r("sort");
        ZD_TRY(radix_sort(raw.p, n, t->key_bits, t->keys, perm.p, hist.p, m));
    }
    {
        NvtxScope r("gather");
        ZD_TRY(launch_gather(d_pts, dim, n, perm.p, t->keys, t->cloud_bit, t->cloud_off, 0, t->pts, s,
                             t->is_float ? nullptr : t->fpts, topo_of(t).fshift));
    }
    {
        NvtxScope r("topology");
        ZD_TRY(build_topology(t->keys, t->pts, n, t->p.leaf_size, dim, t->is_float, t->cloud_bit, topo_of(t),
                              m, /*fpts_ready=*/true));
    }
    return m.failed ? ZD_ERR_OOM : ZD_OK;
}

// Liveness bitmaps of a fresh tree: ids [0, n) live, nothing marked.
__global__ void k_init_bits(u32 *bits, int64_t words, int64_t n)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 2 * words;
         w += (int64_t)gridDim.x * blockDim.x) {
        u32 v = 0;
        if (w < words) {
            const int64_t lo = 32 * w;
            v = lo + 32 <= n ? 0xffffffffu : (lo < n ? (1u << (n - lo)) - 1u : 0u);
        }
        bits[w] = v;
    }
}

// Copy both bitmaps into larger ones (new words zero).
__global__ void k_grow_bits(const u32 *old, int64_t ow, u32 *nw_bits, int64_t nw)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 2 * nw;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t half = w < nw ? 0 : 1, i = w - half * nw;
        nw_bits[w] = i < ow ? old[half * ow + i] : 0u;
    }
}

extern "C" {

const char *zd_status_string(int status)
{
    switch (status) {
    case ZD_OK: return "ok";
    case ZD_ERR_INVALID_ARG: return "invalid argument";
    case ZD_ERR_RANGE: return "coordinate outside [0, 2^coord_bits) after the shift";
    case ZD_ERR_OOM: return "out of device memory";
    case ZD_ERR_CUDA: return "CUDA runtime error";
    case ZD_ERR_NOT_FOUND: return "id not live";
    case ZD_ERR_DUPLICATE_ID: return "id repeated in one batch";
    case ZD_ERR_TIMEOUT: return "bounded device wait timed out";
    case ZD_ERR_UNIMPLEMENTED: return "not implemented for these parameters";
    case ZD_ERR_CAPACITY: return "size limit exceeded";
    case ZD_ERR_INTERNAL: return "internal index check failed (debug build)";
    default: return "unknown status";
    }
}

int zd_check(void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    ZD_CUDA(cudaStreamSynchronize(s));
    u32 *w = status_word();
    if (!w) return ZD_ERR_CUDA;
    u32 v = 0;
    ZD_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    if (v) {
        u32 z = 0;
        ZD_CUDA(cudaMemcpy(w, &z, sizeof(z), cudaMemcpyHostToDevice));
    }
    return (int)v;
}

int zd_morton_encode(const zd_params *p, const int32_t *d_pts, int64_t n, uint64_t *d_keys,
                     void *stream)
{
    NvtxScope nvtx_("zd_morton_encode");
    ZD_TRY(check_params(p));
    if (p->coord_type != ZD_COORD_I32 || n < 0 || (n > 0 && (!d_pts || !d_keys)))
        return ZD_ERR_INVALID_ARG;
    if (!status_word()) return ZD_ERR_CUDA;
    return launch_encode_i32(d_pts, n, p->dim, p->coord_bits, p->shift, nullptr, 0, 0,
                             (u64 *)d_keys, nullptr, 0, (cudaStream_t)stream);
}

int zd_morton_sort(const uint64_t *d_keys_in, int64_t n, int key_bits, uint64_t *d_keys_out,
                   int32_t *d_perm_out, const zd_allocator *alloc, void *stream)
{
    NvtxScope nvtx_("zd_morton_sort");
    if (n < 0 || key_bits < 1 || key_bits > 64) return ZD_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys_in || !d_keys_out || !d_perm_out)) return ZD_ERR_INVALID_ARG;
    if (n > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (!status_word()) return ZD_ERR_CUDA;
    Mem m;
    m.a = alloc;
    m.s = (cudaStream_t)stream;
    int r = radix_sort((const u64 *)d_keys_in, n, key_bits, (u64 *)d_keys_out, d_perm_out, nullptr, m);
    if (r == ZD_OK && m.failed) r = ZD_ERR_OOM;
    return r;
}

int zd_build(const zd_params *p, const zd_allocator *alloc, const void *d_pts, int64_t n,
             void *stream, zd_tree **out)
{
    NvtxScope nvtx_("zd_build");
    if (!out) return ZD_ERR_INVALID_ARG;
    *out = nullptr;
    ZD_TRY(check_params(p));
    if (n < 0 || (n > 0 && !d_pts)) return ZD_ERR_INVALID_ARG;
    if (p->capacity > 0 && p->capacity < n) return ZD_ERR_INVALID_ARG;
    if (n > ZD_MAX_KEYS || p->capacity > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (!status_word()) return ZD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    zd_tree *t = tree_new(p, alloc);
    if (!t) return ZD_ERR_OOM;
    t->n = n;
    t->cap = std::max<int64_t>(p->capacity, n);
    t->next_id = n;
    t->n_clouds = 1;
    t->B = p->coord_bits;
    t->key_bits = p->dim * p->coord_bits;
    t->cloud_bit = 64;
    const bool dynamic = !t->is_float;
    Mem m = mem_of(t, s);
    int r = tree_arrays(t, m, dynamic);
    if (r == ZD_OK && dynamic) {
        t->id_words = (std::max<int64_t>(t->cap, 1) + 31) / 32;
        t->id_cap = 32 * t->id_words;
        if (!tree_alloc(t, m, &t->alive, (size_t)(2 * t->id_words))) r = ZD_ERR_OOM;
        if (r == ZD_OK) {
            k_init_bits<<<grid_for(2 * t->id_words, 256, 4096), 256, 0, s>>>(t->alive, t->id_words, n);
            if (cudaGetLastError() != cudaSuccess) r = ZD_ERR_CUDA;
        }
    }
    if (r == ZD_OK) r = build_core(t, d_pts, nullptr, 1, n, s);
    if (r != ZD_OK) {
        tree_release(t, s);
        free(t);
        return r;
    }
    *out = t;
    return ZD_OK;
}

int zd_build_batched(const zd_params *p, const zd_allocator *alloc, const void *d_pts,
                     const int64_t *h_offsets, const int64_t *d_offsets, int64_t n_clouds,
                     void *stream, zd_tree **out)
{
    NvtxScope nvtx_("zd_build_batched");
    if (!out) return ZD_ERR_INVALID_ARG;
    *out = nullptr;
    ZD_TRY(check_params(p));
    if (n_clouds < 1 || n_clouds > 65535 || !h_offsets || !d_offsets) return ZD_ERR_INVALID_ARG;
    if (h_offsets[0] != 0) return ZD_ERR_INVALID_ARG;
    int64_t max_seg = 0;
    for (int64_t c = 0; c < n_clouds; ++c) {
        int64_t sz = h_offsets[c + 1] - h_offsets[c];
        if (sz < 0) return ZD_ERR_INVALID_ARG;
        max_seg = std::max(max_seg, sz);
    }
    const int64_t n = h_offsets[n_clouds];
    if (n > 0 && !d_pts) return ZD_ERR_INVALID_ARG;
    if (n > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    const int cbits = ceil_log2(n_clouds);
    const int B = std::min(p->coord_bits, (64 - cbits) / p->dim);
    if (B < 1) return ZD_ERR_INVALID_ARG;
    if (!status_word()) return ZD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    zd_tree *t = tree_new(p, alloc);
    if (!t) return ZD_ERR_OOM;
    t->n = n;
    t->cap = n;
    t->next_id = 0;
    t->n_clouds = n_clouds;
    t->B = B;
    t->cloud_bit = p->dim * B;
    t->key_bits = t->cloud_bit + cbits;
    Mem m = mem_of(t, s);
    int r = tree_arrays(t, m, false);
    if (r == ZD_OK && !tree_alloc(t, m, &t->cloud_off, (size_t)n_clouds + 1)) r = ZD_ERR_OOM;
    if (r == ZD_OK && cudaMemcpyAsync(t->cloud_off, d_offsets, sizeof(int64_t) * (n_clouds + 1),
                                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        r = ZD_ERR_CUDA;
    if (r == ZD_OK) r = build_core(t, d_pts, t->cloud_off, n_clouds, max_seg, s);
    // 32-point groups that never cross a cloud, for the warp-group search
    t->max_cloud = max_seg;
    t->n_groups = 0;
    for (int64_t c = 0; c < n_clouds; ++c) t->n_groups += (h_offsets[c + 1] - h_offsets[c] + 31) / 32;
    if (r == ZD_OK && !tree_alloc(t, m, &t->group_start, (size_t)std::max<int64_t>(t->n_groups, 1)))
        r = ZD_ERR_OOM;
    Scratch<int64_t> gpre(m, (size_t)n_clouds + 1);
    if (r == ZD_OK && !gpre.p) r = ZD_ERR_OOM;
    if (r == ZD_OK) r = launch_group_starts(t->cloud_off, n_clouds, t->n_groups, t->group_start, gpre.p, s);
    if (r != ZD_OK) {
        tree_release(t, s);
        free(t);
        return r;
    }
    *out = t;
    return ZD_OK;
}

int zd_free(zd_tree *t, void *stream)
{
    NvtxScope nvtx_("zd_free");
    if (!t) return ZD_OK;
    tree_release(t, (cudaStream_t)stream);
    free(t);
    return ZD_OK;
}

int zd_tree_info_get(const zd_tree *t, zd_tree_info *out, void *stream)
{
    if (!t || !out) return ZD_ERR_INVALID_ARG;
    ZD_TRY(ensure_flat(const_cast<zd_tree *>(t), (cudaStream_t)stream));
    int nl = 1;
    ZD_CUDA(cudaMemcpyAsync(&nl, t->meta, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    ZD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    out->n = t->n;
    out->capacity = t->cap;
    out->next_id = t->next_id;
    out->n_leaves = nl;
    out->n_internal = nl - 1;
    out->dim = t->p.dim;
    out->leaf_size = t->p.leaf_size;
    out->coord_bits = t->B;
    out->coord_type = t->p.coord_type;
    out->n_clouds = t->n_clouds;
    return ZD_OK;
}

} // extern "C"

// Export helpers: split int4 box pairs into [count, dim] corner arrays and
// internal node ranges into lo / hi.
__global__ void k_export_boxes(const int4 *box, const int *meta, int internal, int dim, int32_t *lo,
                               int32_t *hi)
{
    const int count = internal ? meta[0] - 1 : meta[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        int4 a = box[2 * i], b = box[2 * i + 1];
        int va[3] = {a.x, a.y, a.z}, vb[3] = {b.x, b.y, b.z};
        for (int j = 0; j < dim; ++j) {
            if (lo) lo[(int64_t)i * dim + j] = va[j];
            if (hi) hi[(int64_t)i * dim + j] = vb[j];
        }
    }
}

__global__ void k_export_nodes(const int2 *irange, const int2 *ichild, const int *meta, int32_t *lo,
                               int32_t *hi, int32_t *left, int32_t *right)
{
    const int count = meta[0] - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (lo) lo[i] = irange[i].x;
        if (hi) hi[i] = irange[i].y;
        if (left) left[i] = ichild[i].x;
        if (right) right[i] = ichild[i].y;
    }
}

__global__ void k_export_ids(const int4 *pts, int64_t n, int32_t *ids)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        ids[i] = pts[i].w;
}

extern "C" int zd_export_tree(const zd_tree *t, int32_t *d_ids, uint64_t *d_keys, int32_t *d_leaf_lo,
                              int32_t *d_node_lo, int32_t *d_node_hi, int32_t *d_node_bit,
                              int32_t *d_node_left, int32_t *d_node_right, int32_t *d_node_parent,
                              int32_t *d_leaf_parent, void *d_node_box_lo, void *d_node_box_hi,
                              void *d_leaf_box_lo, void *d_leaf_box_hi, void *stream)
{
    if (t) ZD_TRY(ensure_flat(const_cast<zd_tree *>(t), (cudaStream_t)stream));
    NvtxScope nvtx_("zd_export_tree");
    if (!t) return ZD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int nl = 1;
    ZD_CUDA(cudaMemcpyAsync(&nl, t->meta, sizeof(int), cudaMemcpyDeviceToHost, s));
    ZD_CUDA(cudaStreamSynchronize(s));
    const int64_t n = t->n;
    if (d_ids && n > 0) k_export_ids<<<grid_for(n, 256, 4096), 256, 0, s>>>(t->pts, n, d_ids);
    if (d_keys && n > 0)
        ZD_CUDA(cudaMemcpyAsync(d_keys, t->keys, sizeof(u64) * n, cudaMemcpyDeviceToDevice, s));
    if (d_leaf_lo)
        ZD_CUDA(cudaMemcpyAsync(d_leaf_lo, t->leaf_lo, sizeof(int) * (nl + 1), cudaMemcpyDeviceToDevice, s));
    if (nl > 1) {
        k_export_nodes<<<grid_for(nl, 256, 4096), 256, 0, s>>>(t->irange, t->ichild, t->meta, d_node_lo,
                                                              d_node_hi, d_node_left, d_node_right);
        if (d_node_bit)
            ZD_CUDA(cudaMemcpyAsync(d_node_bit, t->ibit, sizeof(int) * (nl - 1), cudaMemcpyDeviceToDevice, s));
        if (d_node_parent)
            ZD_CUDA(cudaMemcpyAsync(d_node_parent, t->iparent, sizeof(int) * (nl - 1),
                                    cudaMemcpyDeviceToDevice, s));
        if (d_node_box_lo || d_node_box_hi)
            k_export_boxes<<<grid_for(nl, 256, 4096), 256, 0, s>>>(t->ibox, t->meta, 1, t->p.dim,
                                                                  (int32_t *)d_node_box_lo,
                                                                  (int32_t *)d_node_box_hi);
    }
    if (d_leaf_parent)
        ZD_CUDA(cudaMemcpyAsync(d_leaf_parent, t->lparent, sizeof(int) * nl, cudaMemcpyDeviceToDevice, s));
    if (d_leaf_box_lo || d_leaf_box_hi)
        k_export_boxes<<<grid_for(nl, 256, 4096), 256, 0, s>>>(t->lbox, t->meta, 0, t->p.dim,
                                                              (int32_t *)d_leaf_box_lo,
                                                              (int32_t *)d_leaf_box_hi);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// Encode, sort and gather external queries into Morton order.
static int prepare_queries(const zd_tree *t, const void *d_q, int64_t m, const int64_t *seg_off,
                           int64_t n_seg, Mem &mem, u64 *qkeys, int4 *q4)
{
    NvtxScope r("prepare queries");
    cudaStream_t s = mem.s;
    const int npasses = (t->key_bits + RADIX_BITS - 1) / RADIX_BITS;
    Scratch<u64> raw(mem, m);
    Scratch<int32_t> perm(mem, m);
    Scratch<u32> hist(mem, MAX_PASSES * RADIX);
    if (!raw.p || !perm.p || !hist.p) return ZD_ERR_OOM;
    ZD_CUDA(cudaMemsetAsync(hist.p, 0, MAX_PASSES * RADIX * sizeof(u32), s));
    const int cloud_shift = seg_off ? t->cloud_bit : 0;
    if (t->is_float)
        ZD_TRY(launch_encode_f32((const float *)d_q, m, t->p.dim, t->B, t->frame, seg_off, n_seg,
                                 cloud_shift, raw.p, hist.p, npasses, s));
    else
        ZD_TRY(launch_encode_i32((const int32_t *)d_q, m, t->p.dim, t->B, t->p.shift, seg_off, n_seg,
                                 cloud_shift, raw.p, hist.p, npasses, s));
    ZD_TRY(radix_sort(raw.p, m, t->key_bits, qkeys, perm.p, hist.p, mem));
    ZD_TRY(launch_gather(d_q, t->p.dim, m, perm.p, qkeys, 64, nullptr, 0, q4, s));
    return ZD_OK;
}

static int run_knn(const zd_tree *t, const int4 *q4, const u64 *qkeys, int64_t m, int k, int mode,
                   int32_t *d_idx, void *d_dist, cudaStream_t s, const int64_t *d_qoff = nullptr)
{
    NvtxScope r("search");
    const int variant = mode & (ZD_KNN_THREAD_PER_QUERY | ZD_KNN_WARP_GROUP);
    mode &= 0xff;
    KnnArgs a;
    memset(&a, 0, sizeof(a));
    a.t = view_of(t);
    a.k = k;
    a.mode = mode;
    a.allpts = q4 == nullptr;
    a.is_float = t->is_float;
    a.q = q4;
    a.qkey = qkeys;
    a.m = m;
    a.out_idx = d_idx;
    a.out_dist = d_dist;
    a.shift = make_uint3(t->p.shift[0], t->p.shift[1], t->p.shift[2]);
    // warp groups: all points, bit-based external queries, and external
    // queries of a forest (grouped per query cloud)
    const bool forest_ext = t->cloud_off && d_qoff;
    // Default mapping: warp groups for all points, and for external queries
    // that are dense relative to the tree (4m >= n); sparse queries lie far
    // apart in a group, whose shared traversal then covers much more than
    // each query needs, and one thread per query is faster (measured: 10^6
    // queries into 5*10^7 points 2.9 vs 5.5 ms; 10^7 into 10^7 13.1 vs 11.1).
    // Warp groups serve leaf-based all points and bit-based external queries;
    // all points started from the root or by key bits run one thread per
    // query (Algorithms 2 / 3 as the paper states them).  By default groups
    // run only where they were measured faster: dense query sets (above),
    // and k >= 3 -- at k <= 2 a query's own traversal is short and the
    // shared one costs more (10^7 points, k = 1: 4.8 vs 5.3 ms clustered,
    // 1.7 vs 2.5 ms on the skewed 2D set) -- or k >= 16 for integer trees
    // without exact float copies (B > 24), whose groups lack the fp32 filter.
    const bool allpts = a.allpts;
    const bool dense = allpts || 4 * m >= t->n;
    const bool k_ok = k >= 3 && (t->fpts || t->is_float || k >= 16);
    const bool group = (variant == ZD_KNN_WARP_GROUP || (variant == 0 && dense && k_ok)) &&
                       (allpts ? mode == ZD_SEARCH_LEAF
                               : ((mode == ZD_SEARCH_BIT && !t->cloud_off) || forest_ext));
    // beyond the register lists: one warp per query
    const bool wide = k > KNN_MAX_K_GROUP || (k > KNN_MAX_K_THREAD && !group);
    if (wide || !group) {
        Mem wmem = mem_of(t, s);
        Scratch<int> ctr(wmem, (size_t)sm_count()); // counters of the SM-affine query feed
        if (!ctr.p) return ZD_ERR_OOM;
        a.chunk_ctr = ctr.p;
        a.n_chunks = sm_count();
        if (wide) return launch_knn_wide(a, s); // one warp per query
        return t->is_float ? launch_knn_f32(a, s) : launch_knn_i32(a, s); // one thread per query
    }
    if (forest_ext) a.mode = ZD_SEARCH_BIT;
    Mem mem = mem_of(t, s);
    Scratch<int64_t> gpre(mem, forest_ext ? (size_t)t->n_clouds + 1 : 1);
    Scratch<int> qstart(mem, forest_ext ? (size_t)((m + 31) / 32 + t->n_clouds) : 1);
    if (!gpre.p || !qstart.p) return ZD_ERR_OOM;
    if (allpts) {
        a.group_start = t->group_start;
        a.n_groups = t->cloud_off ? t->n_groups : (t->n + 31) / 32;
    } else if (forest_ext) {
        a.n_groups = (m + 31) / 32 + t->n_clouds;
        ZD_TRY(launch_group_starts(d_qoff, t->n_clouds, a.n_groups, qstart.p, gpre.p, s));
        a.group_start = qstart.p;
        a.group_count = gpre.p + t->n_clouds;
        a.q_off = d_qoff;
    } else {
        a.n_groups = (m + 31) / 32;
    }
    // queries handed back to the exact one-thread kernel
    const int64_t nfix = allpts ? t->n : m;
    const int nch = sm_count();
    Scratch<int> fix(mem, (size_t)nfix + 1 + nch);
    if (!fix.p) return ZD_ERR_OOM;
    a.fix_count = fix.p;
    a.fix_list = fix.p + 1;
    a.chunk_ctr = fix.p + 1 + nfix;
    a.n_chunks = nch;
    if (t->is_float) return launch_knn_group_f32(a, s);
    // packed keys: the ids need idb bits
    a.idb = std::max(1, ceil_log2(t->cloud_off ? t->max_cloud : t->next_id));
    return launch_knn_group_i32(a, s);
}

extern "C" int zd_knn(const zd_tree *t, const void *d_queries, int64_t m, int k, int mode,
                      int32_t *d_idx, void *d_dist, void *stream)
{
    NvtxScope nvtx_("zd_knn");
    if (!t || !d_idx || k < 1) return ZD_ERR_INVALID_ARG;
    if (k > ZD_MAX_K) return ZD_ERR_UNIMPLEMENTED;
    if (t->cloud_off) return ZD_ERR_INVALID_ARG; // forests: zd_knn_batched
    cudaStream_t s = (cudaStream_t)stream;
    const int flags = mode & ~0xff & ~ZD_KNN_ALL_POINTS;
    if (flags & ~(ZD_KNN_THREAD_PER_QUERY | ZD_KNN_WARP_GROUP)) return ZD_ERR_INVALID_ARG;
    const int base = mode & 0xff;
    if (base != ZD_SEARCH_LEAF && base != ZD_SEARCH_BIT && base != ZD_SEARCH_ROOT) return ZD_ERR_INVALID_ARG;
    zd_tree *tw = const_cast<zd_tree *>(t); // its flat arrays are re-derived on demand
    if (base == ZD_SEARCH_LEAF || (mode & ZD_KNN_ALL_POINTS)) {
        if (d_queries) return ZD_ERR_INVALID_ARG;
        ZD_TRY(ensure_flat(tw, s));
        return run_knn(t, nullptr, nullptr, t->n, k, base | flags, d_idx, d_dist, s);
    }
    mode = base;
    if (m < 0 || (m > 0 && !d_queries)) return ZD_ERR_INVALID_ARG;
    if (m > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (m == 0) return ZD_OK;
    // after small update batches, sparse queries search the pointer form (one
    // thread per query, Algorithms 3 / 2) instead of re-deriving the flat
    // arrays; dense ones re-derive them first and run the flat searches
    const bool on_pointer_form = t->flat_stale && k <= LOCAL_MAX_K && 4 * m < t->n;
    if (!on_pointer_form) ZD_TRY(ensure_flat(tw, s));
    Mem mem = mem_of(t, s);
    Scratch<u64> qkeys(mem, m);
    Scratch<int4> q4(mem, m);
    if (!qkeys.p || !q4.p) return ZD_ERR_OOM;
    ZD_TRY(prepare_queries(t, d_queries, m, nullptr, 1, mem, qkeys.p, q4.p));
    if (on_pointer_form) ZD_TRY(local_knn(t->local, t->p.dim, q4.p, qkeys.p, m, k, mode, d_idx, d_dist, s));
    else ZD_TRY(run_knn(t, q4.p, qkeys.p, m, k, mode | flags, d_idx, d_dist, s));
    return mem.failed ? ZD_ERR_OOM : ZD_OK;
}

extern "C" int zd_knn_batched(const zd_tree *t, const void *d_queries, const int64_t *d_query_offsets,
                              int64_t m, int k, int mode_flags, int32_t *d_idx, void *d_dist, void *stream)
{
    NvtxScope nvtx_("zd_knn_batched");
    if (!t || !d_idx || k < 1) return ZD_ERR_INVALID_ARG;
    if (k > ZD_MAX_K) return ZD_ERR_UNIMPLEMENTED;
    if (!t->cloud_off) return ZD_ERR_INVALID_ARG;
    if (mode_flags & ~(ZD_KNN_THREAD_PER_QUERY | ZD_KNN_WARP_GROUP)) return ZD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!d_queries)
        return run_knn(t, nullptr, nullptr, t->n, k, ZD_SEARCH_LEAF | mode_flags, d_idx, d_dist, s);
    if (!d_query_offsets || m < 0) return ZD_ERR_INVALID_ARG;
    if (m > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (m == 0) return ZD_OK;
    Mem mem = mem_of(t, s);
    Scratch<u64> qkeys(mem, m);
    Scratch<int4> q4(mem, m);
    if (!qkeys.p || !q4.p) return ZD_ERR_OOM;
    ZD_TRY(prepare_queries(t, d_queries, m, d_query_offsets, t->n_clouds, mem, qkeys.p, q4.p));
    ZD_TRY(run_knn(t, q4.p, qkeys.p, m, k, ZD_SEARCH_ROOT | mode_flags, d_idx, d_dist, s, d_query_offsets));
    return mem.failed ? ZD_ERR_OOM : ZD_OK;
}

// --------------------------------------------------------------- updates
namespace zdk {
int update_insert(const TreeView &v, const u64 *keys, const int4 *pts, int64_t n, const void *d_pts,
                  int64_t b, int dim, int B, const uint32_t *shift, int key_bits, int32_t next_id,
                  u64 *keys_out, int4 *pts_out, u32 *live, int32_t *d_new_ids, Mem &mem, float4 *fpts_out);
int update_delete_mark(u32 *live, u32 *marked, int64_t id_cap, const int32_t *ids, int64_t b, Mem &mem,
                       int *result);
int update_delete_unmark(u32 *live, u32 *marked, int64_t id_cap, const int32_t *ids, int64_t b, cudaStream_t s);
int update_delete_compact(const u64 *keys, const int4 *pts, int64_t n, u32 *live, u32 *marked,
                          const int32_t *ids, int64_t b, int64_t id_cap, u64 *keys_out, int4 *pts_out, Mem &mem,
                          float4 *fpts_out, uint3 fsh);
int update_live_bits(u32 *live, int64_t a, int64_t z, int set, cudaStream_t s);
} // namespace zdk

// Grow the liveness bitmaps so that ids below `need` fit.
static int grow_bits(zd_tree *t, int64_t need, Mem &mem)
{
    if (need <= t->id_cap) return ZD_OK;
    const int64_t nw = std::max<int64_t>(2 * t->id_words, (need + 31) / 32);
    const size_t bytes = sizeof(u32) * (size_t)(2 * nw) + 16;
    u32 *na = (u32 *)mem.get(bytes);
    if (!na) return ZD_ERR_OOM;
    k_grow_bits<<<grid_for(2 * nw, 256, 4096), 256, 0, mem.s>>>(t->alive, t->id_words, na, nw);
    for (int i = 0; i < t->nblocks; ++i)
        if (t->blocks[i].p == t->alive) {
            mem.put(t->blocks[i].p, t->blocks[i].bytes);
            t->blocks[i] = Block{na, bytes};
        }
    t->alive = na;
    t->id_words = nw;
    t->id_cap = 32 * nw;
    return ZD_OK;
}

// Insert into the flat arrays (merge, then re-derive the tree), ids first_id..
// Validates by syncing before it commits.
static int flat_insert(zd_tree *t, const void *d_pts, int64_t b, int64_t first_id, int32_t *d_new_ids,
                       cudaStream_t s)
{
    Mem mem = mem_of(t, s);
    // the previous call's device errors must not be mistaken for this one's
    int prior = zd_check(s);
    if (prior != ZD_OK) return prior;
    // the merge writes the float copy of the merged points as well (the
    // copy has one buffer: a rejected batch restores it from the old points)
    int r = update_insert(view_of(t), t->keys, t->pts, t->n, d_pts, b, t->p.dim, t->B, t->p.shift,
                          t->key_bits, (int32_t)first_id, t->keys2, t->pts2, t->alive, d_new_ids, mem, t->fpts);
    if (r != ZD_OK) {
        if (t->fpts) launch_fpts(t->pts, t->n, t->fpts, topo_of(t).fshift, s);
        return r;
    }
    int st = zd_check(s);
    if (st != ZD_OK) {
        // nothing was committed: the new ids are released again
        update_live_bits(t->alive, first_id, first_id + b, 0, s);
        if (t->fpts) launch_fpts(t->pts, t->n, t->fpts, topo_of(t).fshift, s);
        return st;
    }
    std::swap(t->keys, t->keys2);
    std::swap(t->pts, t->pts2);
    t->n += b;
    ZD_TRY(build_topology(t->keys, t->pts, t->n, t->p.leaf_size, t->p.dim, 0, 64, topo_of(t), mem,
                          /*fpts_ready=*/t->fpts != nullptr));
    return mem.failed ? ZD_ERR_OOM : ZD_OK;
}

// Delete from the flat arrays (compact, then re-derive the tree).  Validates
// by syncing before it commits.
static int flat_delete(zd_tree *t, const int32_t *d_ids, int64_t b, cudaStream_t s)
{
    Mem mem = mem_of(t, s);
    int prior = zd_check(s);
    if (prior != ZD_OK) return prior;
    int result = ZD_OK;
    u32 *live = t->alive, *marked = t->alive + t->id_words;
    ZD_TRY(update_delete_mark(live, marked, t->id_cap, d_ids, b, mem, &result));
    if (result != ZD_OK) {
        ZD_TRY(update_delete_unmark(live, marked, t->id_cap, d_ids, b, s));
        ZD_CUDA(cudaStreamSynchronize(s));
        return result;
    }
    // validated above: the compaction writes the float copy too
    ZD_TRY(update_delete_compact(t->keys, t->pts, t->n, live, marked, d_ids, b, t->id_cap, t->keys2, t->pts2,
                                 mem, t->fpts, topo_of(t).fshift));
    std::swap(t->keys, t->keys2);
    std::swap(t->pts, t->pts2);
    t->n -= b;
    ZD_TRY(build_topology(t->keys, t->pts, t->n, t->p.leaf_size, t->p.dim, 0, 64, topo_of(t), mem,
                          /*fpts_ready=*/t->fpts != nullptr));
    int st = zd_check(s);
    if (st != ZD_OK) return st;
    return mem.failed ? ZD_ERR_OOM : ZD_OK;
}

// After small batches, re-derive the flat arrays from the pointer form
// (syncs once); then replay, in order, the updates the pointer form could not
// take (see local.cu).
static int ensure_flat(zd_tree *t, cudaStream_t s)
{
    if (!t->flat_stale) return ZD_OK;
    NvtxScope nvtx_("re-derive the flat tree");
    Mem m = mem_of(t, s);
    LocalLog log;
    int64_t n = 0;
    ZD_TRY(local_flatten(t->local, t->keys, t->pts, &n, &log, m));
    t->n = n;
    ZD_TRY(build_topology(t->keys, t->pts, n, t->p.leaf_size, t->p.dim, 0, 64, topo_of(t), m));
    t->flat_stale = false;
    if (log.n == 0) return m.failed ? ZD_ERR_OOM : ZD_OK;
    t->local_stale = true;
    const int dim = t->p.dim;
    for (int64_t i = 0; i < log.n;) {
        int64_t j = i + 1;
        if (log.op[i] == 1) { // a run of inserts with consecutive ids
            while (j < log.n && log.op[j] == 1 && log.id[j] == log.id[i] + (j - i)) ++j;
            std::vector<int32_t> h((size_t)(j - i) * dim);
            for (int64_t e = i; e < j; ++e)
                for (int c = 0; c < dim; ++c) h[(size_t)(e - i) * dim + c] = log.xyz[3 * e + c];
            Scratch<int32_t> d(m, h.size());
            if (!d.p) return ZD_ERR_OOM;
            ZD_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, s));
            ZD_TRY(flat_insert(t, d.p, j - i, log.id[i], nullptr, s)); // syncs: h outlives the copy
        } else { // a run of deletes
            while (j < log.n && log.op[j] != 1) ++j;
            Scratch<int32_t> d(m, (size_t)(j - i));
            if (!d.p) return ZD_ERR_OOM;
            ZD_CUDA(cudaMemcpyAsync(d.p, log.id.data() + i, sizeof(int32_t) * (j - i), cudaMemcpyHostToDevice, s));
            ZD_TRY(flat_delete(t, d.p, j - i, s));
        }
        i = j;
    }
    return m.failed ? ZD_ERR_OOM : ZD_OK;
}

// Before a small batch: a pointer form in step with the point set, with room
// for b more point updates and ids.
static int ensure_local(zd_tree *t, int64_t b, cudaStream_t s)
{
    if (t->local && !t->local_stale && t->local_ops + b <= LOCAL_BUDGET &&
        t->next_id + b <= local_id_slots(t->local))
        return ZD_OK;
    ZD_TRY(ensure_flat(t, s));
    Mem m = mem_of(t, s);
    ZD_TRY(local_convert(&t->local, view_of(t), t->n, t->p.leaf_size, t->next_id + LOCAL_BUDGET, m));
    t->local_stale = false;
    t->local_ops = 0;
    return m.failed ? ZD_ERR_OOM : ZD_OK;
}

extern "C" int zd_insert_batch(zd_tree *t, const void *d_pts, int64_t b, int32_t *d_new_ids, void *stream)
{
    NvtxScope nvtx_("zd_insert_batch");
    if (!t || b < 0 || (b > 0 && !d_pts)) return ZD_ERR_INVALID_ARG;
    if (t->cloud_off || t->is_float) return ZD_ERR_UNIMPLEMENTED;
    if (b == 0) return ZD_OK;
    if (t->n + b > t->cap) return ZD_ERR_CAPACITY;
    if (t->next_id + b >= ((int64_t)1 << 31) - 2) return ZD_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    Mem mem = mem_of(t, s);
    ZD_TRY(grow_bits(t, t->next_id + b, mem));
    if (b <= ZD_SMALL_BATCH) {
        ZD_TRY(ensure_local(t, b, s));
        ZD_TRY(local_insert(t->local, (const int32_t *)d_pts, b, t->p.dim, t->B, t->p.shift, (int32_t)t->next_id,
                            d_new_ids, t->alive, s));
        t->local_ops += b;
        t->next_id += b;
        t->n += b; // an upper bound until the flat arrays are re-derived
        t->flat_stale = true;
        return ZD_OK;
    }
    ZD_TRY(ensure_flat(t, s));
    t->local_stale = true;
    ZD_TRY(flat_insert(t, d_pts, b, t->next_id, d_new_ids, s));
    t->next_id += b;
    return ZD_OK;
}

extern "C" int zd_delete_batch(zd_tree *t, const int32_t *d_ids, int64_t b, void *stream)
{
    NvtxScope nvtx_("zd_delete_batch");
    if (!t || b < 0 || (b > 0 && !d_ids)) return ZD_ERR_INVALID_ARG;
    if (t->cloud_off || t->is_float) return ZD_ERR_UNIMPLEMENTED;
    if (b == 0) return ZD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (b <= ZD_SMALL_BATCH) {
        ZD_TRY(ensure_local(t, b, s));
        ZD_TRY(local_delete(t->local, d_ids, b, t->alive, t->id_cap, s));
        t->local_ops += b;
        t->flat_stale = true; // n stays an upper bound until then
        return ZD_OK;
    }
    ZD_TRY(ensure_flat(t, s));
    t->local_stale = true;
    return flat_delete(t, d_ids, b, s);
}

extern "C" int zd_knn_dist_backward(const float *d_q, const float *d_ref, const int32_t *d_idx,
                                    int64_t batch, int64_t m, int64_t r, int dim, int k,
                                    const float *d_gout, int gout_per_pair, float *d_gq,
                                    float *d_gref, void *stream)
{
    NvtxScope nvtx_("zd_knn_dist_backward");
    if (batch < 0 || m < 0 || r < 0 || k < 1 || (dim != 2 && dim != 3)) return ZD_ERR_INVALID_ARG;
    // (each factor is bounded first so that the products cannot overflow)
    if (batch > ZD_MAX_KEYS || m > ZD_MAX_KEYS || r > ZD_MAX_KEYS || k > ZD_MAX_K ||
        batch * m > ZD_MAX_KEYS || batch * m * k > ZD_MAX_KEYS || batch * r > ZD_MAX_KEYS)
        return ZD_ERR_CAPACITY;
    if (!d_gout || (batch * m > 0 && (!d_q || !d_idx || !d_gq)) || (batch * r > 0 && (!d_ref || !d_gref)))
        return ZD_ERR_INVALID_ARG;
    if (!status_word()) return ZD_ERR_CUDA;
    Mem mem;
    mem.a = nullptr;
    mem.s = (cudaStream_t)stream;
    int rr = launch_backward(d_q, d_ref, d_idx, batch, m, r, dim, k, d_gout, gout_per_pair, d_gq, d_gref,
                             mem);
    if (rr == ZD_OK && mem.failed) rr = ZD_ERR_OOM;
    return rr;
}
