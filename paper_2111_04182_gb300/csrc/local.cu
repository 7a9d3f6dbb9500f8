// local.cu -- small update batches on the pointer form of the tree
// (local.cuh), and the way back to the flat layout the searches read.
//
// A tree starts flat (the build).  The first small batch copies the flat
// tree into the pointer form (one thread per point, leaf and node; the leaf
// count is read back once); from then on every small batch is one launch of
// one thread that validates the batch on the device and applies it point by
// point -- no host round trip.  The flat layout is re-derived from the
// pointer form (every leaf copies its sorted slab to its in-order position,
// then the topology kernels of the build) before the next dense search,
// export or large batch.
//
// The pools are sized for LOCAL_BUDGET point updates; the host re-derives
// and re-copies before that is exceeded.  Only a leaf of equal keys that
// keeps growing can outrun the slab storage; then the batch kernel stops
// applying, records the rest of the batch and every later small batch in a
// log, and the host replays the log through the flat update path when it
// re-derives the flat layout.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "local.cuh"
#include "morton.cuh"

using namespace zdlocal;

namespace zdk {

constexpr int LOG_INSERT = 1, LOG_DELETE = 2;

struct LocalForm {
    LocalTree t;           // device pointers, counters at t.ctr
    int64_t loc_cap;       // ids the location array covers
    int log_cap;
    int *log_op;           // [log_cap]
    int *log_id;           // [log_cap]
    int *log_xyz;          // [log_cap * 3]
    std::vector<std::pair<void *, size_t>> blocks;
};

// ------------------------------------------------------------- flat -> pointer form
__global__ void k_lf_entries(const u64 *__restrict__ keys, const int4 *__restrict__ pts,
                             const int *__restrict__ leaf_of, const int *__restrict__ leaf_lo, int64_t n, int L,
                             u64 *skeys, P4 *spts, LLoc *loc)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int j = leaf_of[p];
        const int r = (int)(p - leaf_lo[j]);
        // leaf j's slab holds its points with room for L + 1 more
        const int64_t off = (int64_t)leaf_lo[j] + (int64_t)(L + 1) * j;
        const int4 q = pts[p];
        skeys[off + r] = keys[p];
        spts[off + r] = P4{q.x, q.y, q.z, q.w};
        loc[q.w] = LLoc{j, r};
    }
}

__global__ void k_lf_leaves(const int *__restrict__ leaf_lo, const int *__restrict__ lparent,
                            const int4 *__restrict__ lbox, const int *__restrict__ meta, int64_t max_leaves, int L,
                            LLeaf *leaves)
{
    const int nl = meta[0];
    for (int64_t jj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; jj < max_leaves;
         jj += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)jj;
        if (j >= nl) return;
        LLeaf f;
        f.parent = lparent[j];
        f.size = leaf_lo[j + 1] - leaf_lo[j];
        f.cap = f.size + L + 1;
        f.pad = 0;
        f.off = (int64_t)leaf_lo[j] + (int64_t)(L + 1) * j;
        const int4 lo = lbox[2 * j], hi = lbox[2 * j + 1];
        f.lo = P4{lo.x, lo.y, lo.z, 0};
        f.hi = P4{hi.x, hi.y, hi.z, 0};
        leaves[j] = f;
    }
}

__global__ void k_lf_nodes(const u64 *__restrict__ keys, const int2 *__restrict__ ichild,
                           const int *__restrict__ iparent, const int *__restrict__ ibit,
                           const int2 *__restrict__ irange, const int4 *__restrict__ ibox,
                           const int *__restrict__ meta, int64_t max_nodes, LNode *nodes)
{
    const int m = meta[0] - 1;
    for (int64_t ii = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ii < max_nodes;
         ii += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        if (i >= m) return;
        LNode nd;
        const int2 rg = irange[i], ch = ichild[i];
        nd.key = keys[rg.x];
        nd.left = ch.x;
        nd.right = ch.y;
        nd.parent = iparent[i];
        nd.bit = ibit[i];
        nd.size = rg.y - rg.x;
        nd.pad = 0;
        const int4 lo = ibox[2 * i], hi = ibox[2 * i + 1];
        nd.lo = P4{lo.x, lo.y, lo.z, 0};
        nd.hi = P4{hi.x, hi.y, hi.z, 0};
        nodes[i] = nd;
    }
}

__global__ void k_lf_counters(const int *meta, int64_t n, int L, LCounters *c)
{
    const int nl = n > 0 ? meta[0] : 0;
    c->root = n == 0 ? LT_EMPTY : (nl > 1 ? 0 : ~0);
    c->n_nodes = nl > 1 ? nl - 1 : 0;
    c->n_leaves = nl;
    c->count = (int)n;
    c->stor_used = n + (int64_t)(L + 1) * nl;
    c->state = 0;
    c->log_n = 0;
}

// ------------------------------------------------------------- small batches
__device__ void log_entry(LCounters *c, int log_cap, int *log_op, int *log_id, int *log_xyz, int op, int id,
                          int x, int y, int z)
{
    const int e = c->log_n;
    if (e >= log_cap) return; // the host bounds the logged updates by log_cap
    log_op[e] = op;
    log_id[e] = id;
    log_xyz[3 * e] = x;
    log_xyz[3 * e + 1] = y;
    log_xyz[3 * e + 2] = z;
    c->log_n = e + 1;
}

// One thread: insert b points (ids first_id + i).  The whole batch is
// rejected (ZD_ERR_RANGE, nothing applied) if a coordinate is out of range.
template <int DIM>
__global__ void k_lf_insert(LocalTree t, const int32_t *__restrict__ pts, int64_t b, int B, uint3 shift,
                            int32_t first_id, int32_t *new_ids, u32 *live, int log_cap, int *log_op, int *log_id,
                            int *log_xyz, u32 *status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t lim = (int64_t)1 << B;
    for (int64_t i = 0; i < b; ++i)
        for (int j = 0; j < DIM; ++j) {
            const int64_t c = (int64_t)pts[i * DIM + j] + (j == 0 ? shift.x : j == 1 ? shift.y : shift.z);
            if (c < 0 || c >= lim) {
                set_status(status, ZD_ERR_RANGE);
                return;
            }
        }
    if (new_ids)
        for (int64_t i = 0; i < b; ++i) new_ids[i] = first_id + (int32_t)i;
    LCounters *c = t.ctr;
    for (int64_t i = 0; i < b; ++i) {
        const int x = pts[i * DIM], y = pts[i * DIM + 1], z = DIM == 3 ? pts[i * DIM + 2] : 0;
        const int id = first_id + (int)i;
        if (c->state == 0) {
            const u64 key = interleave<DIM>((u64)((int64_t)x + shift.x), (u64)((int64_t)y + shift.y),
                                            (u64)((int64_t)z + (DIM == 3 ? shift.z : 0u)));
            if (insert_point(t, key, P4{x, y, z, id}) == LT_OK) {
                live[id >> 5] |= 1u << (id & 31);
                continue;
            }
            c->state = 1; // out of slab room: this and later updates go to the log
        }
        log_entry(c, log_cap, log_op, log_id, log_xyz, LOG_INSERT, id, x, y, z);
    }
}

// One thread: delete b ids.  The whole batch is rejected (nothing applied)
// if an id is not live or repeats.  Once the form has fallen back, deletes
// are logged unchecked and checked when the log is replayed.
__global__ void k_lf_delete(LocalTree t, const int32_t *__restrict__ ids, int64_t b, u32 *live, int64_t id_cap,
                            int log_cap, int *log_op, int *log_id, int *log_xyz, u32 *status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    LCounters *c = t.ctr;
    if (c->state == 0) {
        for (int64_t i = 0; i < b; ++i) {
            const int id = ids[i];
            if (id < 0 || id >= id_cap || !((live[id >> 5] >> (id & 31)) & 1)) {
                set_status(status, ZD_ERR_NOT_FOUND);
                return;
            }
            for (int64_t k = 0; k < i; ++k)
                if (ids[k] == id) {
                    set_status(status, ZD_ERR_DUPLICATE_ID);
                    return;
                }
        }
    }
    for (int64_t i = 0; i < b; ++i) {
        const int id = ids[i];
        if (c->state == 0) {
            if (delete_point(t, id) == LT_OK) {
                live[id >> 5] &= ~(1u << (id & 31));
                continue;
            }
            c->state = 1;
        }
        log_entry(c, log_cap, log_op, log_id, log_xyz, LOG_DELETE, id, 0, 0, 0);
    }
}

// ------------------------------------------------------------- searches
// k-NN of external queries on the pointer form, one thread per query, exact
// under the (squared distance, id) order: Algorithm 3 from the leaf the
// query's key bits lead to (bit-based), or Algorithm 2 from the root
// (root-based).  A node is visited iff its box distance^2 <= the current
// K-th distance^2; the climb stops once no integer point outside the current
// node's tight box can be within that distance (the node's points are the
// only points inside its box: boxes lie in the nodes' Morton cells).
template <int DIM>
__device__ __forceinline__ long long lf_d2(int4 q, P4 p)
{
    const long long dx = (long long)q.x - p.x, dy = (long long)q.y - p.y;
    long long s = dx * dx + dy * dy;
    if (DIM == 3) {
        const long long dz = (long long)q.z - p.z;
        s += dz * dz;
    }
    return s;
}

template <int DIM>
__device__ __forceinline__ long long lf_boxd2(int4 q, P4 lo, P4 hi)
{
    const long long cx = max(max((long long)lo.x - q.x, (long long)q.x - hi.x), 0ll);
    const long long cy = max(max((long long)lo.y - q.y, (long long)q.y - hi.y), 0ll);
    long long s = cx * cx + cy * cy;
    if (DIM == 3) {
        const long long cz = max(max((long long)lo.z - q.z, (long long)q.z - hi.z), 0ll);
        s += cz * cz;
    }
    return s;
}

// every integer point outside [lo, hi] is farther than sqrt(r2) from q
template <int DIM>
__device__ __forceinline__ bool lf_inside(int4 q, P4 lo, P4 hi, long long r2)
{
    if (r2 == LLONG_MAX) return false;
    const long long qq[3] = {q.x, q.y, q.z}, l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long m = min(qq[j] - l[j] + 1, h[j] + 1 - qq[j]);
        if (m <= 0 || m * m <= r2) return false;
    }
    return true;
}

template <int DIM, int K>
struct LfList {
    long long d[K];
    int id[K];
    __device__ void init()
    {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            d[j] = LLONG_MAX;
            id[j] = -1;
        }
    }
    __device__ __forceinline__ long long r2() const { return d[K - 1]; }
    __device__ __forceinline__ void offer(long long dd, int ii)
    {
        if (!(dd < d[K - 1] || (dd == d[K - 1] && (unsigned)ii < (unsigned)id[K - 1]))) return;
        bool placed = false;
#pragma unroll
        for (int j = K - 1; j > 0; --j) {
            const bool lt = dd < d[j - 1] || (dd == d[j - 1] && (unsigned)ii < (unsigned)id[j - 1]);
            if (!placed) {
                d[j] = lt ? d[j - 1] : dd;
                id[j] = lt ? id[j - 1] : ii;
            }
            placed = placed || !lt;
        }
        if (!placed) {
            d[0] = dd;
            id[0] = ii;
        }
    }
};

template <int DIM, int K>
__device__ void lf_scan_leaf(const LocalTree &t, int j, int4 q, LfList<DIM, K> &L)
{
    const LLeaf &f = t.leaves[j];
    for (int r = 0; r < f.size; ++r) {
        const P4 p = t.spts[f.off + r];
        L.offer(lf_d2<DIM>(q, p), p.w);
    }
}

// Algorithm 2 from node v
template <int DIM, int K>
__device__ void lf_search_down(const LocalTree &t, int v, int4 q, LfList<DIM, K> &L, u32 *status)
{
    int stack[LT_MAX_DEPTH];
    int sp = 0;
    stack[sp++] = v;
    while (sp) {
        const int u = stack[--sp];
        if (u < 0) {
            const LLeaf &f = t.leaves[~u];
            if (lf_boxd2<DIM>(q, f.lo, f.hi) <= L.r2()) lf_scan_leaf<DIM, K>(t, ~u, q, L);
            continue;
        }
        const LNode &nd = t.nodes[u];
        if (lf_boxd2<DIM>(q, nd.lo, nd.hi) > L.r2()) continue;
        if (sp + 2 > LT_MAX_DEPTH) {
            set_status(status, ZD_ERR_CUDA);
            return;
        }
        stack[sp++] = nd.right; // the left child is searched first
        stack[sp++] = nd.left;
    }
}

template <int DIM, int K>
__global__ void __launch_bounds__(128) k_lf_knn(LocalTree t, const int4 *__restrict__ q4,
                                                const u64 *__restrict__ qkeys, int64_t m, int k, int mode,
                                                int32_t *out_idx, long long *out_d2, u32 *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int4 q = q4[i];
        LfList<DIM, K> L;
        L.init();
        const int root = t.ctr->root;
        if (root != LT_EMPTY) {
            if (mode == ZD_SEARCH_ROOT || root < 0) {
                lf_search_down<DIM, K>(t, root, q, L, status);
            } else {
                // bit-based start: follow the key bits down to a leaf
                const u64 key = qkeys[i];
                int v = root;
                while (v >= 0) v = ((key >> t.nodes[v].bit) & 1) ? t.nodes[v].right : t.nodes[v].left;
                lf_scan_leaf<DIM, K>(t, ~v, q, L);
                // Algorithm 3: climb, searching each sibling, until the ball is inside
                int node = v;
                while (true) {
                    const P4 lo = node < 0 ? t.leaves[~node].lo : t.nodes[node].lo;
                    const P4 hi = node < 0 ? t.leaves[~node].hi : t.nodes[node].hi;
                    if (lf_inside<DIM>(q, lo, hi, L.r2())) break;
                    const int p = node < 0 ? t.leaves[~node].parent : t.nodes[node].parent;
                    if (p < 0) break;
                    const int sib = t.nodes[p].left == node ? t.nodes[p].right : t.nodes[p].left;
                    lf_search_down<DIM, K>(t, sib, q, L, status);
                    node = p;
                }
            }
        }
        int32_t *oi = out_idx + (int64_t)q.w * k;
        long long *od = out_d2 ? out_d2 + (int64_t)q.w * k : nullptr;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (j < k) {
                oi[j] = L.id[j];
                if (od) od[j] = L.d[j];
            }
    }
}

template <int DIM>
static void launch_lf_knn(const LocalTree &t, const int4 *q4, const u64 *qkeys, int64_t m, int k, int mode,
                          int32_t *idx, long long *d2, cudaStream_t s)
{
    const unsigned g = grid_for(m, 128, 152 * 64);
    u32 *st = status_word();
    if (k <= 1) k_lf_knn<DIM, 1><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
    else if (k <= 2) k_lf_knn<DIM, 2><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
    else if (k <= 4) k_lf_knn<DIM, 4><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
    else if (k <= 8) k_lf_knn<DIM, 8><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
    else if (k <= 16) k_lf_knn<DIM, 16><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
    else k_lf_knn<DIM, 32><<<g, 128, 0, s>>>(t, q4, qkeys, m, k, mode, idx, d2, st);
}

int local_knn(LocalForm *lf, int dim, const int4 *q4, const u64 *qkeys, int64_t m, int k, int mode,
              int32_t *d_idx, void *d_dist, cudaStream_t s)
{
    if (k > LOCAL_MAX_K) return ZD_ERR_INVALID_ARG;
    if (dim == 3) launch_lf_knn<3>(lf->t, q4, qkeys, m, k, mode, d_idx, (long long *)d_dist, s);
    else launch_lf_knn<2>(lf->t, q4, qkeys, m, k, mode, d_idx, (long long *)d_dist, s);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// ------------------------------------------------------------- pointer form -> flat
// The points in (key, id) order: one thread per leaf finds the leaf's first
// sorted position (leaf_position) and copies its sorted slab into place.  A
// slab longer than PLACE_THREAD entries (a leaf of equal keys) is cut into
// chunks of PLACE_CHUNK entries that whole blocks copy in a second launch.
constexpr int PLACE_THREAD = 64, PLACE_CHUNK = 2048;

struct PlaceChunk {
    int leaf, start;
    int64_t pos;
};

__global__ void k_lf_place(LocalTree t, int n_leaves, u64 *keys_out, int4 *pts_out, PlaceChunk *chunks,
                           int *n_chunks)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_leaves; j += gridDim.x * blockDim.x) {
        const LLeaf f = t.leaves[j];
        if (f.size < 0) continue; // removed from the tree
        const int64_t pos = leaf_position(t, j);
        if (f.size > PLACE_THREAD) {
            const int nc = (f.size + PLACE_CHUNK - 1) / PLACE_CHUNK;
            const int c0 = atomicAdd(n_chunks, nc);
            for (int c = 0; c < nc; ++c) chunks[c0 + c] = PlaceChunk{j, c * PLACE_CHUNK, pos + c * PLACE_CHUNK};
            continue;
        }
        for (int r = 0; r < f.size; ++r) {
            keys_out[pos + r] = t.skeys[f.off + r];
            const P4 q = t.spts[f.off + r];
            pts_out[pos + r] = make_int4(q.x, q.y, q.z, q.w);
        }
    }
}

__global__ void k_lf_place_chunks(LocalTree t, const PlaceChunk *__restrict__ chunks, const int *n_chunks,
                                  u64 *keys_out, int4 *pts_out)
{
    const int nc = *n_chunks;
    for (int e = blockIdx.x; e < nc; e += gridDim.x) {
        const PlaceChunk c = chunks[e];
        const LLeaf f = t.leaves[c.leaf];
        const int end = min(f.size - c.start, PLACE_CHUNK);
        for (int r = threadIdx.x; r < end; r += blockDim.x) {
            const int64_t src = f.off + c.start + r;
            keys_out[c.pos + r] = t.skeys[src];
            const P4 q = t.spts[src];
            pts_out[c.pos + r] = make_int4(q.x, q.y, q.z, q.w);
        }
    }
}

// ------------------------------------------------------------- host side
template <typename T>
static bool lf_alloc(LocalForm *lf, Mem &mem, T **p, size_t count)
{
    const size_t bytes = count * sizeof(T) + 16;
    *p = (T *)mem.get(bytes);
    if (!*p) return false;
    lf->blocks.push_back({(void *)*p, bytes});
    return true;
}

int64_t local_id_slots(const LocalForm *lf) { return lf ? lf->loc_cap : 0; }

void local_release(LocalForm *lf, Mem &mem)
{
    if (!lf) return;
    for (auto &b : lf->blocks) mem.put(b.first, b.second);
    delete lf;
}

int local_convert(LocalForm **out, const TreeView &v, int64_t n, int L, int64_t id_slots, Mem &mem)
{
    cudaStream_t s = mem.s;
    int nl = 0;
    if (n > 0) {
        ZD_CUDA(cudaMemcpyAsync(&nl, v.meta, sizeof(int), cudaMemcpyDeviceToHost, s));
        ZD_CUDA(cudaStreamSynchronize(s));
    }
    local_release(*out, mem);
    *out = nullptr;
    LocalForm *lf = new LocalForm();
    LocalTree &t = lf->t;
    t.L = L;
    t.node_cap = nl + LOCAL_BUDGET + 1;
    t.leaf_cap = nl + LOCAL_BUDGET + 1;
    t.stor_cap = n + (int64_t)(L + 1) * nl + (int64_t)LOCAL_BUDGET * (3 * L + 3) + LOCAL_GROW_RESERVE;
    lf->loc_cap = id_slots;
    lf->log_cap = LOCAL_BUDGET;
    bool ok = lf_alloc(lf, mem, &t.nodes, (size_t)t.node_cap) && lf_alloc(lf, mem, &t.leaves, (size_t)t.leaf_cap) &&
              lf_alloc(lf, mem, &t.skeys, (size_t)t.stor_cap) && lf_alloc(lf, mem, &t.spts, (size_t)t.stor_cap) &&
              lf_alloc(lf, mem, &t.loc, (size_t)id_slots) && lf_alloc(lf, mem, &t.ctr, 1) &&
              lf_alloc(lf, mem, &lf->log_op, (size_t)lf->log_cap) &&
              lf_alloc(lf, mem, &lf->log_id, (size_t)lf->log_cap) &&
              lf_alloc(lf, mem, &lf->log_xyz, 3 * (size_t)lf->log_cap);
    if (!ok) {
        local_release(lf, mem);
        return ZD_ERR_OOM;
    }
    if (n > 0) {
        k_lf_entries<<<grid_for(n, 256, 152 * 32), 256, 0, s>>>(v.keys, v.pts, v.leaf_of, v.leaf_lo, n, L, t.skeys,
                                                                t.spts, t.loc);
        k_lf_leaves<<<grid_for(nl, 256, 152 * 32), 256, 0, s>>>(v.leaf_lo, v.lparent, v.lbox, v.meta, nl, L,
                                                                t.leaves);
        if (nl > 1)
            k_lf_nodes<<<grid_for(nl - 1, 256, 152 * 32), 256, 0, s>>>(v.keys, v.ichild, v.iparent, v.ibit,
                                                                       v.irange, v.ibox, v.meta, nl - 1, t.nodes);
    }
    k_lf_counters<<<1, 1, 0, s>>>(v.meta, n, L, t.ctr);
    ZD_CUDA(cudaGetLastError());
    *out = lf;
    return ZD_OK;
}

int local_insert(LocalForm *lf, const int32_t *d_pts, int64_t b, int dim, int B, const uint32_t *shift,
                 int32_t first_id, int32_t *d_new_ids, u32 *live, cudaStream_t s)
{
    const uint3 sh = make_uint3(shift ? shift[0] : 0, shift ? shift[1] : 0, shift ? shift[2] : 0);
    if (dim == 3)
        k_lf_insert<3><<<1, 1, 0, s>>>(lf->t, d_pts, b, B, sh, first_id, d_new_ids, live, lf->log_cap, lf->log_op,
                                       lf->log_id, lf->log_xyz, status_word());
    else
        k_lf_insert<2><<<1, 1, 0, s>>>(lf->t, d_pts, b, B, sh, first_id, d_new_ids, live, lf->log_cap, lf->log_op,
                                       lf->log_id, lf->log_xyz, status_word());
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int local_delete(LocalForm *lf, const int32_t *d_ids, int64_t b, u32 *live, int64_t id_cap, cudaStream_t s)
{
    k_lf_delete<<<1, 1, 0, s>>>(lf->t, d_ids, b, live, id_cap, lf->log_cap, lf->log_op, lf->log_id, lf->log_xyz,
                                status_word());
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int local_flatten(LocalForm *lf, u64 *keys_out, int4 *pts_out, int64_t *n_out, LocalLog *log, Mem &mem)
{
    cudaStream_t s = mem.s;
    LCounters c;
    ZD_CUDA(cudaMemcpyAsync(&c, lf->t.ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
    ZD_CUDA(cudaStreamSynchronize(s));
    const int64_t n = c.count;
    *n_out = n;
    log->n = c.state ? c.log_n : 0;
    if (log->n > 0) {
        log->op.resize(log->n);
        log->id.resize(log->n);
        log->xyz.resize(3 * (size_t)log->n);
        ZD_CUDA(cudaMemcpyAsync(log->op.data(), lf->log_op, sizeof(int) * log->n, cudaMemcpyDeviceToHost, s));
        ZD_CUDA(cudaMemcpyAsync(log->id.data(), lf->log_id, sizeof(int) * log->n, cudaMemcpyDeviceToHost, s));
        ZD_CUDA(cudaMemcpyAsync(log->xyz.data(), lf->log_xyz, 3 * sizeof(int) * log->n, cudaMemcpyDeviceToHost, s));
        ZD_CUDA(cudaStreamSynchronize(s));
    }
    if (n == 0) return ZD_OK;
    // chunks: at most n / PLACE_CHUNK + (leaves longer than PLACE_THREAD)
    const int64_t chunk_cap = n / PLACE_CHUNK + n / (PLACE_THREAD + 1) + 1;
    Scratch<PlaceChunk> chunks(mem, chunk_cap);
    Scratch<int> n_chunks(mem, 1);
    if (!chunks.p || !n_chunks.p) return ZD_ERR_OOM;
    ZD_CUDA(cudaMemsetAsync(n_chunks.p, 0, sizeof(int), s));
    k_lf_place<<<grid_for(c.n_leaves, 256, 152 * 32), 256, 0, s>>>(lf->t, c.n_leaves, keys_out, pts_out, chunks.p,
                                                                  n_chunks.p);
    ZD_CUDA(cudaGetLastError());
    k_lf_place_chunks<<<152 * 4, 256, 0, s>>>(lf->t, chunks.p, n_chunks.p, keys_out, pts_out);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
