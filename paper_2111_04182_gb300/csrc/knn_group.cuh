// knn_group.cuh -- k-NN with one warp per group of 32 consecutive queries in
// Morton order (integer coordinates): all-points (leaf-based) and external
// bit-based queries.
//
// Lane l owns query g0 + l.  The warp walks ONE traversal for the whole group
// -- Algorithm 3 generalised from a leaf to a group: scan the group's start
// leaves (for all points: the leaves of the group's own points; for external
// queries: the leaves the queries' Morton bits lead to, which are consecutive
// because the queries are sorted), search down their lowest common ancestor C
// (Algorithm 2, skipping the leaves already scanned), then climb from C,
// searching each sibling, until no lane can have a closer point outside the
// current node.  A node is visited iff some lane's box distance^2 is <= that
// lane's k-th distance^2 (ballot), so every lane visits a superset of what
// its own Algorithm 3 would visit and gets the same exact k-NN; in exchange,
// control flow is warp-uniform and every candidate point is loaded once per
// warp (a broadcast) instead of once per lane.
//
// Each lane keeps its k best as 64-bit keys (d^2 << idb) | id, so the order of
// keys is the order (d^2, id) and an insertion step is one 64-bit compare.
// Candidates are first filtered on the plain d^2 against the lane's k-th d^2;
// only survivors are packed.  d^2 saturates at sat = 2^(64-idb) - 1, and a
// lane never searches beyond d^2 = sat - 1: its threshold starts there and
// stays there while its k-th entry is missing or saturated, so a lane whose
// neighbours lie that far (sparse outskirts of skewed data) does not drag
// the whole group through the tree.  A query that ends with a missing or
// saturated entry among its first k is handed to the exact
// one-thread-per-query kernel.
//
// The climb stops on the node's Morton cell -- the box of all coordinates
// whose keys share the node's prefix, which contains every point the node can
// hold -- rather than its tight box: a point outside the node lies outside
// its cell, so if every lane's k-th ball is inside the cell with integer
// margin, nothing above can improve any lane (same answer, earlier stop).
// All-points queries lie in their own cells; external queries use the cell
// only when their key carries the node's prefix, else the tight box.
#pragma once

#include "knn_impl.cuh"

namespace zdk {

constexpr int GROUP_STACK = 96;

__device__ __forceinline__ int node_hi_pos(const TreeView &t, int v)
{
    return v < 0 ? __ldg(t.leaf_lo + ~v + 1) : __ldg(t.irange + v).y;
}
__device__ __forceinline__ int node_lo_pos(const TreeView &t, int v)
{
    return v < 0 ? __ldg(t.leaf_lo + ~v) : __ldg(t.irange + v).x;
}
__device__ __forceinline__ int node_parent(const TreeView &t, int v)
{
    return v < 0 ? __ldg(t.lparent + ~v) : __ldg(t.iparent + v);
}

template <int K>
__device__ __forceinline__ void key_insert(u64 (&key)[K], u64 c)
{
    bool placed = false;
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        const bool lt = c < key[j - 1];
        if (!placed) key[j] = lt ? key[j - 1] : c;
        placed = placed || !lt;
    }
    if (!placed) key[0] = c;
}

struct GroupCtx {
    int qx, qy, qz;
    float fx, fy, fz;    // the shifted coordinates as exact floats
    int self;            // sorted position to skip (all-points), else -1
    bool live;           // the lane has a query
    int idb;             // id bits of the packed key
    u64 sat;             // saturated d^2 field
    u64 qkey;            // the query's Morton key (shifted coordinates)
    unsigned sx, sy, sz; // shift
};

// Search radius^2 of a lane: its k-th d^2, or sat - 1 while that entry is
// missing or saturated.
template <int K>
__device__ __forceinline__ long long thr_of(const u64 (&key)[K], const GroupCtx &c)
{
    const u64 d = key[K - 1] >> c.idb;
    return d >= c.sat ? (long long)(c.sat - 1) : (long long)d;
}

// Float filter threshold: every candidate with d^2 <= thr computes (three
// roundings of nonnegative terms) a float d^2 <= thr * (1 + 2^-24)^3 <
// thr_f, so the filter never drops a true candidate.
__device__ __forceinline__ float thr_float(long long thr)
{
    if (thr == LLONG_MAX) return __int_as_float(0x7f800000);
    return __fmul_ru(__ll2float_ru(thr), 1.0f + 1.0f / 1048576.0f);
}

template <int DIM>
__device__ __forceinline__ float box_d2f(const GroupCtx &c, float4 lo, float4 hi)
{
    const float cx = fmaxf(fmaxf(lo.x - c.fx, c.fx - hi.x), 0.f);
    const float cy = fmaxf(fmaxf(lo.y - c.fy, c.fy - hi.y), 0.f);
    if (DIM == 3) {
        const float cz = fmaxf(fmaxf(lo.z - c.fz, c.fz - hi.z), 0.f);
        return fmaf(cx, cx, fmaf(cy, cy, cz * cz));
    }
    return fmaf(cx, cx, cy * cy);
}

template <int DIM>
__device__ __forceinline__ long long box_d2(const GroupCtx &c, int4 lo, int4 hi)
{
    const int cx = max(max(lo.x - c.qx, c.qx - hi.x), 0);
    const int cy = max(max(lo.y - c.qy, c.qy - hi.y), 0);
    long long s = (long long)cx * cx + (long long)cy * cy;
    if (DIM == 3) {
        const int cz = max(max(lo.z - c.qz, c.qz - hi.z), 0);
        s += (long long)cz * cz;
    }
    return s;
}

// Margin test on one axis: the first integer outside [lo, hi] is more than
// sqrt(thr) away from q.
__device__ __forceinline__ bool axis_inside(long long q, long long lo, long long hi, long long thr)
{
    const long long m = min(q - lo + 1, hi + 1 - q);
    return m > 0 && m * m > thr;
}

// Scan sorted positions [a, b) for every lane.
template <int DIM, int K>
__device__ __forceinline__ void group_scan(const TreeView &t, int a, int b, const GroupCtx &c,
                                           u64 (&key)[K], long long &thr)
{
    for (int p = a; p < b; ++p) {
        const int4 pt = __ldg(t.pts + p);
        const int dx = c.qx - pt.x, dy = c.qy - pt.y;
        long long d2 = (long long)dx * dx + (long long)dy * dy;
        if (DIM == 3) {
            const int dz = c.qz - pt.z;
            d2 += (long long)dz * dz;
        }
        const bool pre = c.live && d2 <= thr && p != c.self;
        if (__any_sync(0xffffffffu, pre)) {
            if (pre) {
                const u64 df = (u64)d2 < c.sat ? (u64)d2 : c.sat;
                const u64 ck = (df << c.idb) | (u64)(unsigned)pt.w;
                if (ck < key[K - 1]) {
                    key_insert<K>(key, ck);
                    thr = thr_of<K>(key, c);
                }
            }
        }
    }
}

// Exact test of one candidate that passed the float filter: the float
// differences are exact integers, so the int64 d^2 is exact.
template <int DIM, int K>
__device__ __forceinline__ void accept_exact(int p, float dxf, float dyf, float dzf, int id,
                                             const GroupCtx &c, u64 (&key)[K], long long &thr, float &thr_f)
{
    if (p == c.self) return;
    const int dx = __float2int_rn(dxf), dy = __float2int_rn(dyf);
    long long d2 = (long long)dx * dx + (long long)dy * dy;
    if (DIM == 3) {
        const int dz = __float2int_rn(dzf);
        d2 += (long long)dz * dz;
    }
    if (d2 > thr) return;
    const u64 df = (u64)d2 < c.sat ? (u64)d2 : c.sat;
    const u64 ck = (df << c.idb) | (u64)(unsigned)id;
    if (ck < key[K - 1]) {
        key_insert<K>(key, ck);
        thr = thr_of<K>(key, c);
        thr_f = thr_float(thr);
    }
}

// Scan sorted positions [a, b) on the float copy, two candidates per step.
template <int DIM, int K>
__device__ __forceinline__ void group_scan_f(const TreeView &t, int a, int b, const GroupCtx &c,
                                             u64 (&key)[K], long long &thr, float &thr_f)
{
    int p = a;
    for (; p + 1 < b; p += 2) {
        const float4 u = __ldg(t.fpts + p), v = __ldg(t.fpts + p + 1);
        const float ux = c.fx - u.x, uy = c.fy - u.y, uz = DIM == 3 ? c.fz - u.z : 0.f;
        const float vx = c.fx - v.x, vy = c.fy - v.y, vz = DIM == 3 ? c.fz - v.z : 0.f;
        const float du = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float dv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
        const bool pu = c.live && du <= thr_f, pv = c.live && dv <= thr_f;
        if (__any_sync(0xffffffffu, pu || pv)) {
            if (pu) accept_exact<DIM, K>(p, ux, uy, uz, __float_as_int(u.w), c, key, thr, thr_f);
            if (pv) accept_exact<DIM, K>(p + 1, vx, vy, vz, __float_as_int(v.w), c, key, thr, thr_f);
        }
    }
    if (p < b) {
        const float4 u = __ldg(t.fpts + p);
        const float ux = c.fx - u.x, uy = c.fy - u.y, uz = DIM == 3 ? c.fz - u.z : 0.f;
        const float du = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const bool pu = c.live && du <= thr_f;
        if (__any_sync(0xffffffffu, pu)) {
            if (pu) accept_exact<DIM, K>(p, ux, uy, uz, __float_as_int(u.w), c, key, thr, thr_f);
        }
    }
}

// searchDown (Algorithm 2) for the whole group from `start`, skipping the
// leaves l0..l1 scanned already; the stack lives in shared memory and every
// lane holds the same stack pointer.  Children are pushed in the order of the
// group's middle key (the side of the split it lies on goes first).
template <int DIM, int K, bool FS>
__device__ __forceinline__ void group_search(const TreeView &t, int start, int l0, int l1, u64 mid_key,
                                             int *stack, const GroupCtx &c, u64 (&key)[K], long long &thr,
                                             float &thr_f, u32 *status)
{
    const int lane = threadIdx.x & 31;
    int sp = 0;
    int v = start;
    while (true) {
        if (!ZD_DCHECK(node_in_range(t, v), status)) return;
        // the nearer child is searched next directly; the farther one waits
        // on the stack (lane 0 writes it, every lane holds the same pointer)
        if (!(v < 0 && ~v >= l0 && ~v <= l1)) { // else scanned already
            bool need;
            float4 flo, fhi;
            if (FS) {
                const float4 *fb = v < 0 ? t.flbox + 2 * (~v) : t.fibox + 2 * v;
                flo = __ldg(fb);
                fhi = __ldg(fb + 1);
                need = c.live && box_d2f<DIM>(c, flo, fhi) <= thr_f;
            } else {
                int4 lo, hi;
                node_box(t, v, lo, hi);
                need = c.live && box_d2<DIM>(c, lo, hi) <= thr;
            }
            if (__any_sync(0xffffffffu, need)) {
                if (v < 0) {
                    if (FS) {
                        group_scan_f<DIM, K>(t, __float_as_int(flo.w), __float_as_int(fhi.w), c, key, thr, thr_f);
                    } else {
                        const int a = __ldg(t.leaf_lo + ~v), b = __ldg(t.leaf_lo + ~v + 1);
                        group_scan<DIM, K>(t, a, b, c, key, thr);
                    }
                } else {
                    const int2 ch = FS ? make_int2(__float_as_int(flo.w), __float_as_int(fhi.w)) : __ldg(t.ichild + v);
                    const bool right_first = (mid_key >> __ldg(t.ibit + v)) & 1;
                    if (sp + 1 > GROUP_STACK) {
                        if (lane == 0) set_status(status, ZD_ERR_CUDA);
                        return;
                    }
                    if (lane == 0) stack[sp] = right_first ? ch.x : ch.y; // the far child waits
                    ++sp;
                    __syncwarp();
                    v = right_first ? ch.y : ch.x;
                    continue;
                }
            }
        }
        if (sp == 0) break;
        v = stack[--sp];
        __syncwarp();
    }
}

// Leaf that the bit-based descent of Sec. 2 reaches for `key`.
__device__ __forceinline__ int descend_by_bits(const TreeView &t, int root, u64 key)
{
    int v = root;
    while (v >= 0) {
        const int2 ch = __ldg(t.ichild + v);
        v = ((key >> __ldg(t.ibit + v)) & 1) ? ch.y : ch.x;
    }
    return ~v;
}

// Steps 1-3 of the group search (see the top of this file).
template <int DIM, int K, bool FS>
__device__ __forceinline__ void group_traverse(const TreeView &t, const KnnArgs &a, const GroupCtx &c,
                                               u64 (&key)[K], long long &thr, float &thr_f, int g0, int gend,
                                               bool allpts, int *stack, u32 *status)
{
    // 1. the start leaves: consecutive in leaf order, since queries are sorted
    int l0, l1;
    if (allpts) {
        l0 = __ldg(t.leaf_of + g0);
        l1 = __ldg(t.leaf_of + gend - 1);
    } else {
        const int root = __ldg(t.meta) > 1 ? 0 : ~0;
        const int mine = descend_by_bits(t, root, c.qkey);
        l0 = __reduce_min_sync(0xffffffffu, c.live ? mine : INT_MAX);
        l1 = __reduce_max_sync(0xffffffffu, c.live ? mine : -1);
    }
    if (t.cloud_off && !allpts) {
        // the bit descent reaches the query's own cloud iff that cloud has points
        const u64 cloud = __shfl_sync(0xffffffffu, c.qkey, 0) >> t.cloud_bit;
        if ((__ldg(t.keys + __ldg(t.leaf_lo + l0)) >> t.cloud_bit) != cloud ||
            (__ldg(t.keys + __ldg(t.leaf_lo + l1)) >> t.cloud_bit) != cloud)
            return;
    }
    if (!ZD_DCHECK(l0 >= 0 && l0 <= l1 && node_in_range(t, ~l1), status)) return;
    const int P0 = __ldg(t.leaf_lo + l0), P1 = __ldg(t.leaf_lo + l1 + 1);
    if (FS) group_scan_f<DIM, K>(t, P0, P1, c, key, thr, thr_f);
    else group_scan<DIM, K>(t, P0, P1, c, key, thr);

    // 2. their lowest common ancestor
    int C = ~l0;
    while (node_hi_pos(t, C) < P1) C = node_parent(t, C);
    const u64 mid_key = __shfl_sync(0xffffffffu, c.qkey, (gend - 1 - g0) >> 1);
    group_search<DIM, K, FS>(t, C, l0, l1, mid_key, stack, c, key, thr, thr_f, status);

    // 3. climb (Algorithm 3) until no lane can improve from outside the node
    int node = C;
    int par = node_parent(t, C);
    while (par >= 0) {
        const int pbit = __ldg(t.ibit + par);
        if (pbit >= t.cloud_bit) break; // never leave the cloud
        bool inside = true;
        if (c.live) {
            // the node's cell: key bits >= pbit are the node's prefix
            const bool in_cell = allpts || ((c.qkey ^ __ldg(t.keys + node_lo_pos(t, node))) >> pbit) == 0;
            if (in_cell) {
                inside = cell_inside<DIM>(make_int4(c.qx, c.qy, c.qz, 0), make_uint3(c.sx, c.sy, c.sz), pbit,
                                          thr);
            } else {
                int4 lo, hi;
                node_box(t, node, lo, hi);
                inside = axis_inside(c.qx, lo.x, hi.x, thr) && axis_inside(c.qy, lo.y, hi.y, thr) &&
                         (DIM == 2 || axis_inside(c.qz, lo.z, hi.z, thr));
            }
        }
        if (__all_sync(0xffffffffu, inside)) break;
        const int2 ch = __ldg(t.ichild + par);
        group_search<DIM, K, FS>(t, ch.x == node ? ch.y : ch.x, l0, l1, mid_key, stack, c, key, thr, thr_f,
                                 status);
        node = par;
        par = __ldg(t.iparent + par);
    }
}

template <int DIM, int K, bool FS>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_group(KnnArgs a, u32 *status)
{
    const TreeView &t = a.t;
    __shared__ int s_stack[KNN_THREADS / 32][GROUP_STACK];
    int *stack = s_stack[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * KNN_THREADS + threadIdx.x) >> 5;
    if (g >= a.n_groups || (a.group_count && g >= *a.group_count)) return; // whole warp
    const bool allpts = a.allpts;
    const int64_t nq = allpts ? t.n : a.m;
    // the group: 32 consecutive queries in Morton order, never across clouds
    const int g0 = a.group_start ? __ldg(a.group_start + g) : (int)(g * 32);
    int gend = (int)min((int64_t)g0 + 32, nq);
    if (t.cloud_off) {
        const u64 key0 = allpts ? __ldg(t.keys + g0) : __ldg(a.qkey + g0);
        const int64_t *off = allpts ? t.cloud_off : a.q_off;
        gend = (int)min((int64_t)gend, __ldg(off + (key0 >> t.cloud_bit) + 1));
    }
    const int qi = g0 + lane;
    GroupCtx c;
    c.live = qi < gend;
    const int qs = c.live ? qi : g0;
    const int4 qp = allpts ? __ldg(t.pts + qs) : __ldg(a.q + qs);
    c.qx = qp.x;
    c.qy = qp.y;
    c.qz = qp.z;
    // the float copies hold shifted coordinates (exact: c + shift < 2^24)
    c.fx = (float)((unsigned)qp.x + a.shift.x);
    c.fy = (float)((unsigned)qp.y + a.shift.y);
    c.fz = (float)((unsigned)qp.z + a.shift.z);
    c.self = allpts && c.live ? qi : -1;
    c.idb = a.idb;
    c.sat = (1ull << (64 - a.idb)) - 1ull;
    c.qkey = allpts ? __ldg(t.keys + qs) : __ldg(a.qkey + qs);
    c.sx = a.shift.x;
    c.sy = a.shift.y;
    c.sz = a.shift.z;
    u64 key[K];
#pragma unroll
    for (int j = 0; j < K; ++j) key[j] = ~0ull;
    long long thr = (long long)(c.sat - 1);
    float thr_f = thr_float(thr);

    if (t.n > 0) group_traverse<DIM, K, FS>(t, a, c, key, thr, thr_f, g0, gend, allpts, stack, status);
    (void)lane;

    if (!c.live) return;
    const int k = a.k;
    // an entry among the first k that is missing (empty slots read as
    // saturated) or saturated: exact fallback
    bool saturated = false; // static indices keep the list in registers
#pragma unroll
    for (int j = 0; j < K; ++j)
        saturated = saturated || (j < k && (key[j] >> c.idb) >= c.sat);
    if (saturated) {
        const int slot = atomicAdd(a.fix_count, 1);
        a.fix_list[slot] = qi;
        return;
    }
    int64_t row = qp.w;
    if (t.cloud_off && allpts) row += __ldg(t.cloud_off + (c.qkey >> t.cloud_bit));
    int32_t *oi = a.out_idx + row * k;
    long long *od = (long long *)a.out_dist;
    if (od) od += row * k;
    const u64 idmask = (1ull << c.idb) - 1ull;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j < k) {
            const bool have = key[j] != ~0ull;
            oi[j] = have ? (int32_t)(key[j] & idmask) : -1;
            if (od) od[j] = have ? (long long)(key[j] >> c.idb) : LLONG_MAX;
        }
    }
}

template <int DIM, int K>
void launch_group_k(const KnnArgs &a, unsigned g, cudaStream_t s, u32 *st)
{
    if (a.t.fpts) k_knn_group<DIM, K, true><<<g, KNN_THREADS, 0, s>>>(a, st);
    else k_knn_group<DIM, K, false><<<g, KNN_THREADS, 0, s>>>(a, st);
}

template <int DIM>
int launch_knn_group_dim(const KnnArgs &a, cudaStream_t s)
{
    if (a.n_groups <= 0) return ZD_OK;
    const unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    u32 *st = status_word();
    if (a.k <= 1) launch_group_k<DIM, 1>(a, g, s, st);
    else if (a.k <= 2) launch_group_k<DIM, 2>(a, g, s, st);
    else if (a.k <= 4) launch_group_k<DIM, 4>(a, g, s, st);
    else if (a.k <= 5) launch_group_k<DIM, 5>(a, g, s, st);
    else if (a.k <= 8) launch_group_k<DIM, 8>(a, g, s, st);
    else if (a.k <= 10) launch_group_k<DIM, 10>(a, g, s, st);
    else if (a.k <= 12) launch_group_k<DIM, 12>(a, g, s, st);
    else if (a.k <= 16) launch_group_k<DIM, 16>(a, g, s, st);
    else if (a.k <= 24) launch_group_k<DIM, 24>(a, g, s, st);
    else if (a.k <= 28) launch_group_k<DIM, 28>(a, g, s, st);
    else if (a.k <= 32) launch_group_k<DIM, 32>(a, g, s, st);
    else launch_group_k<DIM, 40>(a, g, s, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
