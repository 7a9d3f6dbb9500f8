// knn_group_f.cuh -- the warp-group k-NN (see knn_group.cuh) for float trees:
// all points, bit-based external queries, and external queries of a forest
// (each group inside one query cloud).
//
// Neighbours are ranked exactly as the oracle ranks them: by (D, id) with
// D = ((dx*dx + dy*dy) + dz*dz) in fp64, dx = (double)q.x - (double)p.x, no
// contraction.  Each lane keeps its k best as (D, id) pairs, D held as the
// int64 bit pattern of the double (ordered like the value) so that list
// comparisons avoid the fp64 pipe.  Candidates are
// first filtered in fp32: the fp32 estimate of D carries a relative error
// below 2^-20 (two roundings of each difference and square, three of the
// sum), so a candidate with D <= thr always has estimate <= thr * (1 + 2^-18)
// rounded up; only candidates passing that test compute D in fp64.  The same
// margin guards the fp32 box tests.  The climb tests the tight box in fp64
// (the float cell of a node is not a box in coordinates).
#pragma once

#include "knn_group.cuh"

namespace zdk {

struct GroupCtxF {
    float fx, fy, fz;    // the query
    double dx, dy, dz;   // the query in fp64
    int self;            // own sorted position (all points), else -1
    bool live;
};

template <int DIM>
__device__ __forceinline__ double exact_d2(const GroupCtxF &c, float4 p)
{
    const double ex = __dsub_rn(c.dx, (double)p.x), ey = __dsub_rn(c.dy, (double)p.y);
    double s = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
    if (DIM == 3) {
        const double ez = __dsub_rn(c.dz, (double)p.z);
        s = __dadd_rn(s, __dmul_rn(ez, ez));
    }
    return s;
}

template <int DIM, int K>
__device__ __forceinline__ void accept_f(int p, float4 pt, const GroupCtxF &c, long long (&bd)[K], int (&bi)[K],
                                         float &thr_f)
{
    if (p == c.self) return;
    const long long d = __double_as_longlong(exact_d2<DIM>(c, pt));
    const int id = __float_as_int(pt.w);
    if (d < bd[K - 1] || (d == bd[K - 1] && id < bi[K - 1])) {
        kb_insert<K>(bd, bi, d, id);
        thr_f = thr_float_f(bd[K - 1]);
    }
}

template <int DIM>
__device__ __forceinline__ float est_d2(const GroupCtxF &c, float4 p)
{
    const float x = c.fx - p.x, y = c.fy - p.y, z = DIM == 3 ? c.fz - p.z : 0.f;
    return fmaf(x, x, fmaf(y, y, z * z));
}

template <int DIM, int K>
__device__ __forceinline__ void group_scan_ff(const TreeView &t, int a, int b, const GroupCtxF &c,
                                              long long (&bd)[K], int (&bi)[K], float &thr_f)
{
    const float4 *pts = (const float4 *)t.pts;
    int p = a;
    for (; p + 1 < b; p += 2) {
        const float4 u = __ldg(pts + p), v = __ldg(pts + p + 1);
        const bool pu = c.live && est_d2<DIM>(c, u) <= thr_f, pv = c.live && est_d2<DIM>(c, v) <= thr_f;
        if (__any_sync(0xffffffffu, pu || pv)) {
            if (pu) accept_f<DIM, K>(p, u, c, bd, bi, thr_f);
            if (pv) accept_f<DIM, K>(p + 1, v, c, bd, bi, thr_f);
        }
    }
    if (p < b) {
        const float4 u = __ldg(pts + p);
        const bool pu = c.live && est_d2<DIM>(c, u) <= thr_f;
        if (__any_sync(0xffffffffu, pu)) {
            if (pu) accept_f<DIM, K>(p, u, c, bd, bi, thr_f);
        }
    }
}

template <int DIM>
__device__ __forceinline__ float box_est(const GroupCtxF &c, float4 lo, float4 hi)
{
    const float cx = fmaxf(fmaxf(lo.x - c.fx, c.fx - hi.x), 0.f);
    const float cy = fmaxf(fmaxf(lo.y - c.fy, c.fy - hi.y), 0.f);
    if (DIM == 3) {
        const float cz = fmaxf(fmaxf(lo.z - c.fz, c.fz - hi.z), 0.f);
        return fmaf(cx, cx, fmaf(cy, cy, cz * cz));
    }
    return fmaf(cx, cx, cy * cy);
}

template <int DIM, int K>
__device__ __forceinline__ void group_search_ff(const TreeView &t, int start, int l0, int l1, u64 mid_key,
                                                int *stack, const GroupCtxF &c, long long (&bd)[K], int (&bi)[K],
                                                float &thr_f, u32 *status)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) stack[0] = start;
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
        const int v = stack[--sp];
        __syncwarp();
        if (v < 0 && ~v >= l0 && ~v <= l1) continue; // scanned already
        const float4 *b = (const float4 *)(v < 0 ? t.lbox + 2 * (~v) : t.ibox + 2 * v);
        const bool need = c.live && box_est<DIM>(c, __ldg(b), __ldg(b + 1)) <= thr_f;
        if (!__any_sync(0xffffffffu, need)) continue;
        if (v < 0) {
            group_scan_ff<DIM, K>(t, __ldg(t.leaf_lo + ~v), __ldg(t.leaf_lo + ~v + 1), c, bd, bi, thr_f);
            continue;
        }
        const int2 ch = __ldg(t.ichild + v);
        const bool right_first = (mid_key >> __ldg(t.ibit + v)) & 1;
        if (sp + 2 > GROUP_STACK) {
            if (lane == 0) set_status(status, ZD_ERR_CUDA);
            return;
        }
        if (lane == 0) {
            stack[sp] = right_first ? ch.x : ch.y;
            stack[sp + 1] = right_first ? ch.y : ch.x;
        }
        sp += 2;
        __syncwarp();
    }
}

template <int DIM, int K>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_group_f(KnnArgs a, u32 *status)
{
    typedef Metric<true> M;
    const TreeView &t = a.t;
    __shared__ int s_stack[KNN_THREADS / 32][GROUP_STACK];
    int *stack = s_stack[threadIdx.x >> 5];
    const int64_t g = ((int64_t)blockIdx.x * KNN_THREADS + threadIdx.x) >> 5;
    if (g >= a.n_groups || (a.group_count && g >= *a.group_count)) return; // whole warp
    const bool allpts = a.allpts;
    const int64_t nq = allpts ? t.n : a.m;
    const int g0 = a.group_start ? __ldg(a.group_start + g) : (int)(g * 32);
    int gend = (int)min((int64_t)g0 + 32, nq);
    const u64 key0 = allpts ? __ldg(t.keys + g0) : __ldg(a.qkey + g0);
    if (t.cloud_off) {
        const int64_t *off = allpts ? t.cloud_off : a.q_off;
        gend = (int)min((int64_t)gend, __ldg(off + (key0 >> t.cloud_bit) + 1));
    }
    const int lane = threadIdx.x & 31;
    const int qi = g0 + lane;
    GroupCtxF c;
    c.live = qi < gend;
    const int qs = c.live ? qi : g0;
    const int4 qp = allpts ? __ldg(t.pts + qs) : __ldg(a.q + qs);
    c.fx = __int_as_float(qp.x);
    c.fy = __int_as_float(qp.y);
    c.fz = __int_as_float(qp.z);
    c.dx = (double)c.fx;
    c.dy = (double)c.fy;
    c.dz = (double)c.fz;
    c.self = allpts && c.live ? qi : -1;
    const u64 qkey = allpts ? __ldg(t.keys + qs) : __ldg(a.qkey + qs);
    long long bd[K];
    int bi[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        bd[j] = M::inf();
        bi[j] = INT_MAX;
    }
    float thr_f = thr_float_f(M::inf());

    if (t.n > 0) {
        // 1. start leaves (consecutive, since the queries are sorted)
        int l0, l1;
        bool cloud_ok = true;
        if (allpts) {
            l0 = __ldg(t.leaf_of + g0);
            l1 = __ldg(t.leaf_of + gend - 1);
        } else {
            const int root = __ldg(t.meta) > 1 ? 0 : ~0;
            const int mine = descend_by_bits(t, root, qkey);
            l0 = __reduce_min_sync(0xffffffffu, c.live ? mine : INT_MAX);
            l1 = __reduce_max_sync(0xffffffffu, c.live ? mine : -1);
            if (t.cloud_off) {
                // the bit descent reaches the query's own cloud iff it has points
                const u64 cloud = key0 >> t.cloud_bit;
                cloud_ok = (__ldg(t.keys + __ldg(t.leaf_lo + l0)) >> t.cloud_bit) == cloud &&
                           (__ldg(t.keys + __ldg(t.leaf_lo + l1)) >> t.cloud_bit) == cloud;
            }
        }
        if (cloud_ok) {
            const int P0 = __ldg(t.leaf_lo + l0), P1 = __ldg(t.leaf_lo + l1 + 1);
            group_scan_ff<DIM, K>(t, P0, P1, c, bd, bi, thr_f);
            // 2. lowest common ancestor
            int C = ~l0;
            while (node_hi_pos(t, C) < P1) C = node_parent(t, C);
            const u64 mid_key = __shfl_sync(0xffffffffu, qkey, (gend - 1 - g0) >> 1);
            group_search_ff<DIM, K>(t, C, l0, l1, mid_key, stack, c, bd, bi, thr_f, status);
            // 3. climb: stop once every lane's ball is inside the node's tight box
            int node = C;
            int par = node_parent(t, C);
            const M::Q q = {c.dx, c.dy, c.dz};
            while (par >= 0 && __ldg(t.ibit + par) < t.cloud_bit) {
                int4 lo, hi;
                node_box(t, node, lo, hi);
                const bool inside = !c.live || M::template inside<DIM>(q, lo, hi, bd[K - 1]);
                if (__all_sync(0xffffffffu, inside)) break;
                const int2 ch = __ldg(t.ichild + par);
                group_search_ff<DIM, K>(t, ch.x == node ? ch.y : ch.x, l0, l1, mid_key, stack, c, bd, bi, thr_f,
                                        status);
                node = par;
                par = __ldg(t.iparent + par);
            }
        }
    }
    (void)lane;
    if (!c.live) return;
    int64_t row = qp.w;
    if (t.cloud_off && allpts) row += __ldg(t.cloud_off + (qkey >> t.cloud_bit));
    const int k = a.k;
    int32_t *oi = a.out_idx + row * k;
    float *od = (float *)a.out_dist;
    if (od) od += row * k;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j < k) {
            const bool have = bd[j] < M::inf();
            oi[j] = have ? bi[j] : -1;
            if (od) od[j] = have ? M::out_dist(bd[j]) : __int_as_float(0x7f800000);
        }
    }
}

template <int DIM>
int launch_knn_group_f_dim(const KnnArgs &a, cudaStream_t s)
{
    if (a.n_groups <= 0) return ZD_OK;
    const unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    u32 *st = status_word();
    if (a.k <= 1) k_knn_group_f<DIM, 1><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 2) k_knn_group_f<DIM, 2><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 4) k_knn_group_f<DIM, 4><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 5) k_knn_group_f<DIM, 5><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 8) k_knn_group_f<DIM, 8><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 10) k_knn_group_f<DIM, 10><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 16) k_knn_group_f<DIM, 16><<<g, KNN_THREADS, 0, s>>>(a, st);
    else k_knn_group_f<DIM, 32><<<g, KNN_THREADS, 0, s>>>(a, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
