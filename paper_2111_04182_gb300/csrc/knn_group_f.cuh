// knn_group_f.cuh -- the warp-group k-NN (see knn_group.cuh) for float trees:
// all points, bit-based external queries, and external queries of a forest
// (each group inside one query cloud).
//
// Neighbours are ranked exactly as the oracle ranks them: by (D, id) with
// D = ((dx*dx + dy*dy) + dz*dz) in fp64, dx = (double)q.x - (double)p.x, no
// contraction.  GB300's fp64 pipe is narrow, so the traversal never touches
// it: each lane ranks candidates by the fp32 estimate
//   est = fma(x, x, fma(y, y, z*z)),  x = fl32(q.x - p.x), ...
// whose relative error against D is below 2^-20 (one rounding of each
// difference, three roundings in the sum, D itself within 2^-50), and keeps
// the K + FSLACK smallest (est, sorted position) in registers as packed u64
// keys.  Let eK be the K-th smallest estimate seen.  Then K candidates have
// D <= eK (1 + 2^-20), so every true neighbour has est <= B = eK (1 + 2^-18)
// -- the band.  Candidates and boxes are filtered against
// thr = eK (1 + 2^-17) rounded up (which also covers the box estimate's own
// error), and the climb stops on a lower bound of any outside point's
// estimate, so every candidate in the final band is examined.  A candidate
// that passes the filter but is not kept (or is evicted later) records its
// estimate in ovf; if ovf <= B at the end, the band overflowed the list
// (near-ties, duplicates) and the query is handed to the exact
// one-thread-per-query kernel.  Otherwise the band lies in the list: its
// entries get their exact D (the only fp64 arithmetic, <= K + FSLACK
// evaluations per query), are sorted by (D, id), and the first k are the
// answer.  Coordinates are assumed below ~1e19 in magnitude so that the fp32
// squares do not overflow; a tiny absolute slack (1e-36) covers underflow.
#pragma once

#include "knn_group.cuh"

namespace zdk {

constexpr int FSLACK = 2; // list entries kept beyond K

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

template <int DIM>
__device__ __forceinline__ float est_d2(const GroupCtxF &c, float4 p)
{
    const float x = c.fx - p.x, y = c.fy - p.y, z = DIM == 3 ? c.fz - p.z : 0.f;
    return fmaf(x, x, fmaf(y, y, z * z));
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

// Estimate of a packed key (empty slots read as NaN, which no test accepts).
__device__ __forceinline__ float key_est(u64 key) { return __uint_as_float((unsigned)(key >> 32)); }

// Filter threshold from the K-th estimate: eK (1 + 2^-17) + 1e-36, rounded up.
__device__ __forceinline__ float filter_thr(float eK)
{
    if (!(eK < __int_as_float(0x7f800000))) return __int_as_float(0x7f800000);
    return __fadd_ru(__fmul_ru(eK, 1.0f + 1.0f / 131072.0f), 1e-36f);
}

// The band bound B: eK (1 + 2^-18) + 1e-36, rounded up.
__device__ __forceinline__ float band_of(float eK)
{
    if (!(eK < __int_as_float(0x7f800000))) return __int_as_float(0x7f800000);
    return __fadd_ru(__fmul_ru(eK, 1.0f + 1.0f / 262144.0f), 1e-36f);
}

template <int K>
struct EstList {
    static constexpr int KP = K + FSLACK;
    u64 key[KP]; // (est bits << 32) | sorted position, ascending
    float ovf;   // smallest estimate that passed the filter but is not kept
    float thr;   // filter / pruning threshold

    __device__ void init()
    {
#pragma unroll
        for (int j = 0; j < KP; ++j) key[j] = ~0ull;
        ovf = __int_as_float(0x7f800000);
        thr = ovf;
    }
    __device__ __forceinline__ void offer(float est, int p)
    {
        const u64 ck = ((u64)__float_as_uint(est) << 32) | (u64)(unsigned)p;
        if (ck < key[KP - 1]) {
            ovf = fminf(ovf, key_est(key[KP - 1])); // NaN (empty slot) leaves ovf alone
            key_insert<KP>(key, ck);
            thr = filter_thr(key_est(key[K - 1]));
        } else {
            ovf = fminf(ovf, est);
        }
    }
};

// Scan sorted positions [a, b) for every lane, two candidates per step.
template <int DIM, int K>
__device__ __forceinline__ void group_scan_ff(const TreeView &t, int a, int b, const GroupCtxF &c, EstList<K> &L)
{
    const float4 *pts = (const float4 *)t.pts;
    int p = a;
    for (; p + 1 < b; p += 2) {
        const float4 u = __ldg(pts + p), v = __ldg(pts + p + 1);
        const float eu = est_d2<DIM>(c, u), ev = est_d2<DIM>(c, v);
        const bool pu = c.live && eu <= L.thr && p != c.self;
        const bool pv = c.live && ev <= L.thr && p + 1 != c.self;
        if (__any_sync(0xffffffffu, pu || pv)) {
            if (pu) L.offer(eu, p);
            if (pv && ev <= L.thr) L.offer(ev, p + 1);
        }
    }
    if (p < b) {
        const float4 u = __ldg(pts + p);
        const float eu = est_d2<DIM>(c, u);
        const bool pu = c.live && eu <= L.thr && p != c.self;
        if (__any_sync(0xffffffffu, pu)) {
            if (pu) L.offer(eu, p);
        }
    }
}

template <int DIM, int K>
__device__ __forceinline__ void group_search_ff(const TreeView &t, int start, int l0, int l1, u64 mid_key,
                                                int *stack, const GroupCtxF &c, EstList<K> &L, u32 *status)
{
    const int lane = threadIdx.x & 31;
    int sp = 0;
    int v = start;
    while (true) {
        if (!ZD_DCHECK(node_in_range(t, v), status)) return;
        // the nearer child is searched next directly; the farther one waits
        // on the stack (lane 0 writes it, every lane holds the same pointer)
        if (!(v < 0 && ~v >= l0 && ~v <= l1)) { // else scanned already
            const float4 *b = (const float4 *)(v < 0 ? t.lbox + 2 * (~v) : t.ibox + 2 * v);
            const bool need = c.live && box_est<DIM>(c, __ldg(b), __ldg(b + 1)) <= L.thr;
            if (__any_sync(0xffffffffu, need)) {
                if (v < 0) {
                    group_scan_ff<DIM, K>(t, __ldg(t.leaf_lo + ~v), __ldg(t.leaf_lo + ~v + 1), c, L);
                } else {
                    const int2 ch = __ldg(t.ichild + v);
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

// Climb test on one axis: every point outside [lo, hi] along it has an
// estimate above thr.  m <= (true gap)(1 + 2^-24); ml = m (1 - 2^-22) rounded
// down is at most the true gap g, and an outside point's estimate is at least
// g^2 (1 - 2^-21) >= ml^2 (1 - 2^-20) with both products rounded down.
__device__ __forceinline__ bool axis_clear_f(float q, float lo, float hi, float thr)
{
    const float m = fminf(q - lo, hi - q);
    if (!(m >= 0.f)) return false;
    const float ml = __fmul_rd(m, 1.0f - 1.0f / 4194304.0f);
    return __fmul_rd(__fmul_rd(ml, ml), 1.0f - 1.0f / 1048576.0f) > thr;
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
    EstList<K> L;
    L.init();

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
            group_scan_ff<DIM, K>(t, P0, P1, c, L);
            // 2. lowest common ancestor
            int C = ~l0;
            while (node_hi_pos(t, C) < P1) C = node_parent(t, C);
            const u64 mid_key = __shfl_sync(0xffffffffu, qkey, (gend - 1 - g0) >> 1);
            group_search_ff<DIM, K>(t, C, l0, l1, mid_key, stack, c, L, status);
            // 3. climb: stop once no lane's band can reach outside the node's tight box
            int node = C;
            int par = node_parent(t, C);
            while (par >= 0 && __ldg(t.ibit + par) < t.cloud_bit) {
                bool inside = true;
                if (c.live) {
                    const float4 *b = (const float4 *)(node < 0 ? t.lbox + 2 * (~node) : t.ibox + 2 * node);
                    const float4 lo = __ldg(b), hi = __ldg(b + 1);
                    inside = axis_clear_f(c.fx, lo.x, hi.x, L.thr) && axis_clear_f(c.fy, lo.y, hi.y, L.thr) &&
                             (DIM == 2 || axis_clear_f(c.fz, lo.z, hi.z, L.thr));
                }
                if (__all_sync(0xffffffffu, inside)) break;
                const int2 ch = __ldg(t.ichild + par);
                group_search_ff<DIM, K>(t, ch.x == node ? ch.y : ch.x, l0, l1, mid_key, stack, c, L, status);
                node = par;
                par = __ldg(t.iparent + par);
            }
        }
    }
    (void)lane;
    if (!c.live) return;
    // 4. the band must lie in the list, else the exact kernel takes the query
    if (L.ovf <= band_of(key_est(L.key[K - 1]))) {
        const int slot = atomicAdd(a.fix_count, 1);
        a.fix_list[slot] = qi;
        return;
    }
    // 5. exact D of the kept candidates, sorted by (D, id)
    constexpr int KP = EstList<K>::KP;
    long long ed[KP];
    int eid[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        ed[j] = M::inf();
        eid[j] = INT_MAX;
    }
    const float4 *pts = (const float4 *)t.pts;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        if (L.key[j] != ~0ull) {
            const float4 pt = __ldg(pts + (int)(unsigned)(L.key[j] & 0xffffffffu));
            kb_insert<KP>(ed, eid, __double_as_longlong(exact_d2<DIM>(c, pt)), __float_as_int(pt.w));
        }
    }
    int64_t row = qp.w;
    if (t.cloud_off && allpts) row += __ldg(t.cloud_off + (qkey >> t.cloud_bit));
    const int k = a.k;
    int32_t *oi = a.out_idx + row * k;
    float *od = (float *)a.out_dist;
    if (od) od += row * k;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j < k) {
            const bool have = ed[j] < M::inf();
            oi[j] = have ? eid[j] : -1;
            if (od) od[j] = have ? M::out_dist(ed[j]) : __int_as_float(0x7f800000);
        }
    }
}

// Launchers split by list width so that the instantiations compile in
// separate translation units (the wide lists are register-heavy).
template <int DIM>
int launch_knn_group_f_narrow(const KnnArgs &a, cudaStream_t s) // k <= 16
{
    const unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    u32 *st = status_word();
    if (a.k <= 1) k_knn_group_f<DIM, 1><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 2) k_knn_group_f<DIM, 2><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 4) k_knn_group_f<DIM, 4><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 5) k_knn_group_f<DIM, 5><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 8) k_knn_group_f<DIM, 8><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 10) k_knn_group_f<DIM, 10><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 12) k_knn_group_f<DIM, 12><<<g, KNN_THREADS, 0, s>>>(a, st);
    else k_knn_group_f<DIM, 16><<<g, KNN_THREADS, 0, s>>>(a, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

template <int DIM>
int launch_knn_group_f_wide(const KnnArgs &a, cudaStream_t s) // 16 < k <= 40
{
    const unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    u32 *st = status_word();
    if (a.k <= 24) k_knn_group_f<DIM, 24><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 28) k_knn_group_f<DIM, 28><<<g, KNN_THREADS, 0, s>>>(a, st);
    else if (a.k <= 32) k_knn_group_f<DIM, 32><<<g, KNN_THREADS, 0, s>>>(a, st);
    else k_knn_group_f<DIM, 40><<<g, KNN_THREADS, 0, s>>>(a, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
