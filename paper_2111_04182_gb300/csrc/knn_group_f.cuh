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
// difference, three roundings in the sum, D itself within 2^-50).  Let eK be
// the K-th smallest estimate seen.  Then K candidates have
// D <= eK (1 + 2^-20), so every true neighbour has est <= B = eK (1 + 2^-18)
// -- the band.  Candidates and boxes are filtered against
// thr = eK (1 + 2^-17) rounded up (which also covers the box estimate's own
// error), and the climb stops on a lower bound of any outside point's
// estimate, so every candidate in the final band is examined.  A lane keeps
// the K smallest estimates in a min/max network and the sorted positions of
// the candidates it accepts in a shared-memory buffer (FBand, below); at the
// end the buffered candidates inside the band get their exact D (the only
// fp64 arithmetic), are ranked by (D, id), and the first k are the answer --
// near-ties and duplicates included.  Only a band larger than the buffer
// sends the query to the exact one-thread-per-query kernel.  Coordinates are
// assumed below ~1e19 in magnitude so that the fp32 squares do not overflow;
// a tiny absolute slack (1e-36) covers underflow.
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

template <int DIM>
__device__ __forceinline__ float est_d2(const GroupCtxF &c, float4 p)
{
    const float x = c.fx - p.x, y = c.fy - p.y, z = DIM == 3 ? c.fz - p.z : 0.f;
    return fmaf(x, x, fmaf(y, y, z * z));
}

template <int DIM>
__device__ __forceinline__ float box_est(const GroupCtxF &c, float4 lo, float4 hi)
{
    const float cx = fmax3(lo.x - c.fx, c.fx - hi.x, 0.f);
    const float cy = fmax3(lo.y - c.fy, c.fy - hi.y, 0.f);
    if (DIM == 3) {
        const float cz = fmax3(lo.z - c.fz, c.fz - hi.z, 0.f);
        return fmaf(cx, cx, fmaf(cy, cy, cz * cz));
    }
    return fmaf(cx, cx, cy * cy);
}

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

// FBand: the band lane of float trees (BandLane in knn_group.cuh, with the
// float bounds above): the K smallest estimates in a min/max network, the
// sorted positions it accepts in its column of the warp's shared buffer, and
// at the end the exact fp64 (D, id) ranking of the buffered candidates whose
// estimate lies in the band.  Every true neighbour has estimate <= band(eK);
// candidates and boxes are examined up to filter_thr(eK) >= band(eK), and eK
// only shrinks, so every true neighbour is in the buffer (compaction drops
// only entries above the current filter).  A lane whose band alone overflows
// the buffer goes to the exact one-thread kernel.
template <int K>
struct FBand {
    static constexpr int CAP = BandCap<K>::value;
    float e[K]; // the K smallest estimates, ascending
    float thr;  // filter of candidates and boxes
    int cnt;    // buffered candidates; above CAP: the buffer overflowed
    int *buf;   // this lane's column: entry s at buf[32 s]

    __device__ __forceinline__ void init(bool live, int *col)
    {
#pragma unroll
        for (int j = 0; j < K; ++j) e[j] = __int_as_float(0x7f800000);
        thr = live ? __int_as_float(0x7f800000) : -1.f; // a lane without a query accepts nothing
        cnt = 0;
        buf = col;
    }

    __device__ __forceinline__ void take(float est, int p)
    {
        if (cnt < CAP) buf[32 * cnt] = p;
        cnt = min(cnt + 1, CAP + 1);
#pragma unroll
        for (int j = K - 1; j > 0; --j) e[j] = fmaxf(e[j - 1], fminf(e[j], est));
        e[0] = fminf(e[0], est);
        thr = filter_thr(e[K - 1]);
    }

    // Warp-uniform: when some lane has fewer than two free entries, every
    // lane drops its entries above thr.
    template <int DIM>
    __device__ __forceinline__ void settle(const float4 *pts, const GroupCtxF &c)
    {
        if (!__any_sync(0xffffffffu, (unsigned)(cnt - (CAP - 1)) <= 1u)) return; // CAP - 1 or CAP
        if (cnt > CAP) return;
        int w = 0;
        for (int s = 0; s < cnt; ++s) {
            const int p = buf[32 * s];
            if (est_d2<DIM>(c, __ldg(pts + p)) <= thr) buf[32 * w++] = p;
        }
        cnt = w > CAP - 2 ? CAP + 1 : w; // the band alone fills it: overflow
    }

    // Sorted positions [a, b) for every lane, two candidates per step.  SELF:
    // the range may hold the lane's own point (the start leaves).
    template <int DIM, bool SELF = false>
    __device__ __forceinline__ void scan(const TreeView &t, int a, int b, const GroupCtxF &c)
    {
        const float4 *pts = (const float4 *)t.pts;
        int p = a;
        for (; p + 1 < b; p += 2) {
            const float4 u = __ldg(pts + p), v = __ldg(pts + p + 1);
            const float eu = est_d2<DIM>(c, u), ev = est_d2<DIM>(c, v);
            const bool pu = eu <= thr && (!SELF || p != c.self);
            const bool pv = ev <= thr && (!SELF || p + 1 != c.self);
            if (__any_sync(0xffffffffu, pu || pv)) {
                if (pu) take(eu, p);
                if (pv && ev <= thr) take(ev, p + 1);
                settle<DIM>(pts, c);
            }
        }
        if (p < b) {
            const float eu = est_d2<DIM>(c, __ldg(pts + p));
            const bool pu = eu <= thr && (!SELF || p != c.self);
            if (__any_sync(0xffffffffu, pu)) {
                if (pu) take(eu, p);
                settle<DIM>(pts, c);
            }
        }
    }

    // The exact ranking of the band by (D, id); false if the buffer overflowed.
    template <int DIM>
    __device__ __forceinline__ bool finish(const TreeView &t, const GroupCtxF &c, long long (&ed)[K],
                                           int (&eid)[K]) const
    {
        typedef Metric<true> M;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            ed[j] = M::inf();
            eid[j] = INT_MAX;
        }
        if (cnt > CAP) return false;
        const float4 *pts = (const float4 *)t.pts;
        const float band = band_of(e[K - 1]);
        for (int s = 0; s < cnt; ++s) {
            const float4 pt = __ldg(pts + buf[32 * s]);
            if (est_d2<DIM>(c, pt) > band) continue;
            const long long d = __double_as_longlong(exact_d2<DIM>(c, pt));
            const int id = __float_as_int(pt.w);
            if (d < ed[K - 1] || (d == ed[K - 1] && id < eid[K - 1])) kb_insert<K>(ed, eid, d, id);
        }
        return true;
    }
};

template <int DIM, int K>
__device__ __forceinline__ void group_search_ff(const TreeView &t, int start, int l0, int l1, u64 mid_key,
                                                int *stack, const GroupCtxF &c, FBand<K> &L, u32 *status)
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
            const bool need = box_est<DIM>(c, __ldg(b), __ldg(b + 1)) <= L.thr;
            if (__any_sync(0xffffffffu, need)) {
                if (v < 0) {
                    L.template scan<DIM>(t, __ldg(t.leaf_lo + ~v), __ldg(t.leaf_lo + ~v + 1), c);
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

// One group of a float tree: steps 1-3 of the group search, then the exact
// ranking of every lane's band (or the exact fallback).
template <int DIM, int K>
__device__ __forceinline__ void group_run_f(const KnnArgs &a, int64_t g, int *stack, int *band_col, u32 *status)
{
    typedef Metric<true> M;
    const TreeView &t = a.t;
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
    FBand<K> L;
    L.init(c.live, band_col);

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
            L.template scan<DIM, true>(t, P0, P1, c);
            // 2. lowest common ancestor (a node's end and parent loaded together)
            int C = ~l0;
            int hi_pos = node_hi_pos(t, C), Cp = node_parent(t, C);
            while (hi_pos < P1) {
                C = Cp;
                hi_pos = node_hi_pos(t, C);
                Cp = node_parent(t, C);
            }
            const u64 mid_key = __shfl_sync(0xffffffffu, qkey, (gend - 1 - g0) >> 1);
            group_search_ff<DIM, K>(t, C, l0, l1, mid_key, stack, c, L, status);
            // 3. climb: stop once no lane's band can reach outside the node's tight box
            int node = C;
            int par = Cp;
            while (par >= 0 && __ldg(t.ibit + par) < t.cloud_bit) {
                const int2 ch = __ldg(t.ichild + par);
                bool inside = true;
                if (c.live) {
                    const float4 *b = (const float4 *)(node < 0 ? t.lbox + 2 * (~node) : t.ibox + 2 * node);
                    const float4 lo = __ldg(b), hi = __ldg(b + 1);
                    inside = axis_clear_f(c.fx, lo.x, hi.x, L.thr) && axis_clear_f(c.fy, lo.y, hi.y, L.thr) &&
                             (DIM == 2 || axis_clear_f(c.fz, lo.z, hi.z, L.thr));
                }
                if (__all_sync(0xffffffffu, inside)) break;
                group_search_ff<DIM, K>(t, ch.x == node ? ch.y : ch.x, l0, l1, mid_key, stack, c, L, status);
                node = par;
                par = __ldg(t.iparent + par);
            }
        }
    }
    (void)lane;
    if (!c.live) return;
    // 4. the exact ranking of the band (buffer overflow: the exact kernel)
    long long ed[K];
    int eid[K];
    if (!L.template finish<DIM>(t, c, ed, eid)) {
        const int slot = atomicAdd(a.fix_count, 1);
        a.fix_list[slot] = qi;
        return;
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

// With a.chunk_ctr the launch is persistent and warps draw groups from the
// SM-affine feed (GroupFeed); without it warp w searches group w.
template <int DIM, int K>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_group_f(KnnArgs a, u32 *status)
{
    constexpr int NW = KNN_THREADS / 32;
    __shared__ int s_stack[NW][GROUP_STACK];
    __shared__ int s_band[NW][BandCap<K>::value][32];
    const int w = threadIdx.x >> 5;
    int *stack = s_stack[w];
    int *band_col = &s_band[w][0][threadIdx.x & 31];
    if (!a.chunk_ctr) {
        group_run_f<DIM, K>(a, ((int64_t)blockIdx.x * KNN_THREADS + threadIdx.x) >> 5, stack, band_col, status);
        return;
    }
    GroupFeed feed(a);
    for (int64_t g = feed.next(a, status); g >= 0; g = feed.next(a, status))
        group_run_f<DIM, K>(a, g, stack, band_col, status);
}

template <int DIM, int K>
void launch_group_f_k(const KnnArgs &a, cudaStream_t s, u32 *st)
{
    unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    if (a.chunk_ctr) g = persistent_blocks(k_knn_group_f<DIM, K>, KNN_THREADS, g, a.n_chunks);
    k_knn_group_f<DIM, K><<<g, KNN_THREADS, 0, s>>>(a, st);
}

// Launchers split by list width so that the instantiations compile in
// separate translation units (the wide lists are register-heavy).  The
// caller zeroes the feed's chunk counters and sets chunk_len.
template <int DIM>
int launch_knn_group_f_narrow(const KnnArgs &a, cudaStream_t s) // k <= 16
{
    u32 *st = status_word();
    if (a.k <= 1) launch_group_f_k<DIM, 1>(a, s, st);
    else if (a.k <= 2) launch_group_f_k<DIM, 2>(a, s, st);
    else if (a.k <= 4) launch_group_f_k<DIM, 4>(a, s, st);
    else if (a.k <= 5) launch_group_f_k<DIM, 5>(a, s, st);
    else if (a.k <= 8) launch_group_f_k<DIM, 8>(a, s, st);
    else if (a.k <= 10) launch_group_f_k<DIM, 10>(a, s, st);
    else if (a.k <= 12) launch_group_f_k<DIM, 12>(a, s, st);
    else launch_group_f_k<DIM, 16>(a, s, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

template <int DIM>
int launch_knn_group_f_wide(const KnnArgs &a, cudaStream_t s) // 16 < k <= 40
{
    u32 *st = status_word();
    if (a.k <= 24) launch_group_f_k<DIM, 24>(a, s, st);
    else if (a.k <= 28) launch_group_f_k<DIM, 28>(a, s, st);
    else if (a.k <= 32) launch_group_f_k<DIM, 32>(a, s, st);
    else launch_group_f_k<DIM, 40>(a, s, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
