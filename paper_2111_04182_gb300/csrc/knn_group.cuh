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
// The answer of a lane is its k best as 64-bit keys (d^2 << idb) | id, so the
// order of keys is the order (d^2, id).  How a lane gets there depends on the
// tree: with exact float copies of the coordinates (B <= 24) it ranks
// candidates by fp32 estimates during the walk and ranks only the final band
// exactly (BandLane, below); otherwise it inserts every candidate that beats
// its k-th d^2 into the packed list (ExactLane).  d^2 saturates at
// sat = 2^(64-idb) - 1, and a lane never searches beyond d^2 = sat - 1: its
// threshold starts there and stays there while its k-th entry is missing or
// saturated, so a lane whose neighbours lie that far (sparse outskirts of
// skewed data) does not drag the whole group through the tree.  A query that
// ends with a missing or saturated entry among its first k is handed to the
// exact one-thread-per-query kernel.
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

// Float bound of an integer threshold: every candidate with d^2 <= thr has
// a float estimate (three roundings of nonnegative terms) <= thr (1 + 2^-24)^3
// < the returned value.
__device__ __forceinline__ float thr_float(long long thr)
{
    if (thr == LLONG_MAX) return __int_as_float(0x7f800000);
    return __fmul_ru(__ll2float_ru(thr), 1.0f + 1.0f / 1048576.0f);
}

// max(a, b, c) in one instruction (three-operand max.f32, sm_100 and later);
// exact, like two fmaxf.
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int DIM>
__device__ __forceinline__ float box_d2f(const GroupCtx &c, float4 lo, float4 hi)
{
    const float cx = fmax3(lo.x - c.fx, c.fx - hi.x, 0.f);
    const float cy = fmax3(lo.y - c.fy, c.fy - hi.y, 0.f);
    if (DIM == 3) {
        const float cz = fmax3(lo.z - c.fz, c.fz - hi.z, 0.f);
        return fmaf(cx, cx, fmaf(cy, cy, cz * cz));
    }
    return fmaf(cx, cx, cy * cy);
}

// Float estimate of a candidate's d^2 from the exact float copies: the
// differences are exact, the sum rounds at most three times.
template <int DIM>
__device__ __forceinline__ float est_d2f(const GroupCtx &c, float4 p)
{
    const float x = c.fx - p.x, y = c.fy - p.y, z = DIM == 3 ? c.fz - p.z : 0.f;
    return fmaf(x, x, fmaf(y, y, z * z));
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

template <int DIM>
__device__ __forceinline__ long long exact_d2i(const GroupCtx &c, int4 p)
{
    const int dx = c.qx - p.x, dy = c.qy - p.y;
    long long d2 = (long long)dx * dx + (long long)dy * dy;
    if (DIM == 3) {
        const int dz = c.qz - p.z;
        d2 += (long long)dz * dz;
    }
    return d2;
}

// Margin test on one axis: the first integer outside [lo, hi] is more than
// sqrt(thr) away from q.
__device__ __forceinline__ bool axis_inside(long long q, long long lo, long long hi, long long thr)
{
    const long long m = min(q - lo + 1, hi + 1 - q);
    return m > 0 && m * m > thr;
}

// What a lane learns from a node: whether it may hold a closer point, and
// the node's sorted positions [a, b) (a leaf) or its children (a, b).
struct Probe {
    bool need;
    int a, b;
    int bit; // an internal node's split bit
};

// ------------------------------------------------------------------------
// ExactLane: the k best as packed keys (d^2 << idb) | id, exact int64 d^2
// for every candidate.  Trees whose coordinates do not fit fp32 (B > 24).
template <int K>
struct ExactLane {
    u64 key[K];
    long long thr; // the lane's search radius^2 (thr_of)

    __device__ __forceinline__ void init(const GroupCtx &c, int *)
    {
#pragma unroll
        for (int j = 0; j < K; ++j) key[j] = ~0ull;
        thr = (long long)(c.sat - 1);
    }
    __device__ __forceinline__ long long climb_thr() const { return thr; }

    template <int DIM>
    __device__ __forceinline__ Probe probe(const TreeView &t, int v, const GroupCtx &c) const
    {
        int4 lo, hi;
        node_box(t, v, lo, hi);
        Probe r;
        r.need = c.live && box_d2<DIM>(c, lo, hi) <= thr;
        if (v < 0) {
            r.a = __ldg(t.leaf_lo + ~v);
            r.b = __ldg(t.leaf_lo + ~v + 1);
        } else {
            const int2 ch = __ldg(t.ichild + v);
            r.a = ch.x;
            r.b = ch.y;
        }
        r.bit = v >= 0 ? __ldg(t.ibit + v) : 0;
        return r;
    }

    template <int DIM, bool SELF = false>
    __device__ __forceinline__ void scan(const TreeView &t, int a, int b, const GroupCtx &c)
    {
        for (int p = a; p < b; ++p) {
            const int4 pt = __ldg(t.pts + p);
            const long long d2 = exact_d2i<DIM>(c, pt);
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

    template <int DIM>
    __device__ __forceinline__ bool finish(const TreeView &, const GroupCtx &, u64 (&out)[K]) const
    {
#pragma unroll
        for (int j = 0; j < K; ++j) out[j] = key[j];
        return true;
    }
};

// ------------------------------------------------------------------------
// BandLane: trees with exact float copies (B <= 24).  The walk never touches
// int64: a lane keeps only the K smallest fp32 estimates e[] it has seen (a
// min/max network, no payload to move) and appends the sorted position of
// every candidate it accepts to its column of the warp's shared buffer.
//
// Exactness.  With u = 2^-24, an estimate lies in [D (1-u)^3, D (1+u)^3] for
// the exact d^2 = D (2D: squares of u).  K distinct candidates have estimate
// <= eK = e[K-1], so the true K-th distance is <= eK / (1-u)^3 and every true
// neighbour (ties by id included) has estimate <= eK (1+u)^3 / (1-u)^3 <
// eK (1 + 2^-20) <= band.  Candidates are accepted while their estimate is
// <= thr = eK (1 + 2^-19) rounded up; a box is pruned when its (exact-input)
// estimate exceeds thr, which puts every point inside above
// thr (1 - 6.1u) > band; the climb stops when every point outside the node
// has D > ceil(thr), i.e. estimate > band.  eK only shrinks, so every true
// neighbour is accepted when it is examined.  At the end the buffered
// candidates whose estimate is <= band get their exact int64 d^2 and are
// ranked by (d^2, id); the first k are the answer.
//
// thr never exceeds cap, the bound of d^2 = sat - 1 (a lane does not search
// beyond the packed-key limit; see the saturation rule at the top).  A full
// buffer is compacted, for every lane at once, to the entries still <= thr
// (those above are no neighbours); a lane whose buffer stays full is handed
// to the exact one-thread kernel.
template <int K>
struct BandCap { // buffered candidates per lane
    static constexpr int value = K + 12 > 24 ? K + 12 : 24;
};

template <int K>
struct BandLane {
    static constexpr int CAP = BandCap<K>::value;
    float e[K];  // the K smallest estimates, ascending
    float thr;   // filter of candidates and boxes
    float cap;   // thr <= cap
    int cnt;     // buffered candidates; above CAP: the buffer overflowed (exact fallback)
    int *buf;    // this lane's column: entry s at buf[32 s]

    __device__ __forceinline__ void init(const GroupCtx &c, int *col)
    {
#pragma unroll
        for (int j = 0; j < K; ++j) e[j] = __int_as_float(0x7f800000);
        cap = thr_float((long long)(c.sat - 1));
        thr = c.live ? cap : -1.f; // a lane without a query accepts nothing
        cnt = 0;
        buf = col;
    }
    __device__ __forceinline__ long long climb_thr() const { return __float2ll_ru(thr); }

    template <int DIM>
    __device__ __forceinline__ Probe probe(const TreeView &t, int v, const GroupCtx &c) const
    {
        // the float boxes carry the leaf range / the children in w
        const float4 *fb = v < 0 ? t.flbox + 2 * (~v) : t.fibox + 2 * v;
        const float4 lo = __ldg(fb), hi = __ldg(fb + 1);
        Probe r;
        r.bit = v >= 0 ? __ldg(t.ibit + v) : 0; // issued beside the box loads
        r.need = box_d2f<DIM>(c, lo, hi) <= thr;
        r.a = __float_as_int(lo.w);
        r.b = __float_as_int(hi.w);
        return r;
    }

    __device__ __forceinline__ void take(float est, int p)
    {
        if (cnt < CAP) buf[32 * cnt] = p;
        cnt = min(cnt + 1, CAP + 1);
#pragma unroll
        for (int j = K - 1; j > 0; --j) e[j] = fmaxf(e[j - 1], fminf(e[j], est));
        e[0] = fminf(e[0], est);
        thr = fminf(__fmul_ru(e[K - 1], 1.0f + 1.0f / 524288.0f), cap);
    }

    // Warp-uniform: when some lane has fewer than two free entries, every
    // lane drops its entries above thr.
    template <int DIM>
    __device__ __forceinline__ void settle(const TreeView &t, const GroupCtx &c)
    {
        if (!__any_sync(0xffffffffu, (unsigned)(cnt - (CAP - 1)) <= 1u)) return; // CAP - 1 or CAP
        if (cnt > CAP) return;
        int w = 0;
        for (int s = 0; s < cnt; ++s) {
            const int p = buf[32 * s];
            if (est_d2f<DIM>(c, __ldg(t.fpts + p)) <= thr) buf[32 * w++] = p;
        }
        cnt = w > CAP - 2 ? CAP + 1 : w; // the band alone fills it: overflow
    }

    // Sorted positions [a, b) for every lane, two candidates per step.  SELF:
    // the range may hold the lane's own point (the group's start leaves; the
    // searches skip those).
    template <int DIM, bool SELF = false>
    __device__ __forceinline__ void scan(const TreeView &t, int a, int b, const GroupCtx &c)
    {
        int p = a;
        for (; p + 1 < b; p += 2) {
            const float4 u = __ldg(t.fpts + p), v = __ldg(t.fpts + p + 1);
            const float eu = est_d2f<DIM>(c, u), ev = est_d2f<DIM>(c, v);
            const bool pu = eu <= thr && (!SELF || p != c.self);
            const bool pv = ev <= thr && (!SELF || p + 1 != c.self);
            if (__any_sync(0xffffffffu, pu || pv)) {
                if (pu) take(eu, p);
                if (pv && ev <= thr) take(ev, p + 1);
                settle<DIM>(t, c);
            }
        }
        if (p < b) {
            const float eu = est_d2f<DIM>(c, __ldg(t.fpts + p));
            const bool pu = eu <= thr && (!SELF || p != c.self);
            if (__any_sync(0xffffffffu, pu)) {
                if (pu) take(eu, p);
                settle<DIM>(t, c);
            }
        }
    }

    // The exact ranking of the band; false if the buffer overflowed.
    template <int DIM>
    __device__ __forceinline__ bool finish(const TreeView &t, const GroupCtx &c, u64 (&out)[K]) const
    {
#pragma unroll
        for (int j = 0; j < K; ++j) out[j] = ~0ull;
        if (cnt > CAP) return false;
        const float band = __fmul_ru(e[K - 1], 1.0f + 1.0f / 1048576.0f);
        for (int s = 0; s < cnt; ++s) {
            const int p = buf[32 * s];
            if (est_d2f<DIM>(c, __ldg(t.fpts + p)) > band) continue;
            const int4 pt = __ldg(t.pts + p);
            const long long d2 = exact_d2i<DIM>(c, pt);
            const u64 df = (u64)d2 < c.sat ? (u64)d2 : c.sat;
            const u64 ck = (df << c.idb) | (u64)(unsigned)pt.w;
            if (ck < out[K - 1]) key_insert<K>(out, ck);
        }
        return true;
    }
};

template <int K, bool BAND>
struct LaneOf {
    typedef ExactLane<K> type;
};
template <int K>
struct LaneOf<K, true> {
    typedef BandLane<K> type;
};

// searchDown (Algorithm 2) for the whole group from `start`, skipping the
// leaves l0..l1 scanned already; the stack lives in shared memory and every
// lane holds the same stack pointer.  Children are pushed in the order of the
// group's middle key (the side of the split it lies on goes first).
template <int DIM, class Lane>
__device__ __forceinline__ void group_search(const TreeView &t, int start, int l0, int l1, u64 mid_key,
                                             int *stack, const GroupCtx &c, Lane &L, u32 *status)
{
    const int lane = threadIdx.x & 31;
    int sp = 0;
    int v = start;
    while (true) {
        if (!ZD_DCHECK(node_in_range(t, v), status)) return;
        // the nearer child is searched next directly; the farther one waits
        // on the stack (lane 0 writes it, every lane holds the same pointer)
        if (!(v < 0 && ~v >= l0 && ~v <= l1)) { // else scanned already
            const Probe pr = L.template probe<DIM>(t, v, c);
            if (__any_sync(0xffffffffu, pr.need)) {
                if (v < 0) {
                    L.template scan<DIM>(t, pr.a, pr.b, c);
                } else {
                    const bool right_first = (mid_key >> pr.bit) & 1;
                    if (sp + 1 > GROUP_STACK) {
                        if (lane == 0) set_status(status, ZD_ERR_CUDA);
                        return;
                    }
                    if (lane == 0) stack[sp] = right_first ? pr.a : pr.b; // the far child waits
                    ++sp;
                    __syncwarp();
                    v = right_first ? pr.b : pr.a;
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
template <int DIM, class Lane>
__device__ __forceinline__ void group_traverse(const TreeView &t, const KnnArgs &a, const GroupCtx &c, Lane &L,
                                               int g0, int gend, bool allpts, int *stack, u32 *status)
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
    L.template scan<DIM, true>(t, P0, P1, c);

    // 2. their lowest common ancestor (a node's end and parent loaded together)
    int C = ~l0;
    int hi_pos = node_hi_pos(t, C), Cp = node_parent(t, C);
    while (hi_pos < P1) {
        C = Cp;
        hi_pos = node_hi_pos(t, C);
        Cp = node_parent(t, C);
    }
    const u64 mid_key = __shfl_sync(0xffffffffu, c.qkey, (gend - 1 - g0) >> 1);
    group_search<DIM>(t, C, l0, l1, mid_key, stack, c, L, status);

    // 3. climb (Algorithm 3) until no lane can improve from outside the node
    int node = C;
    int par = Cp;
    while (par >= 0) {
        const int pbit = __ldg(t.ibit + par); // the parent's fields, loaded together
        const int2 ch = __ldg(t.ichild + par);
        if (pbit >= t.cloud_bit) break; // never leave the cloud
        bool inside = true;
        if (c.live) {
            const long long thr = L.climb_thr();
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
        group_search<DIM>(t, ch.x == node ? ch.y : ch.x, l0, l1, mid_key, stack, c, L, status);
        node = par;
        par = __ldg(t.iparent + par);
    }
}

// One group: steps 1-3, then the answer of every lane (or the exact fallback).
template <int DIM, int K, bool BAND>
__device__ __forceinline__ void group_run(const KnnArgs &a, int64_t g, int *stack, int *band_col, u32 *status)
{
    typedef typename LaneOf<K, BAND>::type Lane;
    const TreeView &t = a.t;
    if (g >= a.n_groups || (a.group_count && g >= *a.group_count)) return; // whole warp
    const int lane = threadIdx.x & 31;
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
    Lane L;
    L.init(c, band_col);

    if (t.n > 0) group_traverse<DIM>(t, a, c, L, g0, gend, allpts, stack, status);

    if (!c.live) return;
    const int k = a.k;
    u64 key[K];
    bool saturated = !L.template finish<DIM>(t, c, key);
    // an entry among the first k that is missing (empty slots read as
    // saturated) or saturated: exact fallback
#pragma unroll
    for (int j = 0; j < K; ++j) // static indices keep the list in registers
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

// BAND: the tree has exact float copies (BandLane), else ExactLane.  With
// a.chunk_ctr the launch is persistent and warps draw groups from the
// SM-affine feed; without it warp w searches group w.
template <int DIM, int K, bool BAND>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_group(KnnArgs a, u32 *status)
{
    constexpr int NW = KNN_THREADS / 32;
    __shared__ int s_stack[NW][GROUP_STACK];
    __shared__ int s_band[BAND ? NW : 1][BAND ? BandCap<K>::value : 1][32];
    const int w = threadIdx.x >> 5;
    int *stack = s_stack[w];
    int *band_col = &s_band[BAND ? w : 0][0][threadIdx.x & 31];
    if (!a.chunk_ctr) {
        group_run<DIM, K, BAND>(a, ((int64_t)blockIdx.x * KNN_THREADS + threadIdx.x) >> 5, stack, band_col, status);
        return;
    }
    GroupFeed feed(a);
    for (int64_t g = feed.next(a, status); g >= 0; g = feed.next(a, status))
        group_run<DIM, K, BAND>(a, g, stack, band_col, status);
}

template <int DIM, int K, bool BAND>
void launch_group_kb(const KnnArgs &a, unsigned g, cudaStream_t s, u32 *st)
{
    if (a.chunk_ctr) g = persistent_blocks(k_knn_group<DIM, K, BAND>, KNN_THREADS, g, a.n_chunks);
    k_knn_group<DIM, K, BAND><<<g, KNN_THREADS, 0, s>>>(a, st);
}

template <int DIM, int K>
void launch_group_k(const KnnArgs &a, unsigned g, cudaStream_t s, u32 *st)
{
    if (a.t.fpts) launch_group_kb<DIM, K, true>(a, g, s, st);
    else launch_group_kb<DIM, K, false>(a, g, s, st);
}

template <int DIM>
int launch_knn_group_dim(const KnnArgs &a, cudaStream_t s)
{
    if (a.n_groups <= 0) return ZD_OK;
    const unsigned g = (unsigned)((a.n_groups * 32 + KNN_THREADS - 1) / KNN_THREADS);
    u32 *st = status_word();
    KnnArgs b = a;
    if (b.chunk_ctr) {
        ZD_CUDA(cudaMemsetAsync(b.chunk_ctr, 0, sizeof(int) * (size_t)b.n_chunks, s));
        b.chunk_len = (b.n_groups + b.n_chunks - 1) / b.n_chunks;
    }
    if (a.k <= 1) launch_group_k<DIM, 1>(b, g, s, st);
    else if (a.k <= 2) launch_group_k<DIM, 2>(b, g, s, st);
    else if (a.k <= 4) launch_group_k<DIM, 4>(b, g, s, st);
    else if (a.k <= 5) launch_group_k<DIM, 5>(b, g, s, st);
    else if (a.k <= 8) launch_group_k<DIM, 8>(b, g, s, st);
    else if (a.k <= 10) launch_group_k<DIM, 10>(b, g, s, st);
    else if (a.k <= 12) launch_group_k<DIM, 12>(b, g, s, st);
    else if (a.k <= 16) launch_group_k<DIM, 16>(b, g, s, st);
    else if (a.k <= 24) launch_group_k<DIM, 24>(b, g, s, st);
    else if (a.k <= 28) launch_group_k<DIM, 28>(b, g, s, st);
    else if (a.k <= 32) launch_group_k<DIM, 32>(b, g, s, st);
    else launch_group_k<DIM, 40>(b, g, s, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
