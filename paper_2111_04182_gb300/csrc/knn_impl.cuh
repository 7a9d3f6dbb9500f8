// knn_impl.cuh -- exact k-NN over the zd-tree (Algorithms 2 and 3).
//
// One thread per query; queries run in Morton order (Sec. 3.1: sorting the
// queries makes neighbouring threads touch the same nodes, so a warp's loads
// hit the same cache lines).  Each thread keeps its k best candidates in
// registers, sorted by (squared distance, id) -- the total order that makes
// ties have one answer -- and walks the tree with an explicit stack:
//
//   leaf-based / bit-based (Algorithm 3): scan the start leaf (all points:
//     the point's own leaf, or the leaf its key bits lead to from the root;
//     external queries: the leaf their key bits lead to), then climb; at each
//     ancestor, stop once no point outside the current node's box can be
//     within the k-th distance, else search the sibling downwards.
//   root-based (Algorithm 2): search down from the root.
// For all points (a.allpts) the queries are the tree's own points in sorted
// order and each excludes itself, whichever of the three starts is used.
//
// searchDown visits a node iff its box distance^2 <= the current k-th
// distance^2 (non-strict, so an equal distance with a smaller id is never
// pruned) and descends into the nearer child first.  A child's box distance
// is computed once, when its parent is expanded, and kept on the stack; a
// popped entry is re-tested against the k-th distance, which may have shrunk.
#pragma once

#include <algorithm>
#include <atomic>
#include <climits>

#include "common.cuh"

namespace zdk {

constexpr int KNN_THREADS = 128;
constexpr int KNN_STACK = 72; // depth <= 64 internal levels + slack

template <bool FLOAT>
struct Metric;

// Integer coordinates: exact int64 squared distances.  Coordinate
// differences fit in int32 because every coordinate lies in one window of
// width 2^B, B <= 31.
template <>
struct Metric<false> {
    typedef long long D;
    struct Q {
        int x, y, z;
    };
    __device__ static D inf() { return LLONG_MAX; }
    __device__ static float out_dist(D) { return 0.f; } // integer trees report d^2
    __device__ static Q make(int4 p) { return Q{p.x, p.y, p.z}; }
    template <int DIM>
    __device__ static D dist(const Q &q, int4 p)
    {
        int dx = q.x - p.x, dy = q.y - p.y;
        D s = (D)dx * dx + (D)dy * dy;
        if (DIM == 3) {
            int dz = q.z - p.z;
            s += (D)dz * dz;
        }
        return s;
    }
    template <int DIM>
    __device__ static D boxd(const Q &q, int4 lo, int4 hi)
    {
        int cx = max(max(lo.x - q.x, q.x - hi.x), 0);
        int cy = max(max(lo.y - q.y, q.y - hi.y), 0);
        D s = (D)cx * cx + (D)cy * cy;
        if (DIM == 3) {
            int cz = max(max(lo.z - q.z, q.z - hi.z), 0);
            s += (D)cz * cz;
        }
        return s;
    }
    // No integer point outside [lo, hi] can be within thr: in every
    // dimension the first coordinate outside the box (lo-1 or hi+1) is
    // farther than sqrt(thr) from q.
    template <int DIM>
    __device__ static bool inside(const Q &q, int4 lo, int4 hi, D thr)
    {
        if (thr == inf()) return false;
        long long m;
        m = min((long long)q.x - lo.x + 1, (long long)hi.x + 1 - q.x);
        if (m <= 0 || m * m <= thr) return false;
        m = min((long long)q.y - lo.y + 1, (long long)hi.y + 1 - q.y);
        if (m <= 0 || m * m <= thr) return false;
        if (DIM == 3) {
            m = min((long long)q.z - lo.z + 1, (long long)hi.z + 1 - q.z);
            if (m <= 0 || m * m <= thr) return false;
        }
        return true;
    }
};

// Float coordinates: the ranking value is an fp64 squared distance evaluated
// as ((dx*dx + dy*dy) + dz*dz), dx = (double)q.x - (double)p.x, each
// operation rounded to nearest with no contraction.  The value travels as
// the bit pattern of the (non-negative) double read as an int64: for
// non-negative doubles and +inf the patterns are ordered like the values, so
// every comparison runs on the integer pipe, not the much narrower fp64 one.
template <>
struct Metric<true> {
    typedef long long D;
    struct Q {
        double x, y, z;
    };
    __device__ static D inf() { return 0x7ff0000000000000ll; }
    __device__ static D bits(double v) { return __double_as_longlong(v); }
    __device__ static float out_dist(D d) { return (float)sqrt(__longlong_as_double(d)); }
    __device__ static Q make(int4 p)
    {
        return Q{(double)__int_as_float(p.x), (double)__int_as_float(p.y), (double)__int_as_float(p.z)};
    }
    template <int DIM>
    __device__ static D dist(const Q &q, int4 p)
    {
        double dx = __dsub_rn(q.x, (double)__int_as_float(p.x));
        double dy = __dsub_rn(q.y, (double)__int_as_float(p.y));
        double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        if (DIM == 3) {
            double dz = __dsub_rn(q.z, (double)__int_as_float(p.z));
            s = __dadd_rn(s, __dmul_rn(dz, dz));
        }
        return bits(s);
    }
    // Distance from q to [lo, hi] along one axis: l - q if q < l, q - h if
    // q > h, else 0 (a rounded difference of distinct doubles is never 0, so
    // its sign decides the case).
    __device__ static double gap(double q, float lo, float hi)
    {
        const double a = __dsub_rn((double)lo, q), b = __dsub_rn(q, (double)hi);
        return bits(a) > 0 ? a : (bits(b) > 0 ? b : 0.0);
    }
    template <int DIM>
    __device__ static D boxd(const Q &q, int4 lo, int4 hi)
    {
        double cx = gap(q.x, __int_as_float(lo.x), __int_as_float(hi.x));
        double cy = gap(q.y, __int_as_float(lo.y), __int_as_float(hi.y));
        double s = __dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy));
        if (DIM == 3) {
            double cz = gap(q.z, __int_as_float(lo.z), __int_as_float(hi.z));
            s = __dadd_rn(s, __dmul_rn(cz, cz));
        }
        return bits(s);
    }
    // A point outside the box in dimension j differs from q by more than the
    // gap m_j to that face; rounding is monotone, so its ranking value is at
    // least fl(m_j^2).  Stop iff fl(m_j^2) > thr in every dimension.
    __device__ static bool side_ok(double q, float lo, float hi, D thr)
    {
        const double a = __dsub_rn(q, (double)lo), b = __dsub_rn((double)hi, q);
        const D ab = bits(a), bb = bits(b);
        if (ab < 0 || bb < 0) return false; // outside the box (or -0): no stop
        const double m = ab < bb ? a : b;
        return bits(__dmul_rn(m, m)) > thr;
    }
    template <int DIM>
    __device__ static bool inside(const Q &q, int4 lo, int4 hi, D thr)
    {
        if (!(thr < inf())) return false;
        if (!side_ok(q.x, __int_as_float(lo.x), __int_as_float(hi.x), thr)) return false;
        if (!side_ok(q.y, __int_as_float(lo.y), __int_as_float(hi.y), thr)) return false;
        if (DIM == 3 && !side_ok(q.z, __int_as_float(lo.z), __int_as_float(hi.z), thr)) return false;
        return true;
    }
};

// fp32 threshold for the candidate filter of float trees: the fp32 estimate
// of D carries a relative error below 2^-20 (two roundings of each
// difference and square, three of the sum), so a candidate with D <= thr
// always has estimate <= thr * (1 + 2^-18), rounded up.  thr: bit pattern.
__device__ __forceinline__ float thr_float_f(long long thr)
{
    if (thr >= 0x7ff0000000000000ll) return __int_as_float(0x7f800000);
    return __fmul_ru(__double2float_ru(__longlong_as_double(thr)), 1.0f + 1.0f / 262144.0f);
}

// Candidate filter before the exact distance: nothing for integer trees; for
// float trees an fp32 estimate against the margin threshold above, which
// skips the fp64 evaluation of candidates that cannot enter the list.
template <bool FLOAT>
struct Prefilter {
    __device__ explicit Prefilter(int4) {}
    template <int DIM>
    __device__ bool pass(int4) const { return true; }
    __device__ void update(long long) {}
};
template <>
struct Prefilter<true> {
    float x, y, z, thr;
    __device__ explicit Prefilter(int4 q)
    {
        x = __int_as_float(q.x);
        y = __int_as_float(q.y);
        z = __int_as_float(q.z);
        thr = __int_as_float(0x7f800000);
    }
    template <int DIM>
    __device__ bool pass(int4 p) const
    {
        const float ex = x - __int_as_float(p.x), ey = y - __int_as_float(p.y);
        const float ez = DIM == 3 ? z - __int_as_float(p.z) : 0.f;
        return fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= thr;
    }
    __device__ void update(long long kth) { thr = thr_float_f(kth); }
};

// Insert (d, id) into the sorted k-best list (the caller checked that it
// beats the current k-th entry).  Fully unrolled, so the list stays in
// registers.
template <int K, typename D>
__device__ __forceinline__ void kb_insert(D (&bd)[K], int (&bi)[K], D d, int id)
{
    bool placed = false;
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        const bool lt = d < bd[j - 1] || (d == bd[j - 1] && id < bi[j - 1]);
        if (!placed) {
            bd[j] = lt ? bd[j - 1] : d;
            bi[j] = lt ? bi[j - 1] : id;
        }
        placed = placed || !lt;
    }
    if (!placed) {
        bd[0] = d;
        bi[0] = id;
    }
}

template <int DIM, int K, bool FLOAT>
__device__ __forceinline__ void scan_leaf(const TreeView &t, int leaf, int self,
                                          const typename Metric<FLOAT>::Q &q, Prefilter<FLOAT> &pf,
                                          typename Metric<FLOAT>::D (&bd)[K], int (&bi)[K])
{
    typedef Metric<FLOAT> M;
    const int lo = __ldg(t.leaf_lo + leaf), hi = __ldg(t.leaf_lo + leaf + 1);
    for (int p = lo; p < hi; ++p) {
        if (p == self) continue; // all-points mode: the query itself (by position = by id)
        const int4 c = __ldg(t.pts + p);
        if (!pf.template pass<DIM>(c)) continue;
        const typename M::D d = M::template dist<DIM>(q, c);
        if (d < bd[K - 1] || (d == bd[K - 1] && c.w < bi[K - 1])) {
            kb_insert<K>(bd, bi, d, c.w);
            pf.update(bd[K - 1]);
        }
    }
}

// SM-affine feed of work items (warp groups of queries, or single queries of
// the warp-per-query kernel; n_groups of them).  The items are cut into
// n_chunks contiguous chunks (one per SM); a warp first takes items, one
// atomic per item, from the chunk of the SM it runs on, so the warps resident
// on an SM search neighbouring queries (Morton order) and find one another's
// candidate points and boxes in that SM's L1.  When its chunk is drained the warp steals single groups from
// the other chunks (all counters read in one warp-wide pass, from L2) until
// every chunk is drained.  A failed steal means that chunk ran out, so the
// loop ends; the retry count is capped all the same (status ZD_ERR_INTERNAL).
struct GroupFeed {
    int home;      // the chunk of this warp's SM
    bool stealing; // the home chunk is drained

    __device__ __forceinline__ GroupFeed(const KnnArgs &a)
    {
        unsigned sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        home = (int)(sm % (unsigned)a.n_chunks);
        stealing = false;
    }

    __device__ __forceinline__ static bool take(const KnnArgs &a, int c, int64_t &g)
    {
        int gi = 0;
        if ((threadIdx.x & 31) == 0) gi = atomicAdd(a.chunk_ctr + c, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        g = (int64_t)c * a.chunk_len + gi;
        return gi < a.chunk_len && g < a.n_groups;
    }

    // The next group of this warp, or -1.
    __device__ __forceinline__ int64_t next(const KnnArgs &a, u32 *status)
    {
        const int lane = threadIdx.x & 31;
        const int nch = a.n_chunks;
        int64_t g;
        if (!stealing) {
            if (take(a, home, g)) return g;
            stealing = true;
        }
        for (int tries = 0; tries < 4 * nch + 64; ++tries) {
            int found = -1;
            for (int base = 0; base < nch && found < 0; base += 32) {
                const int c = (home + 1 + base + lane) % nch;
                bool left = false;
                if (base + lane < nch) {
                    const int v = __ldcg(a.chunk_ctr + c);
                    left = v < a.chunk_len && (int64_t)c * a.chunk_len + v < a.n_groups;
                }
                const unsigned m = __ballot_sync(0xffffffffu, left);
                if (m) found = __shfl_sync(0xffffffffu, c, __ffs(m) - 1);
            }
            if (found < 0) return -1;
            if (take(a, found, g)) return g;
        }
        if (lane == 0) set_status(status, ZD_ERR_INTERNAL);
        return -1;
    }
};

// Blocks of a persistent launch of `kernel` (`threads` per block): as many as
// fit on the device at once (n_sm SMs), but no more than g.
template <typename Kernel>
unsigned persistent_blocks(Kernel kernel, int threads, unsigned g, int n_sm)
{
    static std::atomic<int> cached{0}; // resident blocks per SM (one per instantiation)
    int occ = cached.load(std::memory_order_relaxed);
    if (occ <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ <= 0)
            occ = 1;
        cached.store(occ, std::memory_order_relaxed);
    }
    return (unsigned)std::min<int64_t>((int64_t)g, (int64_t)occ * n_sm);
}

// Node v names an existing node: internal 0 <= v < n_leaves - 1, or leaf
// ~v < n_leaves (debug-build check).
__device__ __forceinline__ bool node_in_range(const TreeView &t, int v)
{
    const int nl = __ldg(t.meta);
    return v < 0 ? (~v < nl) : (v < nl - 1);
}

__device__ __forceinline__ void node_box(const TreeView &t, int v, int4 &lo, int4 &hi)
{
    const int4 *b = v < 0 ? t.lbox + 2 * (~v) : t.ibox + 2 * v;
    lo = __ldg(b);
    hi = __ldg(b + 1);
}

// Integer margin test against the Morton cell of a node whose parent splits
// on key bit pbit: coordinate j's levels >= ceil((pbit - (d-1-j)) / d) are
// the node's prefix, the rest is free.  True iff in every dimension the first
// integer outside the cell is more than sqrt(thr) from the query.
template <int DIM>
__device__ __forceinline__ bool cell_inside(int4 qp, uint3 shift, int pbit, long long thr)
{
    if (thr == LLONG_MAX) return false;
    const unsigned q3[3] = {(unsigned)qp.x + shift.x, (unsigned)qp.y + shift.y, (unsigned)qp.z + shift.z};
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const int lj = max(0, (pbit - (DIM - 1 - j) + DIM - 1) / DIM);
        const long long mask = (1ll << lj) - 1;
        const long long off = (long long)(q3[j] & (unsigned)mask);
        const long long m = min(off + 1, mask + 1 - off);
        if (m * m <= thr) return false;
    }
    return true;
}

// searchDown (Algorithm 2) from node v whose box distance is dv.
template <int DIM, int K, bool FLOAT>
__device__ __forceinline__ void search_down(const TreeView &t, int v, typename Metric<FLOAT>::D dv,
                                            int self, const typename Metric<FLOAT>::Q &q, Prefilter<FLOAT> &pf,
                                            typename Metric<FLOAT>::D (&bd)[K], int (&bi)[K],
                                            u32 *status)
{
    typedef Metric<FLOAT> M;
    typedef typename M::D D;
    int sn[KNN_STACK];
    D sd[KNN_STACK];
    int sp = 0;
    int u = v;
    D du = dv;
    while (true) {
        if (!ZD_DCHECK(node_in_range(t, u), status)) return;
        if (du <= bd[K - 1]) { // else pruned by the (possibly shrunk) k-th distance
            if (u < 0) {
                scan_leaf<DIM, K, FLOAT>(t, ~u, self, q, pf, bd, bi);
            } else {
                const int2 ch = __ldg(t.ichild + u);
                int4 al, ah, bl, bh;
                node_box(t, ch.x, al, ah);
                node_box(t, ch.y, bl, bh);
                const D da = M::template boxd<DIM>(q, al, ah);
                const D db = M::template boxd<DIM>(q, bl, bh);
                const D thr = bd[K - 1];
                // the farther child waits on the stack; the nearer one is
                // searched next without a round trip through the stack
                const int nf = da <= db ? ch.y : ch.x, nn = da <= db ? ch.x : ch.y;
                const D df = da <= db ? db : da, dn = da <= db ? da : db;
                if (df <= thr) {
                    if (sp + 1 > KNN_STACK) {
                        set_status(status, ZD_ERR_CUDA);
                        return;
                    }
                    sn[sp] = nf;
                    sd[sp] = df;
                    ++sp;
                }
                if (dn <= thr) {
                    u = nn;
                    du = dn;
                    continue;
                }
            }
        }
        if (sp == 0) break;
        --sp;
        u = sn[sp];
        du = sd[sp];
    }
}

template <int DIM, int K, bool FLOAT>
__device__ __forceinline__ void knn_query(const KnnArgs &a, const int64_t qi, u32 *status)
{
    typedef Metric<FLOAT> M;
    typedef typename M::D D;
    const TreeView &t = a.t;

    D bd[K];
    int bi[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        bd[j] = M::inf();
        bi[j] = INT_MAX;
    }
    const int nl = __ldg(t.meta);
    const int root = nl > 1 ? 0 : ~0;
    int4 qp;
    int self = -1;
    int64_t row;
    if (a.allpts) {
        qp = __ldg(t.pts + qi);
        self = (int)qi;
        row = qp.w;
        if (t.cloud_off) row += __ldg(t.cloud_off + (__ldg(t.keys + qi) >> t.cloud_bit));
    } else {
        qp = __ldg(a.q + qi);
        row = qp.w;
    }
    const typename M::Q q = M::make(qp);
    Prefilter<FLOAT> pf(qp);
    const u64 *qkeys = a.allpts ? t.keys : a.qkey;

    if (t.n > 0) {
        if (a.mode == ZD_SEARCH_ROOT) {
            int v = root;
            bool ok = true;
            if (t.cloud_off) {
                // descend to the root of the query's own cloud
                const u64 cloud = __ldg(qkeys + qi) >> t.cloud_bit;
                while (v >= 0 && __ldg(t.ibit + v) >= t.cloud_bit) {
                    const int2 ch = __ldg(t.ichild + v);
                    v = ((cloud >> (__ldg(t.ibit + v) - t.cloud_bit)) & 1) ? ch.y : ch.x;
                }
                const int first = v >= 0 ? __ldg(t.irange + v).x : __ldg(t.leaf_lo + ~v);
                const int last = v >= 0 ? __ldg(t.irange + v).y : __ldg(t.leaf_lo + ~v + 1);
                ok = last > first && (__ldg(t.keys + first) >> t.cloud_bit) == cloud;
            }
            if (ok) {
                int4 lo, hi;
                node_box(t, v, lo, hi);
                search_down<DIM, K, FLOAT>(t, v, M::template boxd<DIM>(q, lo, hi), self, q, pf, bd, bi, status);
            }
        } else {
            int leaf;
            if (a.mode == ZD_SEARCH_LEAF) {
                leaf = __ldg(t.leaf_of + qi);
            } else {
                // bit-based: descend by the query's Morton bits (Sec. 2)
                const u64 key = __ldg(qkeys + qi);
                int v = root;
                while (v >= 0) {
                    const int2 ch = __ldg(t.ichild + v);
                    v = ((key >> __ldg(t.ibit + v)) & 1) ? ch.y : ch.x;
                }
                leaf = ~v;
            }
            // searchUp (Algorithm 3)
            if (!ZD_DCHECK(node_in_range(t, ~leaf), status)) return;
            scan_leaf<DIM, K, FLOAT>(t, leaf, self, q, pf, bd, bi);
            int node = ~leaf;
            int par = __ldg(t.lparent + leaf);
            while (par >= 0 && __ldg(t.ibit + par) < t.cloud_bit) {
                int4 lo, hi;
                if (!FLOAT && a.allpts) {
                    // the query lies in the node's Morton cell, which holds
                    // every point the node can hold: stop on the cell
                    if (cell_inside<DIM>(qp, a.shift, __ldg(t.ibit + par), (long long)bd[K - 1])) break;
                } else {
                    node_box(t, node, lo, hi);
                    if (M::template inside<DIM>(q, lo, hi, bd[K - 1])) break;
                }
                const int2 ch = __ldg(t.ichild + par);
                const int sib = ch.x == node ? ch.y : ch.x;
                node_box(t, sib, lo, hi);
                const D ds = M::template boxd<DIM>(q, lo, hi);
                if (ds <= bd[K - 1]) search_down<DIM, K, FLOAT>(t, sib, ds, self, q, pf, bd, bi, status);
                node = par;
                par = __ldg(t.iparent + par);
            }
        }
    }

    const int k = a.k;
    int32_t *oi = a.out_idx + row * k;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (j < k) oi[j] = bd[j] < M::inf() ? bi[j] : -1;
    if (a.out_dist) {
        if (FLOAT) {
            float *od = (float *)a.out_dist + row * k;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (j < k) od[j] = bd[j] < M::inf() ? M::out_dist(bd[j]) : __int_as_float(0x7f800000);
        } else {
            long long *od = (long long *)a.out_dist + row * k;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (j < k) od[j] = (long long)bd[j];
        }
    }
}

// One thread per query.  With a.chunk_ctr the launch is persistent and each
// warp takes runs of 32 consecutive queries from the SM-affine feed.
template <int DIM, int K, bool FLOAT>
__global__ void __launch_bounds__(KNN_THREADS) k_knn(KnnArgs a, u32 *status)
{
    if (!a.chunk_ctr) {
        const int64_t qi = (int64_t)blockIdx.x * KNN_THREADS + threadIdx.x;
        if (qi < a.m) knn_query<DIM, K, FLOAT>(a, qi, status);
        return;
    }
    GroupFeed feed(a);
    for (int64_t g = feed.next(a, status); g >= 0; g = feed.next(a, status)) {
        const int64_t qi = g * 32 + (threadIdx.x & 31);
        if (qi < a.m) knn_query<DIM, K, FLOAT>(a, qi, status);
    }
}

// The same search for the sorted positions listed in a.sel (all-points mode).
template <int DIM, int K, bool FLOAT>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_sel(KnnArgs a, u32 *status)
{
    const int count = *a.sel_count;
    for (int i = blockIdx.x * KNN_THREADS + threadIdx.x; i < count; i += gridDim.x * KNN_THREADS)
        knn_query<DIM, K, FLOAT>(a, __ldg(a.sel + i), status);
}

template <int DIM, int K, bool FLOAT>
void launch_knn_k(const KnnArgs &a, cudaStream_t s, u32 *st)
{
    if (a.sel) {
        k_knn_sel<DIM, K, FLOAT><<<152 * 2, KNN_THREADS, 0, s>>>(a, st);
        return;
    }
    unsigned g = (unsigned)((a.m + KNN_THREADS - 1) / KNN_THREADS);
    if (a.chunk_ctr) g = persistent_blocks(k_knn<DIM, K, FLOAT>, KNN_THREADS, g, a.n_chunks);
    k_knn<DIM, K, FLOAT><<<g, KNN_THREADS, 0, s>>>(a, st);
}

template <int DIM, bool FLOAT>
int launch_knn_dim(const KnnArgs &a, cudaStream_t s)
{
    if (a.m <= 0 && !a.sel) return ZD_OK;
    u32 *st = status_word();
    KnnArgs b = a;
    if (b.sel) {
        b.chunk_ctr = nullptr; // the exact fallback keeps its own loop
    } else if (b.chunk_ctr) { // runs of 32 queries from the SM-affine feed
        ZD_CUDA(cudaMemsetAsync(b.chunk_ctr, 0, sizeof(int) * (size_t)b.n_chunks, s));
        b.n_groups = (b.m + 31) / 32;
        b.chunk_len = (b.n_groups + b.n_chunks - 1) / b.n_chunks;
    }
    if (a.k <= 1) launch_knn_k<DIM, 1, FLOAT>(b, s, st);
    else if (a.k <= 2) launch_knn_k<DIM, 2, FLOAT>(b, s, st);
    else if (a.k <= 4) launch_knn_k<DIM, 4, FLOAT>(b, s, st);
    else if (a.k <= 5) launch_knn_k<DIM, 5, FLOAT>(b, s, st);
    else if (a.k <= 8) launch_knn_k<DIM, 8, FLOAT>(b, s, st);
    else if (a.k <= 10) launch_knn_k<DIM, 10, FLOAT>(b, s, st);
    else if (a.k <= 12) launch_knn_k<DIM, 12, FLOAT>(b, s, st);
    else if (a.k <= 16) launch_knn_k<DIM, 16, FLOAT>(b, s, st);
    else if (a.k <= 24) launch_knn_k<DIM, 24, FLOAT>(b, s, st);
    else if (a.k <= 28) launch_knn_k<DIM, 28, FLOAT>(b, s, st);
    else if (a.k <= 32) launch_knn_k<DIM, 32, FLOAT>(b, s, st);
    else launch_knn_k<DIM, 40, FLOAT>(b, s, st); // the exact fallback of 40-wide groups
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
