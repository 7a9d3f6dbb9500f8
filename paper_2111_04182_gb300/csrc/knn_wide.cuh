// knn_wide.cuh -- exact k-NN for large k (32 < k <= 128): one warp per query
// (Algorithms 2 and 3).
//
// The k best of a query do not fit one thread's registers, so a whole warp
// serves one query and spreads its k-best list over the lanes: slot
// e = 32 r + lane lives in register r of that lane.  The list is kept sorted
// by (squared distance, id) over e and aligned to the end: the j-th best is
// slot 32 R - k + j, so the k-th best is always register R - 1 of lane 31,
// and slots below 32 R - k hold sentinels that order before every point.
// The traversal -- scan the start leaf, climb, search siblings down with a
// box test against the k-th distance -- is the one of the
// one-thread-per-query kernel (float trees with its fp32 candidate filter
// and int64-ordered fp64 values), executed in lockstep by the
// warp (every branch depends only on warp-uniform values); the DFS stack is
// a per-warp shared-memory array that every lane writes identically.
// Leaves are scanned 32 points at a time, one point per lane; for k <= 64 a
// subtree of at most WIDE_SMALL_SUBTREE points is scanned whole (its points
// are contiguous in sorted order) instead of descending into it, which
// trades box pruning for full-width rounds and fewer node visits.
//
// Filling: until k candidates have been seen the k-th distance is infinite
// and every candidate enters, so the first candidates are appended unsorted
// to a per-warp shared-memory buffer and sorted once (a bitonic sort over
// the 32 R register slots) when the k-th arrives.  After that a candidate
// that beats the k-th best is inserted by the warp: its rank comes from one
// ballot per register, and the slots from the rank up move up by one place
// (a shuffle, lane 0 taking lane 31 of the register below), which drops the
// old k-th best off the top.  For k > 64 (three or four registers) such
// single insertions cost more than batching: candidates that beat the k-th best are
// appended to a per-warp pending block of 32 and merged when it holds
// WIDE_FLUSH or more after a leaf, or would overflow -- the block is sorted
// (bitonic), then, from the top register down, the larger half of (register,
// reversed block) stays and the smaller half moves on (Batcher's bitonic
// split), stopping at the first register the block lies entirely above.
// Until a merge the threshold is the stale, larger k-th distance, which only
// admits more candidates and prunes less; the answer is the same.
#pragma once

#include "knn_impl.cuh"

namespace zdk {

constexpr int WIDE_WARPS = 4;           // queries in flight per block
constexpr int WIDE_STACK = 96;          // DFS stack entries per warp
constexpr int WIDE_SMALL_SUBTREE = 128; // k <= 64: subtrees scanned whole
constexpr int WIDE_FLUSH = 16;          // k > 64: pending candidates merged after a leaf
constexpr unsigned WFULL = 0xffffffffu;

template <typename D>
__device__ __forceinline__ bool wkey_lt(D a, int ai, D b, int bi)
{
    return a < b || (a == b && ai < bi);
}

// Order the pair (a, b): a <= b when up, a >= b otherwise.
template <typename D>
__device__ __forceinline__ void wcmpx(D &ad, int &ai, D &bd, int &bi, bool up)
{
    const bool sw = up ? wkey_lt(bd, bi, ad, ai) : wkey_lt(ad, ai, bd, bi);
    if (sw) {
        const D td = ad;
        const int ti = ai;
        ad = bd;
        ai = bi;
        bd = td;
        bi = ti;
    }
}

// One stage of a bitonic sort over the 32 R entries: compare-exchange e with
// e ^ STRIDE, ascending where bit SIZE of e is clear.  Strides of 32 and more
// pair registers of one lane, smaller strides pair lanes (shuffles).
template <int SIZE, int STRIDE, int R, typename D>
__device__ __forceinline__ void wide_stage(D (&d)[R], int (&id)[R], int lane)
{
    if constexpr (STRIDE >= 32) {
        constexpr int s = STRIDE >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!(r & s)) wcmpx(d[r], id[r], d[r | s], id[r | s], ((r * 32) & SIZE) == 0);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const D pd = __shfl_xor_sync(WFULL, d[r], STRIDE);
            const int pi = __shfl_xor_sync(WFULL, id[r], STRIDE);
            const bool up = ((r * 32 + lane) & SIZE) == 0;
            const bool keep_min = ((lane & STRIDE) == 0) == up;
            if (wkey_lt(pd, pi, d[r], id[r]) == keep_min) {
                d[r] = pd;
                id[r] = pi;
            }
        }
    }
    if constexpr (STRIDE > 1) wide_stage<SIZE, STRIDE / 2, R>(d, id, lane);
}

// Bitonic sort of the 32 R entries (R a power of two), ascending in e.
template <int SIZE, int R, typename D>
__device__ __forceinline__ void wide_sort(D (&d)[R], int (&id)[R], int lane)
{
    wide_stage<SIZE, SIZE / 2, R>(d, id, lane);
    if constexpr (SIZE < 32 * R) wide_sort<SIZE * 2, R>(d, id, lane);
}

template <int DIM, int R, bool FLOAT>
struct WideQuery {
    typedef Metric<FLOAT> M;
    typedef typename M::D D;

    const TreeView &t;
    typename M::Q q;
    Prefilter<FLOAT> pf; // float trees: fp32 candidate filter
    int self;  // sorted position to skip (all-points), else -1
    int lane;
    int k, off; // k, and the slot of the best (32 R - k)
    D d[R];
    int id[R];
    D td; // the k-th best (warp-uniform): infinite while filling
    int ti;
    bool filling;
    int count; // entries appended while filling
    D *bufd;   // this warp's fill buffer [32 R]
    int *bufi;
    D *pend_d; // this warp's pending block [32] (R >= 3)
    int *pend_i;
    int pc;     // pending candidates
    int *stk_n; // this warp's DFS stack [WIDE_STACK]
    D *stk_d;

    __device__ WideQuery(const TreeView &t_, int k_, int lane_, D *bd, int *bi, D *pd, int *pi, int *sn, D *sd)
        : t(t_), pf(make_int4(0, 0, 0, 0)), self(-1), lane(lane_), k(k_), off(32 * R - k_), td(M::inf()),
          ti(INT_MAX), filling(true),
          count(0), bufd(bd), bufi(bi), pend_d(pd), pend_i(pi), pc(0), stk_n(sn), stk_d(sd)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            d[r] = M::inf();
            id[r] = INT_MAX;
        }
    }

    __device__ __forceinline__ void refresh_kth()
    {
        td = __shfl_sync(WFULL, d[R - 1], 31);
        ti = __shfl_sync(WFULL, id[R - 1], 31);
        pf.update(td);
    }

    // Move the fill buffer into slots off .. off + count - 1 (sentinels
    // below, infinite entries above) and sort.
    __device__ __forceinline__ void finish_fill()
    {
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = r * 32 + lane - off;
            d[r] = j < 0 ? D(-1) : j < count ? bufd[j] : M::inf();
            id[r] = j < 0 ? -1 : j < count ? bufi[j] : INT_MAX;
        }
        __syncwarp();
        if constexpr ((R & (R - 1)) == 0) {
            wide_sort<2, R>(d, id, lane);
        } else {
            // not a power of two: sort a padded list (the padding is +inf and
            // ends on top)
            constexpr int RP = R < 4 ? 4 : 8;
            D pd[RP];
            int pi[RP];
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                pd[r] = r < R ? d[r] : M::inf();
                pi[r] = r < R ? id[r] : INT_MAX;
            }
            wide_sort<2, RP>(pd, pi, lane);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                d[r] = pd[r];
                id[r] = pi[r];
            }
        }
        filling = false;
        refresh_kth();
    }

    // Insert (cd, ci), which beats the k-th best, keeping the list sorted.
    __device__ __forceinline__ void insert(D cd, int ci)
    {
        int pos = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) pos += __popc(__ballot_sync(WFULL, wkey_lt(d[r], id[r], cd, ci)));
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            if ((r + 1) * 32 <= pos) break; // registers below are unchanged
            D ud = __shfl_up_sync(WFULL, d[r], 1);
            int ui = __shfl_up_sync(WFULL, id[r], 1);
            if (r > 0) {
                const D cd2 = __shfl_sync(WFULL, d[r - 1], 31);
                const int ci2 = __shfl_sync(WFULL, id[r - 1], 31);
                if (lane == 0) {
                    ud = cd2;
                    ui = ci2;
                }
            }
            const int e = r * 32 + lane;
            if (e == pos) {
                d[r] = cd;
                id[r] = ci;
            } else if (e > pos) {
                d[r] = ud;
                id[r] = ui;
            }
        }
        refresh_kth();
    }

    // Merge the pending block into the list (R >= 3).
    __device__ __forceinline__ void merge_pending()
    {
        __syncwarp();
        D xd[1];
        int xi[1];
        xd[0] = lane < pc ? pend_d[lane] : M::inf();
        xi[0] = lane < pc ? pend_i[lane] : INT_MAX;
        __syncwarp();
        pc = 0;
        wide_sort<2, 1>(xd, xi, lane);
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            const D yd = __shfl_sync(WFULL, xd[0], 31 - lane);
            const int yi = __shfl_sync(WFULL, xi[0], 31 - lane);
            const bool sw = wkey_lt(yd, yi, d[r], id[r]);
            const bool any = __any_sync(WFULL, sw);
            if (r < R - 1) { // the larger half, sorted, is register r + 1
                D hd[1] = {sw ? d[r] : yd};
                int hn[1] = {sw ? id[r] : yi};
                wide_stage<32, 16, 1>(hd, hn, lane);
                d[r + 1] = hd[0];
                id[r + 1] = hn[0];
            }
            if (!any) break; // the block lay above register r: the rest is unchanged
            xd[0] = sw ? yd : d[r];
            xi[0] = sw ? yi : id[r];
            wide_stage<32, 16, 1>(xd, xi, lane);
            if (r == 0) {
                d[0] = xd[0];
                id[0] = xi[0];
            }
        }
        refresh_kth();
    }

    __device__ __forceinline__ void scan_leaf(int leaf)
    {
        scan_range(__ldg(t.leaf_lo + leaf), __ldg(t.leaf_lo + leaf + 1));
    }

    // The candidates at sorted positions [lo, hi), 32 per round.
    __device__ __forceinline__ void scan_range(int lo, int hi)
    {
        for (int base = lo; base < hi; base += 32) {
            const int p = base + lane;
            D cd = M::inf();
            int ci = INT_MAX;
            bool ok = false;
            if (p < hi && p != self) {
                const int4 c = __ldg(t.pts + p);
                if (pf.template pass<DIM>(c)) {
                    cd = M::template dist<DIM>(q, c);
                    ci = c.w;
                    ok = wkey_lt(cd, ci, td, ti);
                }
            }
            unsigned mask = __ballot_sync(WFULL, ok);
            if (filling) {
                const int room = k - count;
                const int rank = __popc(mask & ((1u << lane) - 1u));
                if (ok && rank < room) {
                    bufd[count + rank] = cd;
                    bufi[count + rank] = ci;
                }
                const int n = __popc(mask);
                const int placed = min(n, room);
                count += placed;
                mask = __ballot_sync(WFULL, ok && rank >= placed);
                if (count >= k || mask) finish_fill();
            }
            if (R >= 3 && mask) {
                bool acc = (mask >> lane) & 1;
                int n = __popc(mask);
                if (pc + n > 32) {
                    merge_pending();
                    acc = acc && wkey_lt(cd, ci, td, ti);
                    mask = __ballot_sync(WFULL, acc);
                    n = __popc(mask);
                }
                const int rank = __popc(mask & ((1u << lane) - 1u));
                if (acc) {
                    pend_d[pc + rank] = cd;
                    pend_i[pc + rank] = ci;
                }
                pc += n;
                mask = 0;
            }
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const D xd = __shfl_sync(WFULL, cd, src);
                const int xi = __shfl_sync(WFULL, ci, src);
                if (wkey_lt(xd, xi, td, ti)) insert(xd, xi);
            }
        }
        if (R >= 3 && pc >= WIDE_FLUSH) merge_pending();
    }

    // searchDown (Algorithm 2) from node v whose box distance is dv.  The
    // nearer child is searched next directly; the farther one waits on the
    // stack, which every lane pushes and pops identically -- the __syncwarp
    // after a pop keeps a lane from overwriting the entry before all lanes
    // have read it.
    __device__ __forceinline__ bool search_down(int v, D dv, u32 *status)
    {
        int sp = 0;
        int u = v;
        D du = dv;
        while (true) {
            if (!ZD_DCHECK(node_in_range(t, u), status)) return false;
            if (du <= td) { // else pruned by the (possibly shrunk) k-th distance
                if (u < 0) {
                    scan_leaf(~u);
                } else {
                    bool expand = true;
                    if (R == 2) {
                        const int2 rg = __ldg(t.irange + u);
                        if (rg.y - rg.x <= WIDE_SMALL_SUBTREE) {
                            scan_range(rg.x, rg.y);
                            expand = false;
                        }
                    }
                    if (expand) {
                        const int2 ch = __ldg(t.ichild + u);
                        int4 al, ah, bl, bh;
                        node_box(t, ch.x, al, ah);
                        node_box(t, ch.y, bl, bh);
                        const D da = M::template boxd<DIM>(q, al, ah);
                        const D db = M::template boxd<DIM>(q, bl, bh);
                        const int nf = da <= db ? ch.y : ch.x, nn = da <= db ? ch.x : ch.y;
                        const D df = da <= db ? db : da, dn = da <= db ? da : db;
                        if (df <= td) {
                            if (sp + 1 > WIDE_STACK) {
                                if (lane == 0) set_status(status, ZD_ERR_CUDA);
                                return false;
                            }
                            stk_n[sp] = nf;
                            stk_d[sp] = df;
                            ++sp;
                        }
                        if (dn <= td) {
                            u = nn;
                            du = dn;
                            continue;
                        }
                    }
                }
            }
            if (sp == 0) break;
            --sp;
            u = stk_n[sp];
            du = stk_d[sp];
            __syncwarp();
        }
        return true;
    }
};

template <int DIM, int R, bool FLOAT>
__global__ void __launch_bounds__(32 * WIDE_WARPS, R >= 3 ? 6 : 8) k_knn_wide(KnnArgs a, u32 *status)
{
    typedef Metric<FLOAT> M;
    typedef typename M::D D;
    constexpr int PEND = R >= 3 ? 32 : 1;
    __shared__ D s_bufd[WIDE_WARPS][32 * R];
    __shared__ int s_bufi[WIDE_WARPS][32 * R];
    __shared__ D s_pd[WIDE_WARPS][PEND];
    __shared__ int s_pi[WIDE_WARPS][PEND];
    __shared__ D s_sd[WIDE_WARPS][WIDE_STACK];
    __shared__ int s_sn[WIDE_WARPS][WIDE_STACK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TreeView &t = a.t;
    const int nl = __ldg(t.meta);
    const int root = nl > 1 ? 0 : ~0;

    // queries from the SM-affine feed (persistent launch, a.chunk_ctr), else
    // a grid-stride loop
    GroupFeed feed(a);
    for (int64_t qi = a.chunk_ctr ? feed.next(a, status) : (int64_t)blockIdx.x * WIDE_WARPS + warp;
         qi >= 0 && qi < a.m;
         qi = a.chunk_ctr ? feed.next(a, status) : qi + (int64_t)gridDim.x * WIDE_WARPS) {
        __syncwarp();
        WideQuery<DIM, R, FLOAT> w(t, a.k, lane, s_bufd[warp], s_bufi[warp], s_pd[warp], s_pi[warp], s_sn[warp],
                                   s_sd[warp]);
        int4 qp;
        int64_t row;
        if (a.allpts) {
            qp = __ldg(t.pts + qi);
            w.self = (int)qi;
            row = qp.w;
            if (t.cloud_off) row += __ldg(t.cloud_off + (__ldg(t.keys + qi) >> t.cloud_bit));
        } else {
            qp = __ldg(a.q + qi);
            row = qp.w;
        }
        w.q = M::make(qp);
        w.pf = Prefilter<FLOAT>(qp);

        bool ok = true;
        if (t.n > 0) {
            if (a.mode == ZD_SEARCH_ROOT) {
                int v = root;
                bool has = true;
                if (t.cloud_off) {
                    // descend to the root of the query's own cloud
                    const u64 cloud = __ldg((a.allpts ? t.keys : a.qkey) + qi) >> t.cloud_bit;
                    while (v >= 0 && __ldg(t.ibit + v) >= t.cloud_bit) {
                        const int2 ch = __ldg(t.ichild + v);
                        v = ((cloud >> (__ldg(t.ibit + v) - t.cloud_bit)) & 1) ? ch.y : ch.x;
                    }
                    const int first = v >= 0 ? __ldg(t.irange + v).x : __ldg(t.leaf_lo + ~v);
                    const int last = v >= 0 ? __ldg(t.irange + v).y : __ldg(t.leaf_lo + ~v + 1);
                    has = last > first && (__ldg(t.keys + first) >> t.cloud_bit) == cloud;
                }
                if (has) {
                    int4 lo, hi;
                    node_box(t, v, lo, hi);
                    ok = w.search_down(v, M::template boxd<DIM>(w.q, lo, hi), status);
                }
            } else {
                int leaf;
                if (a.mode == ZD_SEARCH_LEAF) {
                    leaf = __ldg(t.leaf_of + qi);
                } else {
                    // bit-based: descend by the query's Morton bits (Sec. 2)
                    const u64 key = __ldg((a.allpts ? t.keys : a.qkey) + qi);
                    int v = root;
                    while (v >= 0) {
                        const int2 ch = __ldg(t.ichild + v);
                        v = ((key >> __ldg(t.ibit + v)) & 1) ? ch.y : ch.x;
                    }
                    leaf = ~v;
                }
                // searchUp (Algorithm 3)
                w.scan_leaf(leaf);
                int node = ~leaf;
                int par = __ldg(t.lparent + leaf);
                while (ok && par >= 0 && __ldg(t.ibit + par) < t.cloud_bit) {
                    int4 lo, hi;
                    if (!FLOAT && a.allpts) {
                        if (cell_inside<DIM>(qp, a.shift, __ldg(t.ibit + par), (long long)w.td)) break;
                    } else {
                        node_box(t, node, lo, hi);
                        if (M::template inside<DIM>(w.q, lo, hi, w.td)) break;
                    }
                    const int2 ch = __ldg(t.ichild + par);
                    const int sib = ch.x == node ? ch.y : ch.x;
                    node_box(t, sib, lo, hi);
                    const D ds = M::template boxd<DIM>(w.q, lo, hi);
                    if (ds <= w.td) ok = w.search_down(sib, ds, status);
                    node = par;
                    par = __ldg(t.iparent + par);
                }
            }
        }
        if (w.filling) w.finish_fill();
        if (R >= 3 && w.pc > 0) w.merge_pending();

        const int k = a.k;
        int32_t *oi = a.out_idx + row * k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane - w.off;
            if (e >= 0) oi[e] = w.d[r] < M::inf() ? w.id[r] : -1;
        }
        if (a.out_dist) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = r * 32 + lane - w.off;
                if (e < 0) continue;
                if (FLOAT)
                    ((float *)a.out_dist)[row * k + e] =
                        w.d[r] < M::inf() ? M::out_dist(w.d[r]) : __int_as_float(0x7f800000);
                else
                    ((long long *)a.out_dist)[row * k + e] = (long long)w.d[r];
            }
        }
    }
}

template <int DIM, int R, bool FLOAT>
void launch_wide_r(const KnnArgs &a, unsigned grid, cudaStream_t s, u32 *st)
{
    if (a.chunk_ctr) grid = persistent_blocks(k_knn_wide<DIM, R, FLOAT>, 32 * WIDE_WARPS, grid, a.n_chunks);
    k_knn_wide<DIM, R, FLOAT><<<grid, 32 * WIDE_WARPS, 0, s>>>(a, st);
}

template <int DIM, bool FLOAT>
int launch_knn_wide_dim(const KnnArgs &a, cudaStream_t s)
{
    if (a.m <= 0) return ZD_OK;
    u32 *st = status_word();
    KnnArgs b = a;
    const unsigned grid = grid_for(a.m, WIDE_WARPS, 152 * 64);
    if (b.chunk_ctr) { // one query per feed item
        ZD_CUDA(cudaMemsetAsync(b.chunk_ctr, 0, sizeof(int) * (size_t)b.n_chunks, s));
        b.n_groups = b.m;
        b.chunk_len = (b.m + b.n_chunks - 1) / b.n_chunks;
    }
    const unsigned want = (unsigned)std::min<int64_t>((a.m + WIDE_WARPS - 1) / WIDE_WARPS, 1 << 30);
    if (a.k <= 64) launch_wide_r<DIM, 2, FLOAT>(b, b.chunk_ctr ? want : grid, s, st);
    else if (a.k <= 96) launch_wide_r<DIM, 3, FLOAT>(b, b.chunk_ctr ? want : grid, s, st);
    else launch_wide_r<DIM, 4, FLOAT>(b, b.chunk_ctr ? want : grid, s, st);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
