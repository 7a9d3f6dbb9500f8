// build.cu -- the canonical pruned zd-tree (Algorithm 1 with the empty-cut
// pruning of Sec. 2.1) built from Morton-sorted keys without recursion.
//
// Algorithm 1 splits a node on the highest bit where its keys differ
// (splitUsingBit); with empty cuts pruned, every node is a maximal run of the
// sorted keys in which all adjacent "highest differing bits" delta_i =
// hibit(k_i ^ k_{i+1}) are below the two deltas that bound the run (a
// max-Cartesian tree of delta).  A node is internal iff it holds more than L
// points and its keys are not all equal, so boundary i separates two leaves
// iff keys i and i+1 differ and the run bounded by the nearest larger deltas
// on either side holds more than L points.  Deciding that only needs the
// deltas within L positions of i: a stencil, one thread per boundary.
//
// The leaves are then the runs between flagged boundaries; the internal
// nodes form the binary radix tree of the leaves' first keys, built with one
// thread per internal node by the search of Karras (2012), and the boxes are
// merged bottom-up with one arrival counter per internal node.
#include "common.cuh"

namespace zdk {

// ----------------------------------------------------------------- gather
template <int DIM>
__global__ void __launch_bounds__(256) k_gather(const int32_t *__restrict__ pts, int64_t n,
                                                const int32_t *__restrict__ perm,
                                                const u64 *__restrict__ keys, int cloud_bit,
                                                const int64_t *__restrict__ cloud_off,
                                                int32_t base_id, int4 *__restrict__ out,
                                                float4 *__restrict__ fout, uint3 fshift, u32 *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t src = perm[i];
        if (!ZD_DCHECK(src >= 0 && src < n, status)) continue;
        int4 r;
        r.x = pts[src * DIM + 0];
        r.y = pts[src * DIM + 1];
        r.z = DIM == 3 ? pts[src * DIM + 2] : 0;
        if (cloud_off) r.w = (int)(src - cloud_off[keys[i] >> cloud_bit]);
        else r.w = (int)(base_id + src);
        out[i] = r;
        if (fout) fout[i] = shifted_float4(r, fshift);
    }
}

int launch_gather(const void *pts_in, int dim, int64_t n, const int32_t *perm,
                  const u64 *sorted_keys, int cloud_bit, const int64_t *cloud_off, int32_t base_id,
                  int4 *pts_out, cudaStream_t s, float4 *fpts_out, uint3 fshift)
{
    if (n <= 0) return ZD_OK;
    unsigned g = grid_for(n, 256, 152 * 32);
    if (dim == 3)
        k_gather<3><<<g, 256, 0, s>>>((const int32_t *)pts_in, n, perm, sorted_keys, cloud_bit,
                                      cloud_off, base_id, pts_out, fpts_out, fshift, status_word());
    else
        k_gather<2><<<g, 256, 0, s>>>((const int32_t *)pts_in, n, perm, sorted_keys, cloud_bit,
                                      cloud_off, base_id, pts_out, fpts_out, fshift, status_word());
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// ------------------------------------------------------------ leaf splits
constexpr int FLAG_THREADS = 256;
constexpr int FLAG_ITEMS = 4;
constexpr int FLAG_TILE = FLAG_THREADS * FLAG_ITEMS; // boundaries per block
constexpr int MAX_LEAF = 256;                        // largest L the stencil serves

__device__ __forceinline__ int delta_of(u64 a, u64 b) { return a == b ? -1 : 63 - __clzll(a ^ b); }

// flag[i] = 1 iff boundary i (between sorted points i and i+1) separates two
// leaves; block_count[b] = flags in block b's tile.
//
// Boundary i's run is bounded by the nearest boundaries on either side with a
// larger delta.  Both are found by binary lifting over a shared-memory table
// of window maxima, F_j[e] = max(delta[e .. e + 2^j - 1]): from the
// neighbour of i outward, skip the largest power-of-two block whose maximum
// is <= delta_i, for j = J..0, never beyond L - 1 positions.  Every boundary
// takes the same J + 1 steps per side (no divergent scans).  Positions
// outside [0, n-1) count as larger than every delta (the ends of the array
// bound every run).
constexpr int DELTA_OUT = 1 << 20; // "larger than every delta" (deltas are < 64)

__global__ void __launch_bounds__(FLAG_THREADS) k_split_flags(const u64 *__restrict__ keys, int64_t n,
                                                              int L, int levels, int force_bit,
                                                              unsigned char *__restrict__ flag,
                                                              int *__restrict__ block_count)
{
    extern __shared__ int s_tab[]; // [levels][wn]
    __shared__ int s_cnt[FLAG_THREADS / 32];
    const int64_t nb = n - 1; // number of boundaries
    const int64_t t0 = (int64_t)blockIdx.x * FLAG_TILE;
    // deltas of boundaries [t0 - L, t0 + FLAG_TILE + L)
    const int64_t w0 = t0 - L;
    const int wn = FLAG_TILE + 2 * L;
    for (int e = threadIdx.x; e < wn; e += FLAG_THREADS) {
        const int64_t j = w0 + e;
        s_tab[e] = (j >= 0 && j < nb) ? delta_of(keys[j], keys[j + 1]) : DELTA_OUT;
    }
    __syncthreads();
    for (int lv = 1; lv < levels; ++lv) {
        const int h = 1 << (lv - 1);
        const int *prev = s_tab + (lv - 1) * wn;
        int *cur = s_tab + lv * wn;
        for (int e = threadIdx.x; e < wn; e += FLAG_THREADS)
            cur[e] = e + h < wn ? max(prev[e], prev[e + h]) : prev[e];
        __syncthreads();
    }
    int cnt = 0;
#pragma unroll
    for (int it = 0; it < FLAG_ITEMS; ++it) {
        const int e = it * FLAG_THREADS + threadIdx.x;
        const int64_t i = t0 + e;
        if (i >= nb) continue;
        const int ei = e + L; // window index of boundary i
        const int di = s_tab[ei];
        unsigned char f = 0;
        if (di >= 0) {
            // left: skipped positions ei-1, ei-2, ... whose deltas are <= di
            int lskip = 0, rskip = 0;
            for (int lv = levels - 1; lv >= 0; --lv) {
                const int len = 1 << lv;
                if (lskip + len <= L - 1 && s_tab[lv * wn + ei - lskip - len] <= di) lskip += len;
                if (rskip + len <= L - 1 && s_tab[lv * wn + ei + rskip + 1] <= di) rskip += len;
            }
            // nearest larger at distance lskip + 1 / rskip + 1, or farther than
            // L - 1 (then the run already holds more than L points)
            const int64_t pg = i - (lskip + 1), ng = i + (rskip + 1);
            f = (ng - pg > L || di >= force_bit) ? 1 : 0;
        }
        flag[i] = f;
        cnt += f;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < FLAG_THREADS / 32; ++w) t += s_cnt[w];
        block_count[blockIdx.x] = t;
    }
}

// Exclusive scan of the block counts (one block); meta[0] = leaves.
__global__ void __launch_bounds__(1024) k_scan_counts(int *__restrict__ count, int64_t nblocks,
                                                      int64_t n, int *__restrict__ meta,
                                                      int *__restrict__ leaf_lo)
{
    __shared__ int s_w[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nblocks; base += 1024) {
        int64_t i = base + threadIdx.x;
        int v = i < nblocks ? count[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        int excl = s_carry + (warp ? s_w[warp - 1] : 0) + x - v;
        if (i < nblocks) count[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int leaves = s_carry + 1;
        meta[0] = leaves;
        leaf_lo[0] = 0;
        leaf_lo[leaves] = (int)n;
    }
}

// leaf_of[p] = number of flagged boundaries before point p; leaf_lo[j] =
// first point of leaf j.
__global__ void __launch_bounds__(FLAG_THREADS) k_leaf_index(const unsigned char *__restrict__ flag,
                                                             int64_t n,
                                                             const int *__restrict__ block_off,
                                                             int *__restrict__ leaf_of,
                                                             int *__restrict__ leaf_lo)
{
    __shared__ int s_w[FLAG_THREADS / 32];
    const int64_t nb = n - 1;
    const int64_t t0 = (int64_t)blockIdx.x * FLAG_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread owns FLAG_ITEMS consecutive boundaries
    int f[FLAG_ITEMS];
    int sum = 0;
#pragma unroll
    for (int it = 0; it < FLAG_ITEMS; ++it) {
        int64_t i = t0 + threadIdx.x * FLAG_ITEMS + it;
        f[it] = i < nb ? flag[i] : 0;
        sum += f[it];
    }
    int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    int wo = 0;
    for (int w = 0; w < warp; ++w) wo += s_w[w];
    int run = block_off[blockIdx.x] + wo + x - sum; // flags before this thread's first boundary
#pragma unroll
    for (int it = 0; it < FLAG_ITEMS; ++it) {
        int64_t i = t0 + threadIdx.x * FLAG_ITEMS + it;
        if (i < nb) {
            run += f[it];
            leaf_of[i + 1] = run;
            if (f[it]) leaf_lo[run] = (int)(i + 1);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && n > 0) leaf_of[0] = 0;
}

// --------------------------------------------------------- internal nodes
// Common-prefix length of the first keys of leaves a and b (-1 outside).
__device__ __forceinline__ int lcp(const u64 *__restrict__ keys, const int *__restrict__ leaf_lo,
                                   int nl, int a, int b)
{
    if (b < 0 || b >= nl) return -1;
    return __clzll(keys[leaf_lo[a]] ^ keys[leaf_lo[b]]);
}

__global__ void __launch_bounds__(256) k_internal(const u64 *__restrict__ keys,
                                                  const int *__restrict__ leaf_lo,
                                                  const int *__restrict__ meta, int64_t max_nodes,
                                                  int2 *__restrict__ ichild, int *__restrict__ iparent,
                                                  int *__restrict__ ibit, int2 *__restrict__ irange,
                                                  int *__restrict__ lparent, u32 *status)
{
    const int nl = meta[0];
    const int m = nl - 1; // internal nodes
    for (int64_t ii = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ii < max_nodes;
         ii += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        if (i == 0) {
            if (m == 0) lparent[0] = -1;
            else iparent[0] = -1;
        }
        if (i >= m) return;
        // direction of the node's range, its far end, then the split
        const int dn = lcp(keys, leaf_lo, nl, i, i + 1) - lcp(keys, leaf_lo, nl, i, i - 1) > 0 ? 1 : -1;
        const int dmin = lcp(keys, leaf_lo, nl, i, i - dn);
        int lmax = 2;
        while (lcp(keys, leaf_lo, nl, i, i + lmax * dn) > dmin) lmax <<= 1;
        int l = 0;
        for (int t = lmax >> 1; t >= 1; t >>= 1)
            if (lcp(keys, leaf_lo, nl, i, i + (l + t) * dn) > dmin) l += t;
        const int j = i + l * dn;
        const int dnode = lcp(keys, leaf_lo, nl, i, j);
        int s = 0;
        int t = l;
        do {
            t = (t + 1) >> 1;
            if (lcp(keys, leaf_lo, nl, i, i + (s + t) * dn) > dnode) s += t;
        } while (t > 1);
        const int g = i + s * dn + min(dn, 0);
        const int a = min(i, j), b = max(i, j);
        if (!ZD_DCHECK(a >= 0 && b < nl && a <= g && g < b, status)) continue;
        const int left = (a == g) ? ~g : g;
        const int right = (b == g + 1) ? ~(g + 1) : g + 1;
        ichild[i] = make_int2(left, right);
        ibit[i] = 63 - dnode;
        irange[i] = make_int2(leaf_lo[a], leaf_lo[b + 1]);
        if (left < 0) lparent[~left] = i;
        else iparent[left] = i;
        if (right < 0) lparent[~right] = i;
        else iparent[right] = i;
    }
}

// ------------------------------------------------------------------ boxes
template <bool FLOAT>
struct BoxOps;
template <>
struct BoxOps<false> {
    __device__ static int4 empty_lo() { return make_int4(INT_MAX, INT_MAX, INT_MAX, 0); }
    __device__ static int4 empty_hi() { return make_int4(INT_MIN, INT_MIN, INT_MIN, 0); }
    __device__ static int4 mn(int4 a, int4 b) { return make_int4(min(a.x, b.x), min(a.y, b.y), min(a.z, b.z), 0); }
    __device__ static int4 mx(int4 a, int4 b) { return make_int4(max(a.x, b.x), max(a.y, b.y), max(a.z, b.z), 0); }
};
template <>
struct BoxOps<true> {
    __device__ static int4 f(float x, float y, float z)
    {
        return make_int4(__float_as_int(x), __float_as_int(y), __float_as_int(z), 0);
    }
    __device__ static int4 empty_lo() { return f(INFINITY, INFINITY, INFINITY); }
    __device__ static int4 empty_hi() { return f(-INFINITY, -INFINITY, -INFINITY); }
    __device__ static int4 mn(int4 a, int4 b)
    {
        return f(fminf(__int_as_float(a.x), __int_as_float(b.x)), fminf(__int_as_float(a.y), __int_as_float(b.y)),
                 fminf(__int_as_float(a.z), __int_as_float(b.z)));
    }
    __device__ static int4 mx(int4 a, int4 b)
    {
        return f(fmaxf(__int_as_float(a.x), __int_as_float(b.x)), fmaxf(__int_as_float(a.y), __int_as_float(b.y)),
                 fmaxf(__int_as_float(a.z), __int_as_float(b.z)));
    }
};

__device__ __forceinline__ float4 as_float4(int4 v, uint3 sh)
{
    return shifted_float4(v, sh);
}

// Float copy of integer points (shifted_float4).  The search filters
// candidates on it.
__global__ void k_fpts(const int4 *__restrict__ pts, int64_t n, float4 *__restrict__ fpts, uint3 sh)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        fpts[i] = shifted_float4(pts[i], sh);
}

// Atomic add with acquire-release semantics at device scope: it publishes
// the calling thread's earlier writes and makes the writes published by
// earlier adds to the same counter visible to it.
__device__ __forceinline__ int atomic_add_acq_rel(int *p, int v)
{
    int old;
    asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <bool FLOAT>
__global__ void __launch_bounds__(256) k_boxes(const int4 *__restrict__ pts,
                                               const int *__restrict__ leaf_lo,
                                               const int *__restrict__ meta, int64_t max_leaves,
                                               const int2 *__restrict__ ichild,
                                               const int *__restrict__ iparent,
                                               const int *__restrict__ lparent, int4 *ibox,
                                               int4 *lbox, int *counter, float4 *fibox, float4 *flbox,
                                               uint3 fshift, u32 *status)
{
    typedef BoxOps<FLOAT> B;
    const int nl = meta[0];
    for (int64_t jj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; jj < max_leaves;
         jj += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)jj;
        if (j >= nl) return;
        int4 lo = B::empty_lo(), hi = B::empty_hi();
        for (int p = leaf_lo[j], e = leaf_lo[j + 1]; p < e; ++p) {
            int4 c = pts[p];
            lo = B::mn(lo, c);
            hi = B::mx(hi, c);
        }
        lbox[2 * j] = lo;
        lbox[2 * j + 1] = hi;
        if (flbox) {
            // spare w lanes: the leaf's range of sorted positions
            float4 flo = as_float4(lo, fshift), fhi = as_float4(hi, fshift);
            flo.w = __int_as_float(leaf_lo[j]);
            fhi.w = __int_as_float(leaf_lo[j + 1]);
            flbox[2 * j] = flo;
            flbox[2 * j + 1] = fhi;
        }
        int p = lparent[j];
        while (p >= 0) {
            if (!ZD_DCHECK(p < nl - 1, status)) break;
            // acq_rel: publishes this thread's boxes, and the second arriver
            // sees its sibling's
            if (atomic_add_acq_rel(&counter[p], 1) == 0) break; // the sibling finishes this node
            int2 ch = ichild[p];
            const int4 *ba = ch.x < 0 ? lbox + 2 * (~ch.x) : ibox + 2 * ch.x;
            const int4 *bb = ch.y < 0 ? lbox + 2 * (~ch.y) : ibox + 2 * ch.y;
            int4 l0 = __ldcg(ba), h0 = __ldcg(ba + 1), l1 = __ldcg(bb), h1 = __ldcg(bb + 1);
            const int4 lo2 = B::mn(l0, l1), hi2 = B::mx(h0, h1);
            ibox[2 * p] = lo2;
            ibox[2 * p + 1] = hi2;
            if (fibox) {
                // spare w lanes: the two children
                float4 flo = as_float4(lo2, fshift), fhi = as_float4(hi2, fshift);
                flo.w = __int_as_float(ch.x);
                fhi.w = __int_as_float(ch.y);
                fibox[2 * p] = flo;
                fibox[2 * p + 1] = fhi;
            }
            p = iparent[p];
        }
    }
}

// ---------------------------------------------------------- group starts
// gpre[c] = number of 32-point groups in clouds before c (one block).
__global__ void __launch_bounds__(1024) k_group_prefix(const int64_t *__restrict__ off, int64_t nc,
                                                       int64_t *__restrict__ gpre)
{
    __shared__ int64_t s_w[32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nc; base += 1024) {
        const int64_t c = base + threadIdx.x;
        const int64_t v = c < nc ? (off[c + 1] - off[c] + 31) / 32 : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const int64_t excl = s_carry + (warp ? s_w[warp - 1] : 0) + x - v;
        if (c < nc) gpre[c] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) gpre[nc] = s_carry;
}

__global__ void k_group_starts(const int64_t *__restrict__ off, const int64_t *__restrict__ gpre, int64_t nc,
                               int64_t ng, int *__restrict__ start)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = 0, z = nc - 1; // last cloud with gpre[c] <= g
        while (a < z) {
            int64_t mid = (a + z + 1) >> 1;
            if (gpre[mid] <= g) a = mid;
            else z = mid - 1;
        }
        if (g < gpre[nc]) start[g] = (int)(off[a] + 32 * (g - gpre[a]));
    }
}

int launch_group_starts(const int64_t *cloud_off, int64_t n_clouds, int64_t n_groups, int *group_start,
                        int64_t *gpre, cudaStream_t s)
{
    k_group_prefix<<<1, 1024, 0, s>>>(cloud_off, n_clouds, gpre);
    if (n_groups > 0)
        k_group_starts<<<grid_for(n_groups, 256, 152 * 16), 256, 0, s>>>(cloud_off, gpre, n_clouds, n_groups,
                                                                        group_start);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int launch_fpts(const int4 *pts, int64_t n, float4 *fpts, uint3 shift, cudaStream_t s)
{
    if (n > 0) k_fpts<<<grid_for(n, 256, 152 * 32), 256, 0, s>>>(pts, n, fpts, shift);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int build_topology(const u64 *keys, const int4 *pts, int64_t n, int leaf_size, int dim,
                   int is_float, int force_bit, const TopoBuffers &b, Mem &mem, bool fpts_ready)
{
    (void)dim;
    cudaStream_t s = mem.s;
    if (leaf_size < 1 || leaf_size > MAX_LEAF) return ZD_ERR_INVALID_ARG;
    const int64_t nb = n > 1 ? n - 1 : 0;
    const int64_t nblocks = nb > 0 ? (nb + FLAG_TILE - 1) / FLAG_TILE : 0;
    Scratch<unsigned char> flag(mem, nb > 0 ? nb : 1);
    Scratch<int> bcount(mem, nblocks > 0 ? nblocks : 1);
    if (!flag.p || !bcount.p) return ZD_ERR_OOM;
    if (nblocks > 0) {
        // table levels: spans 1, 2, 4, ... up to the largest <= L - 1
        int levels = 1;
        while ((1 << levels) <= leaf_size - 1) ++levels;
        const size_t smem = sizeof(int) * (size_t)levels * (FLAG_TILE + 2 * leaf_size);
        ZD_CUDA(cudaFuncSetAttribute(k_split_flags, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_split_flags<<<(unsigned)nblocks, FLAG_THREADS, smem, s>>>(keys, n, leaf_size, levels, force_bit, flag.p,
                                                                    bcount.p);
        ZD_CUDA(cudaGetLastError());
    }
    k_scan_counts<<<1, 1024, 0, s>>>(bcount.p, nblocks, n, b.meta, b.leaf_lo);
    ZD_CUDA(cudaGetLastError());
    if (n > 0) {
        k_leaf_index<<<(unsigned)(nblocks > 0 ? nblocks : 1), FLAG_THREADS, 0, s>>>(flag.p, n, bcount.p,
                                                                                 b.leaf_of, b.leaf_lo);
        ZD_CUDA(cudaGetLastError());
    }
    const int64_t max_nodes = n > 1 ? n - 1 : 1;
    k_internal<<<grid_for(max_nodes, 256, 152 * 64), 256, 0, s>>>(keys, b.leaf_lo, b.meta, max_nodes,
                                                                 b.ichild, b.iparent, b.ibit, b.irange,
                                                                 b.lparent, status_word());
    ZD_CUDA(cudaGetLastError());
    ZD_CUDA(cudaMemsetAsync(b.counter, 0, sizeof(int) * (size_t)max_nodes, s));
    const int64_t max_leaves = n > 0 ? n : 1;
    if (is_float)
        k_boxes<true><<<grid_for(max_leaves, 256, 152 * 64), 256, 0, s>>>(
            pts, b.leaf_lo, b.meta, max_leaves, b.ichild, b.iparent, b.lparent, b.ibox, b.lbox, b.counter,
            nullptr, nullptr, make_uint3(0, 0, 0), status_word());
    else
        k_boxes<false><<<grid_for(max_leaves, 256, 152 * 64), 256, 0, s>>>(
            pts, b.leaf_lo, b.meta, max_leaves, b.ichild, b.iparent, b.lparent, b.ibox, b.lbox, b.counter,
            b.fibox, b.flbox, b.fshift, status_word());
    if (!is_float && b.fpts && n > 0 && !fpts_ready)
        k_fpts<<<grid_for(n, 256, 152 * 32), 256, 0, s>>>(pts, n, b.fpts, b.fshift);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
