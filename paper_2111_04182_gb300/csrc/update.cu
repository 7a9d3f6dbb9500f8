// update.cu -- batch insert and delete (Sec. 2 "Batch-dynamic updates",
// Algorithm 4; deletion "uses an almost identical algorithm").
//
// The tree after an update must equal the canonical tree of the new point
// set.  The canonical tree is a function of the sorted key array, and its
// leaf boundaries depend only on keys within L positions, so an update is:
// place the sorted batch into the sorted array (insert: a merge of two
// sorted runs by (key, id); delete: a stable compaction), then re-derive the
// leaves, internal nodes and boxes with the same kernels as a build.  The
// merge is the splitUsingBit routing of Algorithm 4 done for all batch keys
// at once by binary search.
#include "common.cuh"

namespace zdk {

// number of entries of a[0, n) that are < key (lower) or <= key (upper)
__device__ __forceinline__ int64_t lower_bound_u64(const u64 *a, int64_t lo, int64_t hi, u64 key)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t upper_bound_u64(const u64 *a, int64_t lo, int64_t hi, u64 key)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int MERGE_TILE = 1024;

// Existing element i goes to i + #(batch keys < key_i); batch element j to
// j + #(existing keys <= key_j).  Existing ids are all smaller than the new
// ids, so on equal keys the existing points come first: the result is sorted
// by (key, id).
__global__ void __launch_bounds__(256) k_merge_old(const u64 *__restrict__ keys, const int4 *__restrict__ pts,
                                                   int64_t n, const u64 *__restrict__ bkeys, int64_t b,
                                                   u64 *__restrict__ keys_out, int4 *__restrict__ pts_out,
                                                   float4 *__restrict__ fpts_out, uint3 fsh)
{
    __shared__ int64_t s_rng[2];
    const int64_t i0 = (int64_t)blockIdx.x * MERGE_TILE;
    if (i0 >= n) return;
    const int64_t i1 = min(i0 + MERGE_TILE, n);
    if (threadIdx.x == 0) {
        s_rng[0] = lower_bound_u64(bkeys, 0, b, keys[i0]);
        s_rng[1] = lower_bound_u64(bkeys, s_rng[0], b, keys[i1 - 1]);
    }
    __syncthreads();
    const int64_t lo = s_rng[0], hi = s_rng[1];
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const u64 key = keys[i];
        const int64_t c = lower_bound_u64(bkeys, lo, hi, key);
        const int4 p = pts[i];
        keys_out[i + c] = key;
        pts_out[i + c] = p;
        if (fpts_out) fpts_out[i + c] = shifted_float4(p, fsh);
    }
}

__global__ void __launch_bounds__(256) k_merge_new(const u64 *__restrict__ keys, int64_t n,
                                                   const u64 *__restrict__ bkeys, const int4 *__restrict__ bpts,
                                                   int64_t b, u64 *__restrict__ keys_out,
                                                   int4 *__restrict__ pts_out, float4 *__restrict__ fpts_out,
                                                   uint3 fsh)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b;
         j += (int64_t)gridDim.x * blockDim.x) {
        const u64 key = bkeys[j];
        const int64_t c = upper_bound_u64(keys, 0, n, key);
        const int4 p = bpts[j];
        keys_out[j + c] = key;
        pts_out[j + c] = p;
        if (fpts_out) fpts_out[j + c] = shifted_float4(p, fsh);
    }
}

// Liveness of ids is kept as two bitmaps: live bits in words [0, W) and
// marked-for-delete bits in words [W, 2W) (W = ceil(id capacity / 32)).  At 4
// bytes per 32 ids both stay resident in L2 for tens of millions of ids.
__global__ void k_live_bits(u32 *live, int64_t a, int64_t z, int set)
{
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < z;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u32 bit = 1u << (i & 31);
        if (set) atomicOr(&live[i >> 5], bit);
        else atomicAnd(&live[i >> 5], ~bit);
    }
}

__global__ void k_iota(int32_t *p, int64_t n, int32_t first)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)(first + i);
}

int update_live_bits(u32 *live, int64_t a, int64_t z, int set, cudaStream_t s)
{
    if (z <= a) return ZD_OK;
    k_live_bits<<<grid_for(z - a, 256, 4096), 256, 0, s>>>(live, a, z, set);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int update_insert(const TreeView &v, const u64 *keys, const int4 *pts, int64_t n, const void *d_pts,
                  int64_t b, int dim, int B, const uint32_t *shift, int key_bits, int32_t next_id,
                  u64 *keys_out, int4 *pts_out, u32 *live, int32_t *d_new_ids, Mem &mem, float4 *fpts_out)
{
    const uint3 fsh = make_uint3(shift ? shift[0] : 0u, shift ? shift[1] : 0u, shift ? shift[2] : 0u);
    (void)v;
    cudaStream_t s = mem.s;
    const int npasses = (key_bits + RADIX_BITS - 1) / RADIX_BITS;
    Scratch<u64> raw(mem, b), bkeys(mem, b);
    Scratch<int32_t> perm(mem, b);
    Scratch<int4> bpts(mem, b);
    Scratch<u32> hist(mem, MAX_PASSES * RADIX);
    if (!raw.p || !bkeys.p || !perm.p || !bpts.p || !hist.p) return ZD_ERR_OOM;
    ZD_CUDA(cudaMemsetAsync(hist.p, 0, MAX_PASSES * RADIX * sizeof(u32), s));
    ZD_TRY(launch_encode_i32((const int32_t *)d_pts, b, dim, B, shift, nullptr, 0, 0, raw.p, hist.p,
                             npasses, s));
    ZD_TRY(radix_sort(raw.p, b, key_bits, bkeys.p, perm.p, hist.p, mem));
    ZD_TRY(launch_gather(d_pts, dim, b, perm.p, bkeys.p, 64, nullptr, next_id, bpts.p, s));
    if (d_new_ids) k_iota<<<grid_for(b, 256, 4096), 256, 0, s>>>(d_new_ids, b, next_id);
    if (n > 0)
        k_merge_old<<<(unsigned)((n + MERGE_TILE - 1) / MERGE_TILE), 256, 0, s>>>(keys, pts, n, bkeys.p, b,
                                                                               keys_out, pts_out, fpts_out, fsh);
    k_merge_new<<<grid_for(b, 256, 152 * 16), 256, 0, s>>>(keys, n, bkeys.p, bpts.p, b, keys_out, pts_out,
                                                            fpts_out, fsh);
    k_live_bits<<<grid_for(b, 256, 4096), 256, 0, s>>>(live, next_id, next_id + b, 1);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// ----------------------------------------------------------------- delete
__global__ void k_mark(const u32 *live, u32 *marked, int64_t id_cap, const int32_t *__restrict__ ids, int64_t b,
                       int *err)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = ids[j];
        if (id < 0 || id >= id_cap) {
            atomicCAS(err, 0, ZD_ERR_NOT_FOUND);
            continue;
        }
        const u32 bit = 1u << (id & 31);
        if (!(live[id >> 5] & bit)) {
            atomicCAS(err, 0, ZD_ERR_NOT_FOUND);
            continue;
        }
        if (atomicOr(&marked[id >> 5], bit) & bit) atomicCAS(err, 0, ZD_ERR_DUPLICATE_ID);
    }
}

// Clear the marked bits of the batch's ids (and, with retire, their live bits).
__global__ void k_unmark(u32 *live, u32 *marked, int64_t id_cap, const int32_t *__restrict__ ids, int64_t b,
                         int retire)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = ids[j];
        if (id < 0 || id >= id_cap) continue;
        const u32 bit = 1u << (id & 31);
        atomicAnd(&marked[id >> 5], ~bit);
        if (retire) atomicAnd(&live[id >> 5], ~bit);
    }
}

int update_delete_mark(u32 *live, u32 *marked, int64_t id_cap, const int32_t *ids, int64_t b, Mem &mem,
                       int *result)
{
    cudaStream_t s = mem.s;
    Scratch<int> err(mem, 1);
    if (!err.p) return ZD_ERR_OOM;
    ZD_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_mark<<<grid_for(b, 256, 4096), 256, 0, s>>>(live, marked, id_cap, ids, b, err.p);
    ZD_CUDA(cudaGetLastError());
    int h = 0;
    ZD_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ZD_CUDA(cudaStreamSynchronize(s));
    *result = h;
    return ZD_OK;
}

int update_delete_unmark(u32 *live, u32 *marked, int64_t id_cap, const int32_t *ids, int64_t b, cudaStream_t s)
{
    k_unmark<<<grid_for(b, 256, 4096), 256, 0, s>>>(live, marked, id_cap, ids, b, 0);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// Stable compaction of the points whose id is not marked.  Element e of a
// tile is handled by thread e % 256 in step e / 256, so loads and stores of a
// warp touch consecutive elements; within a tile, kept elements are ranked in
// element order with ballots.
constexpr int CMP_THREADS = 256;
constexpr int CMP_ITEMS = 8;
constexpr int CMP_TILE = CMP_THREADS * CMP_ITEMS;

__global__ void __launch_bounds__(CMP_THREADS) k_keep_flags(const int4 *__restrict__ pts, int64_t n,
                                                           const u32 *__restrict__ marked,
                                                           unsigned char *__restrict__ keep, int *count)
{
    __shared__ int s_w[CMP_THREADS / 32];
    const int64_t t0 = (int64_t)blockIdx.x * CMP_TILE;
    int c = 0;
#pragma unroll
    for (int it = 0; it < CMP_ITEMS; ++it) {
        const int64_t i = t0 + it * CMP_THREADS + threadIdx.x;
        if (i < n) {
            const int id = pts[i].w;
            const unsigned char k = (marked[id >> 5] >> (id & 31)) & 1u ? 0 : 1;
            keep[i] = k;
            c += k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < CMP_THREADS / 32; ++w) t += s_w[w];
        count[blockIdx.x] = t;
    }
}

// in-place exclusive scan of count[0, nb) by one block
__global__ void __launch_bounds__(1024) k_excl_scan(int *count, int64_t nb)
{
    __shared__ int s_w[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        int v = i < nb ? count[i] : 0;
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
        if (i < nb) count[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CMP_THREADS) k_keep_scatter(const u64 *__restrict__ keys,
                                                             const int4 *__restrict__ pts, int64_t n,
                                                             const unsigned char *__restrict__ keep,
                                                             const int *__restrict__ off,
                                                             u64 *__restrict__ keys_out,
                                                             int4 *__restrict__ pts_out,
                                                             float4 *__restrict__ fpts_out, uint3 fsh)
{
    __shared__ int s_cnt[CMP_ITEMS][CMP_THREADS / 32];
    const int64_t t0 = (int64_t)blockIdx.x * CMP_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned ball[CMP_ITEMS];
#pragma unroll
    for (int it = 0; it < CMP_ITEMS; ++it) {
        const int64_t i = t0 + it * CMP_THREADS + threadIdx.x;
        ball[it] = __ballot_sync(0xffffffffu, i < n && keep[i]);
        if (lane == 0) s_cnt[it][warp] = __popc(ball[it]);
    }
    __syncthreads();
    // element order within the tile is (it, warp, lane): exclusive scan of the
    // (it, warp) counts in that order
    if (threadIdx.x == 0) {
        int run = 0;
        for (int q = 0; q < CMP_ITEMS * (CMP_THREADS / 32); ++q) {
            int &cq = s_cnt[q / (CMP_THREADS / 32)][q % (CMP_THREADS / 32)];
            const int c = cq;
            cq = run;
            run += c;
        }
    }
    __syncthreads();
    const int base = off[blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < CMP_ITEMS; ++it) {
        const int before = s_cnt[it][warp];
        if (ball[it] & (1u << lane)) {
            const int64_t i = t0 + it * CMP_THREADS + threadIdx.x;
            const int64_t pos = base + before + __popc(ball[it] & lt);
            const int4 p = pts[i];
            keys_out[pos] = keys[i];
            pts_out[pos] = p;
            if (fpts_out) fpts_out[pos] = shifted_float4(p, fsh);
        }
    }
}

int update_delete_compact(const u64 *keys, const int4 *pts, int64_t n, u32 *live, u32 *marked,
                          const int32_t *ids, int64_t b, int64_t id_cap, u64 *keys_out, int4 *pts_out, Mem &mem,
                          float4 *fpts_out, uint3 fsh)
{
    cudaStream_t s = mem.s;
    const int64_t nb = (n + CMP_TILE - 1) / CMP_TILE;
    Scratch<int> count(mem, nb > 0 ? nb : 1);
    Scratch<unsigned char> keep(mem, n > 0 ? n : 1);
    if (!count.p || !keep.p) return ZD_ERR_OOM;
    if (nb > 0) {
        k_keep_flags<<<(unsigned)nb, CMP_THREADS, 0, s>>>(pts, n, marked, keep.p, count.p);
        k_excl_scan<<<1, 1024, 0, s>>>(count.p, nb);
        k_keep_scatter<<<(unsigned)nb, CMP_THREADS, 0, s>>>(keys, pts, n, keep.p, count.p, keys_out, pts_out,
                                                            fpts_out, fsh);
    }
    k_unmark<<<grid_for(b, 256, 4096), 256, 0, s>>>(live, marked, id_cap, ids, b, 1);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
