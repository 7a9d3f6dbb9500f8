// sort.cu -- Morton encoding (Sec. 1.1) and the stable LSD radix sort by
// Morton key (Sec. 2 "Construction"; Theorem 1 argues a linear-work radix
// sort suffices).
//
// The sort is a "onesweep" LSD radix sort: one read-only pass (fused into the
// encoder) builds the digit histograms of every pass; then each pass ranks a
// tile of keys in shared memory and finds its global offsets by a decoupled
// look-back over the tiles before it, so a pass reads and writes the keys
// exactly once.  Passes whose digit is the same for every key are skipped on
// the device (no host round trip).  Every look-back wait is bounded.
#include <atomic>

#include "common.cuh"
#include "morton.cuh"

namespace zdk {

// ------------------------------------------------------------------ keys
// (the bit interleave itself is in morton.cuh)

// Cloud (segment) of row i: the last c with seg_off[c] <= i.
__device__ __forceinline__ int64_t segment_of(const int64_t *seg_off, int64_t n_seg, int64_t i)
{
    int64_t a = 0, z = n_seg - 1;
    while (a < z) {
        int64_t mid = (a + z + 1) >> 1;
        if (seg_off[mid] <= i) a = mid;
        else z = mid - 1;
    }
    return a;
}

// Digit histogram update.  The top digits repeat across neighbouring input
// points (a spatially coherent input shares its high Morton bits), so lanes
// holding the same top digit add once (match_any); the low digits are close
// to random and take plain shared-memory atomics.  All 32 lanes must call it
// (valid = false for padding lanes).
__device__ __forceinline__ void hist_add(u32 *sh, u64 key, bool valid, int npasses)
{
    const unsigned lane = threadIdx.x & 31;
    const int top = npasses > 3 ? npasses - 3 : 0;
    if (valid)
        for (int p = 0; p < top; ++p) atomicAdd(&sh[p * RADIX + (int)((key >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
    for (int p = top; p < npasses; ++p) {
        int d = valid ? (int)((key >> (RADIX_BITS * p)) & (RADIX - 1)) : RADIX;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < RADIX && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&sh[p * RADIX + d], __popc(peers));
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_encode_i32(const int32_t *__restrict__ pts, int64_t n, int B,
                                                    uint3 shift, const int64_t *__restrict__ seg_off,
                                                    int64_t n_seg, int cloud_shift,
                                                    u64 *__restrict__ keys, u32 *__restrict__ hist,
                                                    int npasses, u32 *status)
{
    __shared__ u32 sh[MAX_PASSES * RADIX];
    if (hist)
        for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t lim = (int64_t)1 << B;
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        u64 key = 0;
        if (valid) {
            int64_t c0 = (int64_t)pts[i * DIM + 0] + shift.x;
            int64_t c1 = (int64_t)pts[i * DIM + 1] + shift.y;
            int64_t c2 = DIM == 3 ? (int64_t)pts[i * DIM + 2] + shift.z : 0;
            bool ok = c0 >= 0 && c0 < lim && c1 >= 0 && c1 < lim && c2 >= 0 && c2 < lim;
            if (ok) key = interleave<DIM>((u64)c0, (u64)c1, (u64)c2);
            else bad = true;
            if (seg_off) key |= (u64)segment_of(seg_off, n_seg, i) << cloud_shift;
            keys[i] = key;
        }
        if (hist) hist_add(sh, key, valid, npasses);
    }
    if (bad) set_status(status, ZD_ERR_RANGE);
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

__global__ void __launch_bounds__(256) k_hist(const u64 *__restrict__ keys, int64_t n, u32 *hist,
                                              int npasses)
{
    __shared__ u32 sh[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        hist_add(sh, valid ? keys[i] : 0, valid, npasses);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ------------------------------------------------------ float quantization
// Order-preserving map float -> int, so atomicMin/atomicMax order floats.
__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Per-segment min / max of every coordinate.  grid = (chunks, n_seg).
__global__ void k_minmax(const float *__restrict__ pts, int64_t n, int dim,
                         const int64_t *__restrict__ seg_off, int *mm /* [n_seg][6] */)
{
    const int64_t seg = blockIdx.y;
    const int64_t a = seg_off ? seg_off[seg] : 0, z = seg_off ? seg_off[seg + 1] : n;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < z;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < dim; ++j) {
            int v = f2ord(pts[i * dim + j]);
            lo[j] = min(lo[j], v);
            hi[j] = max(hi[j], v);
        }
    for (int j = 0; j < 3; ++j)
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = min(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = max(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int j = 0; j < dim; ++j) {
            atomicMin(&mm[seg * 6 + j], lo[j]);
            atomicMax(&mm[seg * 6 + 3 + j], hi[j]);
        }
}

// frame[seg] = (lo_x, lo_y, lo_z, scale): scale = (2^B - 1) / (largest extent).
__global__ void k_frames(const int *mm, int64_t n_seg, int dim, int B, double *frame)
{
    int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= n_seg) return;
    double ext = 0.0;
    for (int j = 0; j < 3; ++j) {
        double lo = 0.0;
        if (j < dim && mm[seg * 6 + j] != INT_MAX) {
            lo = (double)ord2f(mm[seg * 6 + j]);
            double e = __dsub_rn((double)ord2f(mm[seg * 6 + 3 + j]), lo);
            ext = fmax(ext, e);
        }
        frame[seg * 4 + j] = lo;
    }
    double top = (double)((1ll << B) - 1);
    frame[seg * 4 + 3] = ext > 0.0 ? __ddiv_rn(top, ext) : 1.0;
}

__global__ void k_minmax_init(int *mm, int64_t n_seg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_seg * 6;
         i += (int64_t)gridDim.x * blockDim.x)
        mm[i] = (i % 6) < 3 ? INT_MAX : INT_MIN;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_encode_f32(const float *__restrict__ pts, int64_t n, int B,
                                                    const double *__restrict__ frame,
                                                    const int64_t *__restrict__ seg_off,
                                                    int64_t n_seg, int cloud_shift,
                                                    u64 *__restrict__ keys, u32 *__restrict__ hist,
                                                    int npasses, u32 *status)
{
    __shared__ u32 sh[MAX_PASSES * RADIX];
    if (hist)
        for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const double top = (double)((1ll << B) - 1);
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        u64 key = 0;
        if (valid) {
            int64_t seg = seg_off ? segment_of(seg_off, n_seg, i) : 0;
            const double *f = frame + seg * 4;
            u64 c[3] = {0, 0, 0};
            for (int j = 0; j < DIM; ++j) {
                // finite and at most 1e18 in magnitude (the search's fp32
                // estimates square coordinate differences)
                bad = bad || !(fabsf(pts[i * DIM + j]) <= 1e18f);
                double v = floor(__dmul_rn(__dsub_rn((double)pts[i * DIM + j], f[j]), f[3]));
                if (!(v >= 0.0)) v = 0.0;
                if (v > top) v = top;
                c[j] = (u64)v;
            }
            key = interleave<DIM>(c[0], c[1], c[2]);
            if (seg_off) key |= (u64)seg << cloud_shift;
            keys[i] = key;
        }
        if (hist) hist_add(sh, key, valid, npasses);
    }
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
    if (bad) set_status(status, ZD_ERR_RANGE);
}

int launch_encode_i32(const int32_t *pts, int64_t n, int dim, int coord_bits, const uint32_t *shift,
                      const int64_t *seg_off, int64_t n_seg, int cloud_shift, u64 *keys, u32 *hist,
                      int npasses, cudaStream_t s)
{
    if (n <= 0) return ZD_OK;
    uint3 sh = make_uint3(shift ? shift[0] : 0, shift ? shift[1] : 0, shift ? shift[2] : 0);
    unsigned g = grid_for(n, 256, 152 * 16);
    if (dim == 3)
        k_encode_i32<3><<<g, 256, 0, s>>>(pts, n, coord_bits, sh, seg_off, n_seg, cloud_shift, keys,
                                          hist, npasses, status_word());
    else
        k_encode_i32<2><<<g, 256, 0, s>>>(pts, n, coord_bits, sh, seg_off, n_seg, cloud_shift, keys,
                                          hist, npasses, status_word());
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int launch_float_frames(const float *pts, int64_t n, int dim, int coord_bits,
                        const int64_t *seg_off, int64_t n_seg, int64_t max_seg, double *frame,
                        int *mm, cudaStream_t s)
{
    if (n_seg <= 0) return ZD_OK;
    k_minmax_init<<<grid_for(n_seg * 6, 256, 4096), 256, 0, s>>>(mm, n_seg);
    int64_t chunks = (max_seg + 256 * 8 - 1) / (256 * 8);
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    if (n_seg > 65535) return ZD_ERR_INVALID_ARG;
    dim3 g((unsigned)chunks, (unsigned)n_seg);
    k_minmax<<<g, 256, 0, s>>>(pts, n, dim, seg_off, mm);
    k_frames<<<grid_for(n_seg, 128, 1 << 16), 128, 0, s>>>(mm, n_seg, dim, coord_bits, frame);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

int launch_encode_f32(const float *pts, int64_t n, int dim, int coord_bits, const double *frame,
                      const int64_t *seg_off, int64_t n_seg, int cloud_shift, u64 *keys, u32 *hist,
                      int npasses, cudaStream_t s)
{
    if (n <= 0) return ZD_OK;
    unsigned g = grid_for(n, 256, 152 * 16);
    if (dim == 3)
        k_encode_f32<3><<<g, 256, 0, s>>>(pts, n, coord_bits, frame, seg_off, n_seg, cloud_shift,
                                          keys, hist, npasses, status_word());
    else
        k_encode_f32<2><<<g, 256, 0, s>>>(pts, n, coord_bits, frame, seg_off, n_seg, cloud_shift,
                                          keys, hist, npasses, status_word());
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// ------------------------------------------------------------ radix sort
constexpr int SORT_THREADS = 256; // one thread per digit in the look-back
constexpr int SORT_ITEMS = 12; // 3072-key tiles: 4 blocks per SM (measured: sort -6% vs 16 keys, 2 blocks)
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SORT_WARPS = SORT_THREADS / 32;
// look-back word: 2 flag bits + a 30-bit count.  The count is a digit's
// running total over all tiles up to this one, so it is bounded by n, and n
// is at most ZD_MAX_KEYS = 2^30 - 1 (checked in radix_sort).
constexpr u32 LB_AGG = 1u << 30;
constexpr u32 LB_INC = 2u << 30;
constexpr u32 LB_COUNT = (1u << 30) - 1;
constexpr u64 LB_TIMEOUT_NS = 2000000000ull; // 2 s of wall time per wait
constexpr int LB_MAX_POLLS = 1 << 25;

struct SortPlan {
    u32 off[MAX_PASSES][RADIX]; // global start of every digit, per pass
    int qidx[MAX_PASSES];       // rank among the passes that run, -1 if skipped
    int Q;                      // passes that run
};


// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ u32 block_excl_scan256(u32 v, u32 *s_warp /* [8] */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 x = v;
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    u32 w = 0;
    for (int i = 0; i < warp; ++i) w += s_warp[i];
    __syncthreads();
    return w + x - v;
}

__global__ void __launch_bounds__(256) k_sort_plan(const u32 *hist, int64_t n, int npasses,
                                                   SortPlan *plan)
{
    __shared__ u32 s_warp[8];
    __shared__ int triv[MAX_PASSES];
    const int d = threadIdx.x;
    for (int p = 0; p < MAX_PASSES; ++p) {
        u32 c = p < npasses ? hist[p * RADIX + d] : 0;
        u32 excl = block_excl_scan256(c, s_warp);
        plan->off[p][d] = excl;
        int t = __syncthreads_or(p >= npasses || (int64_t)c == n);
        if (d == 0) triv[p] = t;
    }
    __syncthreads();
    if (d == 0) {
        int q = 0;
        for (int p = 0; p < MAX_PASSES; ++p) plan->qidx[p] = triv[p] ? -1 : q++;
        plan->Q = q;
    }
}

struct PassArgs {
    const u64 *keys_in;
    u64 *ktmp[2];
    u32 *vtmp[2];
    u64 *keys_out;
    u32 *vals_out;
    int64_t n;
    const SortPlan *plan;
    u32 *lookback;     // [MAX_PASSES][num_tiles][RADIX], zeroed
    u32 *tile_counter; // [MAX_PASSES], zeroed
    int64_t num_tiles;
    u32 *status;
};

__global__ void __launch_bounds__(SORT_THREADS, 4) k_onesweep(PassArgs a, int pass)
{
    const int q = a.plan->qidx[pass];
    if (q < 0) return; // every key has the same digit: nothing to do
    const int Q = a.plan->Q;
    // (selects, not indexing: a runtime index into the parameter arrays would
    // copy the parameters to local memory)
    const bool odd = q & 1;
    const u64 *ksrc = q == 0 ? a.keys_in : (odd ? a.ktmp[0] : a.ktmp[1]);
    const u32 *vsrc = q == 0 ? nullptr : (odd ? a.vtmp[0] : a.vtmp[1]);
    u64 *kdst = q == Q - 1 ? a.keys_out : (odd ? a.ktmp[1] : a.ktmp[0]);
    u32 *vdst = q == Q - 1 ? a.vals_out : (odd ? a.vtmp[1] : a.vtmp[0]);
    const int shift = pass * RADIX_BITS;

    extern __shared__ __align__(16) unsigned char smem[];
    u64 *s_keys = (u64 *)smem;                       // [SORT_TILE]
    u32 *s_vals = (u32 *)(s_keys + SORT_TILE);        // [SORT_TILE]
    u32 *s_whist = s_vals + SORT_TILE;                // [SORT_WARPS][RADIX]
    u32 *s_excl = s_whist + SORT_WARPS * RADIX;       // [RADIX] tile-local digit starts
    u32 *s_glob = s_excl + RADIX;                     // [RADIX] global digit bases
    u32 *s_misc = s_glob + RADIX;                     // [16]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_misc[8] = atomicAdd(&a.tile_counter[pass], 1u);
    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS) s_whist[i] = 0;
    __syncthreads();
    const int64_t tile = s_misc[8];
    const int64_t base = tile * SORT_TILE;
    const int valid_count = (int)min((int64_t)SORT_TILE, a.n - base);

    // Load: warp w owns a contiguous run of 32 * SORT_ITEMS keys; item i of
    // lane l is element w*32*ITEMS + i*32 + l, so (item, lane) order is the
    // input order and ranks come out stable.
    u64 k[SORT_ITEMS];
    u32 v[SORT_ITEMS];
    int dg[SORT_ITEMS];
    u32 rk[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        int e = warp * 32 * SORT_ITEMS + i * 32 + lane;
        int64_t g = base + e;
        bool valid = e < valid_count;
        k[i] = valid ? ksrc[g] : 0ull;
        v[i] = valid ? (vsrc ? vsrc[g] : (u32)g) : 0u;
        dg[i] = valid ? (int)((k[i] >> shift) & (RADIX - 1)) : RADIX;
    }
    // Rank inside the warp.  The lanes holding the same digit ("peers") are
    // found by one ballot per digit bit: a lane's peers agree with it on
    // every bit.  Unlike match_any, whose cost grows with the number of
    // distinct values in the warp, this costs the same for the near-random
    // low digits as for the coherent high ones (measured: the ranking of a
    // 4096-key tile 4.0 -> 2.8 us on the low digits).
    u32 *wh = s_whist + warp * RADIX;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool full = valid_count == SORT_TILE;
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < RADIX_BITS; ++b) {
            const bool bit = (dg[i] >> b) & 1;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        if (!full) { // padding lanes (digit RADIX) must not join digit 0
            const bool v = dg[i] < RADIX;
            const unsigned vb = __ballot_sync(0xffffffffu, v);
            peers &= v ? vb : ~vb;
        }
        int leader = __ffs(peers) - 1;
        u32 before = 0;
        if (lane == leader && dg[i] < RADIX) {
            before = wh[dg[i]];
            wh[dg[i]] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rk[i] = before + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();

    // Thread d owns digit d: tile count, warp offsets, look-back.
    const int d = tid;
    u32 cnt = 0;
    for (int w = 0; w < SORT_WARPS; ++w) {
        u32 c = s_whist[w * RADIX + d];
        s_whist[w * RADIX + d] = cnt;
        cnt += c;
    }
    u32 *lb = a.lookback + ((int64_t)pass * a.num_tiles) * RADIX;
    volatile u32 *my = lb + tile * RADIX + d;
    *my = (tile == 0 ? LB_INC : LB_AGG) | cnt;
    u32 excl_tile = block_excl_scan256(cnt, s_misc);
    s_excl[d] = excl_tile;

    u32 prefix = 0;
    if (tile > 0) {
        int64_t t = tile - 1;
        for (;;) {
            volatile const u32 *p = lb + t * RADIX + d;
            u32 w;
            if (!wait_for_flag(p, ~LB_COUNT, LB_TIMEOUT_NS, LB_MAX_POLLS, w)) {
                set_status(a.status, ZD_ERR_TIMEOUT);
                w = LB_INC; // give up: treat as complete so the pass ends
            }
            prefix += w & LB_COUNT;
            if ((w & ~LB_COUNT) == LB_INC || t == 0) break;
            --t;
        }
        *my = LB_INC | (prefix + cnt);
    }
    s_glob[d] = a.plan->off[pass][d] + prefix;
    __syncthreads();

    // Stage the tile in digit order in shared memory ...
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        if (dg[i] < RADIX) {
            u32 pos = s_excl[dg[i]] + s_whist[warp * RADIX + dg[i]] + rk[i];
            if (!ZD_DCHECK(pos < (u32)valid_count, a.status)) continue;
            s_keys[pos] = k[i];
            s_vals[pos] = v[i];
        }
    }
    __syncthreads();
    // ... and write runs of equal digits to their global places.
    for (int j = tid; j < valid_count; j += SORT_THREADS) {
        u64 key = s_keys[j];
        int dj = (int)((key >> shift) & (RADIX - 1));
        u64 gpos = (u64)s_glob[dj] + (u64)(j - (int)s_excl[dj]);
        if (!ZD_DCHECK(gpos < (u64)a.n, a.status)) continue;
        kdst[gpos] = key;
        vdst[gpos] = s_vals[j];
    }
}

// No pass ran (n <= 1 or every key equal): output = input, identity order.
__global__ void k_sort_finish(const SortPlan *plan, const u64 *keys_in, int64_t n, u64 *keys_out,
                              u32 *vals_out)
{
    if (plan->Q != 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        keys_out[i] = keys_in[i];
        vals_out[i] = (u32)i;
    }
}

static size_t onesweep_smem()
{
    return (size_t)SORT_TILE * 8 + (size_t)SORT_TILE * 4 + (size_t)SORT_WARPS * RADIX * 4 +
           2 * RADIX * 4 + 16 * 4;
}

int radix_sort(const u64 *keys_in, int64_t n, int key_bits, u64 *keys_out, int32_t *perm_out,
               u32 *hist, Mem &mem)
{
    if (n < 0 || key_bits < 1 || key_bits > 64) return ZD_ERR_INVALID_ARG;
    static_assert(ZD_MAX_KEYS <= LB_COUNT, "look-back counts must hold n");
    if (n > ZD_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (n == 0) return ZD_OK;
    cudaStream_t s = mem.s;
    const int npasses = (key_bits + RADIX_BITS - 1) / RADIX_BITS;
    const int64_t num_tiles = (n + SORT_TILE - 1) / SORT_TILE;

    Scratch<u32> own_hist(mem, hist ? 1 : MAX_PASSES * RADIX);
    if (!own_hist.p) return ZD_ERR_OOM;
    if (!hist) {
        hist = own_hist.p;
        ZD_CUDA(cudaMemsetAsync(hist, 0, MAX_PASSES * RADIX * sizeof(u32), s));
        k_hist<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(keys_in, n, hist, npasses);
        ZD_CUDA(cudaGetLastError());
    }
    Scratch<SortPlan> plan(mem, 1);
    Scratch<u32> lookback(mem, (size_t)npasses * num_tiles * RADIX + MAX_PASSES);
    const int ntmp = npasses >= 3 ? 2 : (npasses == 2 ? 1 : 0);
    Scratch<u64> k0(mem, ntmp >= 1 ? n : 1), k1(mem, ntmp >= 2 ? n : 1);
    Scratch<u32> v0(mem, ntmp >= 1 ? n : 1), v1(mem, ntmp >= 2 ? n : 1);
    if (!plan.p || !lookback.p || !k0.p || !k1.p || !v0.p || !v1.p) return ZD_ERR_OOM;
    u32 *tile_counter = lookback.p + (size_t)npasses * num_tiles * RADIX;
    ZD_CUDA(cudaMemsetAsync(lookback.p, 0,
                            ((size_t)npasses * num_tiles * RADIX + MAX_PASSES) * sizeof(u32), s));
    k_sort_plan<<<1, 256, 0, s>>>(hist, n, npasses, plan.p);
    ZD_CUDA(cudaGetLastError());

    ZD_CUDA(cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem()));
    PassArgs a;
    a.keys_in = keys_in;
    a.ktmp[0] = k0.p;
    a.ktmp[1] = k1.p;
    a.vtmp[0] = v0.p;
    a.vtmp[1] = v1.p;
    a.keys_out = keys_out;
    a.vals_out = (u32 *)perm_out;
    a.n = n;
    a.plan = plan.p;
    a.lookback = lookback.p;
    a.tile_counter = tile_counter;
    a.num_tiles = num_tiles;
    a.status = status_word();
    for (int p = 0; p < npasses; ++p) {
        k_onesweep<<<(unsigned)num_tiles, SORT_THREADS, onesweep_smem(), s>>>(a, p);
        ZD_CUDA(cudaGetLastError());
    }
    k_sort_finish<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(plan.p, keys_in, n, keys_out,
                                                           (u32 *)perm_out);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk

// ------------------------------------------------- sort without allocation
// zd_morton_sort_noalloc: the same passes as radix_sort, with every scratch
// buffer carved out of one file-scope device array instead of allocated.
// The array is a static __device__ object of this library, so every GPU
// that loads the library keeps it until the process exits.
namespace zdk {

constexpr int64_t NOALLOC_TILES = (ZD_NOALLOC_MAX_KEYS + SORT_TILE - 1) / SORT_TILE;
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_HIST = 0;
constexpr size_t NA_PLAN = na_align(NA_HIST + sizeof(u32) * MAX_PASSES * RADIX);
constexpr size_t NA_LB = na_align(NA_PLAN + sizeof(SortPlan));
constexpr size_t NA_LB_WORDS = (size_t)MAX_PASSES * NOALLOC_TILES * RADIX + MAX_PASSES;
constexpr size_t NA_K0 = na_align(NA_LB + sizeof(u32) * NA_LB_WORDS);
constexpr size_t NA_K1 = NA_K0 + sizeof(u64) * ZD_NOALLOC_MAX_KEYS;
constexpr size_t NA_V0 = NA_K1 + sizeof(u64) * ZD_NOALLOC_MAX_KEYS;
constexpr size_t NA_V1 = NA_V0 + sizeof(u32) * ZD_NOALLOC_MAX_KEYS;
constexpr size_t NA_BYTES = NA_V1 + sizeof(u32) * ZD_NOALLOC_MAX_KEYS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the scratch array on the current device.  In host code
// the symbol itself is only a host-side stand-in, so the address is looked
// up once per device (cudaGetSymbolAddress, with that device current) and
// cached.  The cache entries are atomics: two host threads making their first
// call at once both look the address up and store the same value.
static unsigned char *noalloc_scratch()
{
    static std::atomic<unsigned char *> addr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    unsigned char *a = addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        a = (unsigned char *)p;
        addr[dev].store(a, std::memory_order_release);
    }
    return a;
}

} // namespace zdk

extern "C" int zd_morton_sort_noalloc(const uint64_t *d_keys_in, int64_t n, int key_bits, uint64_t *d_keys_out,
                                      int32_t *d_perm_out, void *stream)
{
    zdk::NvtxScope nvtx_("zd_morton_sort_noalloc");
    using namespace zdk;
    if (n < 0 || key_bits < 1 || key_bits > 64) return ZD_ERR_INVALID_ARG;
    if (n > ZD_NOALLOC_MAX_KEYS) return ZD_ERR_CAPACITY;
    if (n > 0 && (!d_keys_in || !d_keys_out || !d_perm_out)) return ZD_ERR_INVALID_ARG;
    unsigned char *base = noalloc_scratch();
    u32 *status = status_word();
    if (!base || !status) return ZD_ERR_CUDA;
    if (n == 0) return ZD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const u64 *keys_in = (const u64 *)d_keys_in;
    const int npasses = (key_bits + RADIX_BITS - 1) / RADIX_BITS;
    const int64_t num_tiles = (n + SORT_TILE - 1) / SORT_TILE;
    u32 *hist = (u32 *)(base + NA_HIST);
    SortPlan *plan = (SortPlan *)(base + NA_PLAN);
    u32 *lookback = (u32 *)(base + NA_LB);
    u32 *tile_counter = lookback + (size_t)npasses * num_tiles * RADIX;
    // the array keeps the previous call's contents: clear what counts
    ZD_CUDA(cudaMemsetAsync(hist, 0, sizeof(u32) * MAX_PASSES * RADIX, s));
    ZD_CUDA(cudaMemsetAsync(lookback, 0, sizeof(u32) * ((size_t)npasses * num_tiles * RADIX + MAX_PASSES), s));
    k_hist<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(keys_in, n, hist, npasses);
    k_sort_plan<<<1, 256, 0, s>>>(hist, n, npasses, plan);
    ZD_CUDA(cudaGetLastError());
    ZD_CUDA(cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem()));
    PassArgs a;
    a.keys_in = keys_in;
    a.ktmp[0] = (u64 *)(base + NA_K0);
    a.ktmp[1] = (u64 *)(base + NA_K1);
    a.vtmp[0] = (u32 *)(base + NA_V0);
    a.vtmp[1] = (u32 *)(base + NA_V1);
    a.keys_out = (u64 *)d_keys_out;
    a.vals_out = (u32 *)d_perm_out;
    a.n = n;
    a.plan = plan;
    a.lookback = lookback;
    a.tile_counter = tile_counter;
    a.num_tiles = num_tiles;
    a.status = status;
    for (int p = 0; p < npasses; ++p) {
        k_onesweep<<<(unsigned)num_tiles, SORT_THREADS, onesweep_smem(), s>>>(a, p);
        ZD_CUDA(cudaGetLastError());
    }
    k_sort_finish<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(plan, keys_in, n, (u64 *)d_keys_out, (u32 *)d_perm_out);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

// ------------------------------------------------ failure-detection check
namespace zdk {
static __device__ u32 g_never_set; // no code ever writes it

__global__ void k_wait_selftest(const u32 *flag, unsigned long long timeout_ns, u32 *status)
{
    u32 w;
    if (!wait_for_flag(flag, 0xffffffffu, timeout_ns, LB_MAX_POLLS, w)) set_status(status, ZD_ERR_TIMEOUT);
}
} // namespace zdk

extern "C" int zd_selftest_wait_timeout(int timeout_ms, void *stream)
{
    using namespace zdk;
    if (timeout_ms < 1 || timeout_ms > 2000) return ZD_ERR_INVALID_ARG;
    u32 *status = status_word();
    void *flag = nullptr;
    if (!status || cudaGetSymbolAddress(&flag, g_never_set) != cudaSuccess) return ZD_ERR_CUDA;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>((const u32 *)flag, (unsigned long long)timeout_ms * 1000000ull,
                                                       status);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}
