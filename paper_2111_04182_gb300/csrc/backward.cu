// backward.cu -- gradient of loss = sum gout * || q_i - ref_idx(i,j) ||
// (an extension: the paper has no differentiable form).
//
// dq_i   =  sum_j g_ij * u_ij,        u_ij = (q_i - ref_t) / || q_i - ref_t ||
// dref_t = -sum_{(i,j): idx(i,j) = t} g_ij * u_ij
//
// The forward keeps only the neighbour ids; distances are recomputed here
// from the fp32 coordinates.  A gradient component is a sum of unit-vector
// components that often nearly cancel, so plain fp32 unit vectors (relative
// error ~2^-22 each) leave components near 1e-3 with relative errors of a few
// 1e-4.  Every term is therefore carried as an unevaluated sum of two fp32
// numbers ("double-float", Dekker 1971): the exact difference by TwoSum
// (Knuth), exact squares by FMA, 1/|d| by one Newton step on the fp32
// reciprocal square root, and the sums by TwoSum.  All of it runs on the
// fp32 pipe (GB300's fp64 pipe is narrow); each output is the double-float
// result rounded once to fp32.
//
// dq is a plain per-row sum.  dref is made deterministic without atomics:
// the (i, j) pairs are stably sorted by target (the library's radix sort), so
// each target's contributions are contiguous and are summed in pair order by
// one thread.
#include "common.cuh"

namespace zdk {

// s + e = a + b exactly (TwoSum).  The _rn intrinsics are never contracted
// or reassociated by the compiler.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// g * (q - r) / |q - r| as uh + ul (double-float, relative error ~2^-44);
// zero when q == r.
template <int DIM>
__device__ __forceinline__ void unit_diff(const float *q, const float *r, float g, float *uh, float *ul)
{
    float dh[3] = {0.f, 0.f, 0.f}, dl[3] = {0.f, 0.f, 0.f};
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        two_sum(q[c], -r[c], dh[c], dl[c]); // q - r = dh + dl exactly
        mx = fmaxf(mx, fabsf(dh[c]));
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) uh[c] = ul[c] = 0.f;
    if (mx == 0.f) return; // fl(q - r) = 0 only when q == r
    // u does not depend on the scale of d: bring the largest component into
    // [1, 2) by an exact power of two so that squares neither under- nor
    // overflow.
    unsigned ex = (__float_as_uint(mx) >> 23) & 0xffu;
    ex = ex > 253u ? 253u : ex;
    const float sc = __uint_as_float((254u - ex) << 23); // 2^(127 - ex)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        dh[c] = __fmul_rn(dh[c], sc);
        dl[c] = __fmul_rn(dl[c], sc);
    }
    // s = |d|^2 = sh + sl
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const float p = __fmul_rn(dh[c], dh[c]);
        const float pe = __fmaf_rn(dh[c], dh[c], -p); // dh^2 = p + pe exactly
        float e;
        two_sum(sh, p, sh, e);
        sl = __fadd_rn(sl, __fadd_rn(e, __fadd_rn(pe, __fmul_rn(2.f, __fmul_rn(dh[c], dl[c])))));
    }
    {
        float e;
        two_sum(sh, sl, sh, e);
        sl = e;
    }
    // y = 1/sqrt(s): y0 from the fp32 reciprocal square root, then one Newton
    // step y = y0 (1 + (1 - s y0^2) / 2) with the residual taken in
    // double-float (quadratic convergence: ~2^-44 from ~2^-22).
    const float y0 = rsqrtf(sh);
    const float qh = __fmul_rn(y0, y0);
    const float ql = __fmaf_rn(y0, y0, -qh);
    float res = __fmaf_rn(-sh, qh, 1.f);
    res = __fsub_rn(res, __fadd_rn(__fmul_rn(sh, ql), __fmul_rn(sl, qh)));
    const float yh = y0, yl = __fmul_rn(0.5f, __fmul_rn(y0, res));
    // w = g y
    const float wh = __fmul_rn(g, yh);
    const float wl = __fadd_rn(__fmaf_rn(g, yh, -wh), __fmul_rn(g, yl));
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        uh[c] = __fmul_rn(wh, dh[c]);
        ul[c] = __fadd_rn(__fmaf_rn(wh, dh[c], -uh[c]), __fadd_rn(__fmul_rn(wh, dl[c]), __fmul_rn(wl, dh[c])));
    }
}

// acc (hi, lo) += (uh, ul)
__device__ __forceinline__ void df_add(float &ah, float &al, float uh, float ul)
{
    float e;
    two_sum(ah, uh, ah, e);
    al = __fadd_rn(al, __fadd_rn(ul, e));
}

template <int DIM>
__global__ void __launch_bounds__(256) k_grad_q(const float *__restrict__ q, const float *__restrict__ ref,
                                                const int32_t *__restrict__ idx, int64_t batch, int64_t m,
                                                int64_t r, int k, const float *__restrict__ gout, int per,
                                                float *__restrict__ gq)
{
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < batch * m;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = row / m;
        float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < k; ++j) {
            const int32_t t = idx[row * k + j];
            if (t < 0 || t >= r) continue;
            float uh[3], ul[3];
            unit_diff<DIM>(q + row * DIM, ref + (p * r + t) * DIM, per ? gout[row * k + j] : gout[0], uh, ul);
#pragma unroll
            for (int c = 0; c < DIM; ++c) df_add(ah[c], al[c], uh[c], ul[c]);
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) gq[row * DIM + c] = __fadd_rn(ah[c], al[c]);
    }
}

// Key of pair e: its global target p*r + t, or batch*r for a skipped pair.
__global__ void k_pair_keys(const int32_t *__restrict__ idx, int64_t batch, int64_t m, int64_t r, int k,
                            u64 *__restrict__ keys)
{
    const int64_t P = batch * m * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / (m * k);
        const int32_t t = idx[e];
        keys[e] = (t < 0 || t >= r) ? (u64)(batch * r) : (u64)(p * r + t);
    }
}

__global__ void k_seg_start(const u64 *__restrict__ skeys, int64_t P, int64_t nt, int *__restrict__ seg)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < P;
         s += (int64_t)gridDim.x * blockDim.x) {
        const u64 key = skeys[s];
        if (key < (u64)nt && (s == 0 || skeys[s - 1] != key)) seg[key] = (int)s;
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_grad_ref(const float *__restrict__ q, const float *__restrict__ ref,
                                                  const u64 *__restrict__ skeys,
                                                  const int32_t *__restrict__ perm, const int *__restrict__ seg,
                                                  int64_t P, int64_t nt, int k, const float *__restrict__ gout,
                                                  int per, float *__restrict__ gref)
{
    for (int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; T < nt;
         T += (int64_t)gridDim.x * blockDim.x) {
        float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
        int64_t s = seg[T];
        if (s >= 0) {
            for (; s < P && skeys[s] == (u64)T; ++s) {
                const int64_t e = perm[s];
                const int64_t row = e / k;
                float uh[3], ul[3];
                unit_diff<DIM>(q + row * DIM, ref + T * DIM, per ? gout[e] : gout[0], uh, ul);
#pragma unroll
                for (int c = 0; c < DIM; ++c) df_add(ah[c], al[c], uh[c], ul[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) gref[T * DIM + c] = -__fadd_rn(ah[c], al[c]);
    }
}

__global__ void k_fill_i32(int *p, int64_t n, int v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

int launch_backward(const float *q, const float *ref, const int32_t *idx, int64_t batch, int64_t m,
                    int64_t r, int dim, int k, const float *gout, int gout_per, float *gq, float *gref,
                    Mem &mem)
{
    cudaStream_t s = mem.s;
    const int64_t rows = batch * m, P = rows * k, nt = batch * r;
    if (rows > 0) {
        if (dim == 3)
            k_grad_q<3><<<grid_for(rows, 256, 152 * 32), 256, 0, s>>>(q, ref, idx, batch, m, r, k, gout,
                                                                     gout_per, gq);
        else
            k_grad_q<2><<<grid_for(rows, 256, 152 * 32), 256, 0, s>>>(q, ref, idx, batch, m, r, k, gout,
                                                                     gout_per, gq);
        ZD_CUDA(cudaGetLastError());
    }
    if (nt == 0) return ZD_OK;
    Scratch<u64> keys(mem, P > 0 ? P : 1), skeys(mem, P > 0 ? P : 1);
    Scratch<int32_t> perm(mem, P > 0 ? P : 1);
    Scratch<int> seg(mem, nt);
    if (!keys.p || !skeys.p || !perm.p || !seg.p) return ZD_ERR_OOM;
    k_fill_i32<<<grid_for(nt, 256, 4096), 256, 0, s>>>(seg.p, nt, -1);
    if (P > 0) {
        k_pair_keys<<<grid_for(P, 256, 152 * 32), 256, 0, s>>>(idx, batch, m, r, k, keys.p);
        int bits = 1;
        while (bits < 64 && ((u64)1 << bits) <= (u64)nt) ++bits;
        ZD_TRY(radix_sort(keys.p, P, bits, skeys.p, perm.p, nullptr, mem));
        k_seg_start<<<grid_for(P, 256, 152 * 32), 256, 0, s>>>(skeys.p, P, nt, seg.p);
    }
    if (dim == 3)
        k_grad_ref<3><<<grid_for(nt, 256, 152 * 32), 256, 0, s>>>(q, ref, skeys.p, perm.p, seg.p, P, nt, k,
                                                                  gout, gout_per, gref);
    else
        k_grad_ref<2><<<grid_for(nt, 256, 152 * 32), 256, 0, s>>>(q, ref, skeys.p, perm.p, seg.p, P, nt, k,
                                                                  gout, gout_per, gref);
    ZD_CUDA(cudaGetLastError());
    return ZD_OK;
}

} // namespace zdk
