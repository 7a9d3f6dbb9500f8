// backward.cu -- gradient of loss = sum gout * || q_i - ref_idx(i,j) ||
// (an extension: the paper has no differentiable form).
//
// dq_i   =  sum_j g_ij * u_ij,        u_ij = (q_i - ref_t) / || q_i - ref_t ||
// dref_t = -sum_{(i,j): idx(i,j) = t} g_ij * u_ij
//
// The forward keeps only the neighbour ids; distances are recomputed in fp32.
// dq is a plain per-row sum.  dref is made deterministic without atomics:
// the (i, j) pairs are stably sorted by target (the library's radix sort), so
// each target's contributions are contiguous and are summed in pair order by
// one thread.
#include "common.cuh"

namespace zdk {

template <int DIM>
__device__ __forceinline__ void unit_diff(const float *q, const float *r, float g, float *u)
{
    float d[3] = {0.f, 0.f, 0.f};
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        d[c] = q[c] - r[c];
        s += d[c] * d[c];
    }
    const float dist = sqrtf(s);
    const float w = dist > 0.f ? g / dist : 0.f;
#pragma unroll
    for (int c = 0; c < DIM; ++c) u[c] = w * d[c];
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
        float acc[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < k; ++j) {
            const int32_t t = idx[row * k + j];
            if (t < 0 || t >= r) continue;
            float u[3];
            unit_diff<DIM>(q + row * DIM, ref + (p * r + t) * DIM, per ? gout[row * k + j] : gout[0], u);
#pragma unroll
            for (int c = 0; c < DIM; ++c) acc[c] += u[c];
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) gq[row * DIM + c] = acc[c];
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
        float acc[3] = {0.f, 0.f, 0.f};
        int64_t s = seg[T];
        if (s >= 0) {
            for (; s < P && skeys[s] == (u64)T; ++s) {
                const int64_t e = perm[s];
                const int64_t row = e / k;
                float u[3];
                unit_diff<DIM>(q + row * DIM, ref + T * DIM, per ? gout[e] : gout[0], u);
#pragma unroll
                for (int c = 0; c < DIM; ++c) acc[c] += u[c];
            }
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) gref[T * DIM + c] = -acc[c];
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
