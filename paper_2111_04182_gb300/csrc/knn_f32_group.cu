// knn_f32_group.cu -- float-coordinate warp-group k-NN search (fp32
// estimates, exact fp64 finish) and its exact fallback.  The kernels are
// instantiated in knn_f32_group_{3,2}{n,w}.cu (by dimension and list width)
// so that they compile in parallel.
#include "common.cuh"

namespace zdk {
int launch_knn_group_f_3n(const KnnArgs &a, cudaStream_t s);
int launch_knn_group_f_3w(const KnnArgs &a, cudaStream_t s);
int launch_knn_group_f_2n(const KnnArgs &a, cudaStream_t s);
int launch_knn_group_f_2w(const KnnArgs &a, cudaStream_t s);

// Warp groups, then the exact kernel for the queries whose band overflowed
// the buffer.
int launch_knn_group_f32(const KnnArgs &a, cudaStream_t s)
{
    ZD_CUDA(cudaMemsetAsync(a.fix_count, 0, sizeof(int), s));
    if (a.n_groups > 0) {
        KnnArgs b = a;
        if (b.chunk_ctr) { // the SM-affine group feed
            ZD_CUDA(cudaMemsetAsync(b.chunk_ctr, 0, sizeof(int) * (size_t)b.n_chunks, s));
            b.chunk_len = (b.n_groups + b.n_chunks - 1) / b.n_chunks;
        }
        if (b.t.dim == 3) ZD_TRY(b.k <= 16 ? launch_knn_group_f_3n(b, s) : launch_knn_group_f_3w(b, s));
        else ZD_TRY(b.k <= 16 ? launch_knn_group_f_2n(b, s) : launch_knn_group_f_2w(b, s));
    }
    KnnArgs f = a;
    f.sel = a.fix_list;
    f.sel_count = a.fix_count;
    // forest external queries fall back to the root-based search, which
    // descends to the query's own cloud first
    if (a.t.cloud_off && a.mode == ZD_SEARCH_BIT) f.mode = ZD_SEARCH_ROOT;
    return launch_knn_f32(f, s);
}
} // namespace zdk
