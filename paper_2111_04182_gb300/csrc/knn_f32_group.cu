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

// Warp groups, then the exact kernel for the queries whose band overflowed.
int launch_knn_group_f32(const KnnArgs &a, cudaStream_t s)
{
    ZD_CUDA(cudaMemsetAsync(a.fix_count, 0, sizeof(int), s));
    if (a.n_groups > 0) {
        if (a.t.dim == 3) ZD_TRY(a.k <= 16 ? launch_knn_group_f_3n(a, s) : launch_knn_group_f_3w(a, s));
        else ZD_TRY(a.k <= 16 ? launch_knn_group_f_2n(a, s) : launch_knn_group_f_2w(a, s));
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
