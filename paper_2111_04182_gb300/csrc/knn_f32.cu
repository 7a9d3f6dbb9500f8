// knn_f32.cu -- float-coordinate instantiations of the k-NN search (fp64
// neighbour ranking): one thread per query, and warp groups.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_f32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_dim<3, true>(a, s) : launch_knn_dim<2, true>(a, s);
}

// Warp groups, then the exact kernel for the queries whose band overflowed.
int launch_knn_group_f32(const KnnArgs &a, cudaStream_t s)
{
    ZD_CUDA(cudaMemsetAsync(a.fix_count, 0, sizeof(int), s));
    ZD_TRY(a.t.dim == 3 ? launch_knn_group_f_dim<3>(a, s) : launch_knn_group_f_dim<2>(a, s));
    KnnArgs f = a;
    f.sel = a.fix_list;
    f.sel_count = a.fix_count;
    // forest external queries fall back to the root-based search, which
    // descends to the query's own cloud first
    if (a.t.cloud_off && a.mode == ZD_SEARCH_BIT) f.mode = ZD_SEARCH_ROOT;
    return launch_knn_f32(f, s);
}
} // namespace zdk
