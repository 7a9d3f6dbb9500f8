// knn_f32.cu -- float-coordinate instantiations of the k-NN search (fp64
// neighbour ranking): one thread per query, and warp groups.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_f32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_dim<3, true>(a, s) : launch_knn_dim<2, true>(a, s);
}

int launch_knn_group_f32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_group_f_dim<3>(a, s) : launch_knn_group_f_dim<2>(a, s);
}
} // namespace zdk
