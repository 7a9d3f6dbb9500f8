// knn_f32.cu -- float-coordinate instantiations of the one-thread-per-query
// k-NN search (fp64 neighbour ranking), 3D.  The 2D ones live in
// knn_f32_2d.cu and the warp groups in knn_f32_group.cu, so that the three
// compile in parallel.
#include "knn_impl.cuh"

namespace zdk {
int launch_knn_f32_2d(const KnnArgs &a, cudaStream_t s);

int launch_knn_f32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_dim<3, true>(a, s) : launch_knn_f32_2d(a, s);
}
} // namespace zdk
