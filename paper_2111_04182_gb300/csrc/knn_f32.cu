// knn_f32.cu -- float-coordinate instantiations of the k-NN search (fp64
// neighbour ranking).
#include "knn_impl.cuh"

namespace zdk {
int launch_knn_f32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_dim<3, true>(a, s) : launch_knn_dim<2, true>(a, s);
}
} // namespace zdk
