// knn_i32.cu -- integer-coordinate instantiations of the k-NN search.
#include "knn_impl.cuh"

namespace zdk {
int launch_knn_i32(const KnnArgs &a, cudaStream_t s)
{
    return a.t.dim == 3 ? launch_knn_dim<3, false>(a, s) : launch_knn_dim<2, false>(a, s);
}
} // namespace zdk
