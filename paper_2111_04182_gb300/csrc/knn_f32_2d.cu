// knn_f32_2d.cu -- float-coordinate one-thread-per-query k-NN search, 2D.
#include "knn_impl.cuh"

namespace zdk {
int launch_knn_f32_2d(const KnnArgs &a, cudaStream_t s)
{
    return launch_knn_dim<2, true>(a, s);
}
} // namespace zdk
