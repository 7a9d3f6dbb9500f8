// knn_f32_group_2n.cu -- float warp-group k-NN kernels, 2D, narrow lists.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_group_f_2n(const KnnArgs &a, cudaStream_t s)
{
    return launch_knn_group_f_narrow<2>(a, s);
}
} // namespace zdk
