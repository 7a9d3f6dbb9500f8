// knn_f32_group_2w.cu -- float warp-group k-NN kernels, 2D, wide lists.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_group_f_2w(const KnnArgs &a, cudaStream_t s)
{
    return launch_knn_group_f_wide<2>(a, s);
}
} // namespace zdk
