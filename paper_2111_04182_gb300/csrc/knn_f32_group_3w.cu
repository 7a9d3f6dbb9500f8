// knn_f32_group_3w.cu -- float warp-group k-NN kernels, 3D, wide lists.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_group_f_3w(const KnnArgs &a, cudaStream_t s)
{
    return launch_knn_group_f_wide<3>(a, s);
}
} // namespace zdk
