// knn_f32_group_3n.cu -- float warp-group k-NN kernels, 3D, narrow lists.
#include "knn_group_f.cuh"

namespace zdk {
int launch_knn_group_f_3n(const KnnArgs &a, cudaStream_t s)
{
    return launch_knn_group_f_narrow<3>(a, s);
}
} // namespace zdk
