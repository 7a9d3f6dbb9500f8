// knn_wide.cu -- instantiations of the large-k search (32 < k <= 128, one
// warp per query) for integer and float trees, 2D and 3D.
#include "knn_wide.cuh"

namespace zdk {
int launch_knn_wide(const KnnArgs &a, cudaStream_t s)
{
    if (a.k > ZD_MAX_K) return ZD_ERR_UNIMPLEMENTED;
    if (a.is_float) return a.t.dim == 3 ? launch_knn_wide_dim<3, true>(a, s) : launch_knn_wide_dim<2, true>(a, s);
    return a.t.dim == 3 ? launch_knn_wide_dim<3, false>(a, s) : launch_knn_wide_dim<2, false>(a, s);
}
} // namespace zdk
