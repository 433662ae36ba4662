// FP32 3D team collide kernel (two lanes per line transform): instantiations and their launch
// entry points, variants 5 (one row per team) and 6 (two rows per team).
#include "ef_cluster_launch.h"
#include "ef_collide_tm.cuh"
#include "ef_launch.h"

namespace ef {

namespace {

// launch bound (0: not built for N) and the CTAs per SM the registers are sized for
template <int N>
constexpr int tm_bound() { return N == 24 ? 288 : N == 32 ? 256 : N == 40 ? 400 : N == 48 ? 384 : 0; }
template <int N>
constexpr int tm_minb() { return (N == 24 || N == 32) ? 2 : 1; }
template <int N, int V>
constexpr auto tm_kernel()
{
    return collide_kernel_tm<3, N, V == 6 ? 2 : 1, tm_bound<N>(), tm_minb<N>()>;
}

}  // namespace

#define EF_TM_SIZES(X) X(24) X(32) X(40) X(48)

int tm_maxthreads_f32(int N)
{
    switch (N) {
#define EF_CASE(n) case n: return tm_bound<n>();
        EF_TM_SIZES(EF_CASE)
#undef EF_CASE
    default: return 0;
    }
}

cudaError_t tm_setup_f32(int N, int v, size_t smem, int cluster, int tpb, int *max_clusters)
{
    switch (N) {
#define EF_CASE(n)                                                                                       \
    case n:                                                                                              \
        return v == 5 ? setup_kernel(tm_kernel<n, 5>(), smem, cluster, tpb, max_clusters)                \
                      : setup_kernel(tm_kernel<n, 6>(), smem, cluster, tpb, max_clusters);
        EF_TM_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t tm_launch_f32(int N, int v, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    switch (N) {
#define EF_CASE(n)                                                                                       \
    case n:                                                                                              \
        return v == 5 ? launch_kernel(tm_kernel<n, 5>(), a, grid_clusters, tpb, smem, s)                 \
                      : launch_kernel(tm_kernel<n, 6>(), a, grid_clusters, tpb, smem, s);
        EF_TM_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ef
