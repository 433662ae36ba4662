// FP32 3D register-accumulator collide kernels: instantiations and their launch entry points
// (variants 1 - 4: collide_kernel_rg, one thread per line; 5, 6: collide_kernel_tm, two lanes per
// line, one or two rows per team, compiled in ef_collide_tm_f32.cu).
#include "ef_cluster_launch.h"
#include "ef_collide_rg.cuh"
#include "ef_launch.h"

namespace ef {

namespace {

template <int N, int V>
constexpr auto rg_kernel()
{
    return collide_kernel_rg<3, N, rg_rpt<V>(), (rg_bound<N, V>() > 0 ? rg_bound<N, V>() : 32), V == 4>;
}

template <int N>
cudaError_t rg_setup_n(int v, size_t smem, int cluster, int tpb, int *max_clusters)
{
    if (v == 5 || v == 6) return tm_setup_f32(N, v, smem, cluster, tpb, max_clusters);
    if (v == 1) return setup_kernel(rg_kernel<N, 1>(), smem, cluster, tpb, max_clusters);
    if (v == 2) return setup_kernel(rg_kernel<N, 2>(), smem, cluster, tpb, max_clusters);
    if constexpr (rg_bound<N, 3>() > 0) {
        if (v == 3) return setup_kernel(rg_kernel<N, 3>(), smem, cluster, tpb, max_clusters);
    }
    if (v == 4) return setup_kernel(rg_kernel<N, 4>(), smem, cluster, tpb, max_clusters);
    return cudaErrorInvalidValue;
}

template <int N>
cudaError_t rg_launch_n(int v, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    if (v == 5 || v == 6) return tm_launch_f32(N, v, a, grid_clusters, tpb, smem, s);
    if (v == 1) return launch_kernel(rg_kernel<N, 1>(), a, grid_clusters, tpb, smem, s);
    if (v == 2) return launch_kernel(rg_kernel<N, 2>(), a, grid_clusters, tpb, smem, s);
    if constexpr (rg_bound<N, 3>() > 0) {
        if (v == 3) return launch_kernel(rg_kernel<N, 3>(), a, grid_clusters, tpb, smem, s);
    }
    if (v == 4) return launch_kernel(rg_kernel<N, 4>(), a, grid_clusters, tpb, smem, s);
    return cudaErrorInvalidValue;
}

}  // namespace

#define EF_RG_SIZES(X) X(16) X(24) X(32) X(40) X(48) X(64)

int rg_maxthreads_f32(int N, int v)
{
    if (v < 1 || v > 6) return 0;
    switch (N) {
#define EF_CASE(n)                                                                                  \
    case n:                                                                                         \
        return v == 1 ? rg_bound<n, 1>() : v == 2 ? rg_bound<n, 2>() : v == 3 ? rg_bound<n, 3>() \
             : v == 4 ? rg_bound<n, 4>() : tm_maxthreads_f32(n);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return 0;
    }
}

int rg_rows_per_thread(int v) { return (v == 2 || v == 6) ? 2 : v == 4 ? 0 : 1; }

int rg_team(int v) { return v >= 5 ? 2 : 1; }

size_t rg_smem_f32(int N, int planes, int v)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_smem_bytes<n>(planes, rg_npc(n, n / planes), v == 4);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return 0;
    }
}

cudaError_t rg_setup_f32(int N, int v, size_t smem, int cluster, int tpb, int *max_clusters)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_setup_n<n>(v, smem, cluster, tpb, max_clusters);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rg_launch_f32(int N, int v, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_launch_n<n>(v, a, grid_clusters, tpb, smem, s);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ef
