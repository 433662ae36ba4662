// FP32 3D register-accumulator collide kernel: instantiations and their launch entry points.
#include "ef_cluster_launch.h"
#include "ef_collide_rg.cuh"
#include "ef_launch.h"

namespace ef {

namespace {

template <int N>
cudaError_t rg_setup_n(int rpt, size_t smem, int cluster, int tpb, int *max_clusters)
{
    if (rpt == 1) return setup_kernel(collide_kernel_rg<3, N, 1>, smem, cluster, tpb, max_clusters);
    if (rpt == 2) return setup_kernel(collide_kernel_rg<3, N, 2>, smem, cluster, tpb, max_clusters);
    return cudaErrorInvalidValue;
}

template <int N>
cudaError_t rg_launch_n(int rpt, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    if (rpt == 1) return launch_kernel(collide_kernel_rg<3, N, 1>, a, grid_clusters, tpb, smem, s);
    if (rpt == 2) return launch_kernel(collide_kernel_rg<3, N, 2>, a, grid_clusters, tpb, smem, s);
    return cudaErrorInvalidValue;
}

}  // namespace

#define EF_RG_SIZES(X) X(16) X(24) X(32) X(40) X(48) X(64)

int rg_maxthreads_f32(int N, int rpt)
{
    if (rpt != 1 && rpt != 2) return 0;
    switch (N) {
#define EF_CASE(n) case n: return rpt == 1 ? rg_max_threads<n, 1>() : rg_max_threads<n, 2>();
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return 0;
    }
}

size_t rg_smem_f32(int N, int planes)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_smem_bytes<n>(planes, rg_npc(n, n / planes));
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return 0;
    }
}

cudaError_t rg_setup_f32(int N, int rpt, size_t smem, int cluster, int tpb, int *max_clusters)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_setup_n<n>(rpt, smem, cluster, tpb, max_clusters);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rg_launch_f32(int N, int rpt, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    switch (N) {
#define EF_CASE(n) case n: return rg_launch_n<n>(rpt, a, grid_clusters, tpb, smem, s);
        EF_RG_SIZES(EF_CASE)
#undef EF_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ef
