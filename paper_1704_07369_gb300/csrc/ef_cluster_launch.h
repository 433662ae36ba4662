// ef_cluster_launch.h -- occupancy query and launch of a collide kernel as thread-block clusters
// (one cluster of `cluster` CTAs per cell), shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "ef_internal.h"

namespace ef {
namespace {

template <typename K>
cudaError_t setup_kernel(K k, size_t smem, int cluster, int tpb, int *max_clusters)
{
    // allow the device's opt-in maximum so plans with different shapes can share the kernel
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (tpb > fa.maxThreadsPerBlock) return cudaErrorInvalidValue;
    const int dyn_max = smem_max - (int)fa.sharedSizeBytes;
    if ((long)smem > (long)dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(tpb, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, k, &cfg);
}

template <typename K>
cudaError_t launch_kernel(K k, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid_clusters * a.cluster), 1, 1);
    cfg.blockDim = dim3(tpb, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace
}  // namespace ef
