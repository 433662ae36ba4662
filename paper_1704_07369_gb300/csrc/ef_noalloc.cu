// ef_noalloc.cu -- ef_collide_noalloc: the collision operator for callers that cannot allocate
// device memory when they run it.
//
// Some callers cannot call cudaMalloc at the point where they evaluate the operator: code that
// runs inside a memory-budgeted host framework whose allocator owns all device memory, code that
// is enqueued from callbacks or real-time loops where an allocation may block or fail, or code
// that must not change the device's memory footprint after start-up.  ef_collide keeps its
// scratch (the forward-spectrum slots and, for shapes whose S/G accumulators live in global
// memory, that workspace) in buffers the plan allocates when it is created.  This entry point
// instead takes all scratch from one file-scope static device array of fixed size, which every
// GPU that loads the library holds until the process exits.  It always keeps the S/G accumulators
// in that array (global memory), whatever shape the plan's autotuner chose, with the plan's
// cluster size, threads per CTA, occupancy variant and L1-prefetch choice; on shapes whose
// accumulators ef_collide keeps in shared memory it can therefore be slower than ef_collide.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "ef.h"
#include "ef_launch.h"

namespace {

// 16 MiB per device: the cell-queue counter (first 256 bytes) and the S/G accumulators of the
// clusters in flight (the launch uses only as many clusters as fit).
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr size_t kCounterBytes = 256;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (the host-side symbol is only a stand-in).
// Looked up once per device, with that device current.
ef_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        ef::set_last_error("ef_collide_noalloc: device index out of range");
        return EF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            char buf[160];
            std::snprintf(buf, sizeof(buf), "ef_collide_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            ef::set_last_error(buf);
            return EF_ERR_CUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return EF_OK;
}

}  // namespace

extern "C" ef_status ef_collide_noalloc(ef_plan_t plan, const void *F_dev, void *Q_dev, int64_t ncells,
                                        ef_stream_t stream)
{
    ef::PlanView v;
    if (!ef::plan_view(plan, &v)) {
        ef::set_last_error("ef_collide_noalloc: needs a plan from ef_plan_create / ef_plan_create_ex");
        return EF_ERR_INVALID_ARG;
    }
    if (ncells < 0) {
        ef::set_last_error("ef_collide_noalloc: ncells < 0");
        return EF_ERR_INVALID_ARG;
    }
    if (ncells == 0) return EF_OK;
    if (!F_dev || !Q_dev || F_dev == Q_dev || (((uintptr_t)F_dev | (uintptr_t)Q_dev) % 16)) {
        ef::set_last_error("ef_collide_noalloc: null, equal or not 16-byte aligned F / Q");
        return EF_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != v.device) {
        ef::set_last_error("ef_collide_noalloc: the plan's device is not current");
        return EF_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    ef_status st = scratch_address(dev, &base);
    if (st != EF_OK) return st;

    // per cluster: S and G of each CTA in global memory (2 * rows * N values per CTA) and the
    // forward-spectrum workspace; layout [counter][S/G of grid * C CTAs][spectra of grid clusters].
    // The register-accumulator variants (occ >= 3) keep both on chip and need only the counter.
    const bool onchip = v.occ >= 3;
    const int64_t rows = (int64_t)v.planes * (v.d == 3 ? v.N : 1);
    const size_t el = v.prec == EF_PREC_F32 ? 4 : 8;
    const size_t per_cta = onchip ? 0 : ((size_t)2 * rows * v.N * el + 255) / 256 * 256;
    const size_t per_fh = onchip ? 0 : (ef::collide_fh_bytes(v.prec, v.d, v.N) + 255) / 256 * 256;
    const size_t per_cluster = per_cta * v.cluster + per_fh;
    const size_t avail = kScratchBytes - kCounterBytes;
    const int64_t clusters_fit = onchip ? (int64_t)v.max_clusters : (int64_t)(avail / per_cluster);
    if (clusters_fit < 1) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "ef_collide_noalloc: one cell cluster needs %zu bytes of scratch, more than the %zu available",
                      per_cluster, avail);
        ef::set_last_error(buf);
        return EF_ERR_UNSUPPORTED;
    }
    const int grid = (int)std::min<int64_t>(std::min<int64_t>(ncells, v.max_clusters), clusters_fit);
    const size_t smem = onchip ? v.smem : ef::collide_smem(v.prec, v.d, v.N, v.planes, 1, v.paired, v.occ);

    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(base, 0, sizeof(unsigned long long), s);      // the cell queue starts at 0
    if (e != cudaSuccess) {
        ef::set_last_error(cudaGetErrorString(e));
        return EF_ERR_CUDA;
    }
    ef::CollideArgs a{};
    a.F = F_dev;
    a.Q = Q_dev;
    a.ncells = ncells;
    a.mult = v.mult;
    a.ops = v.ops;
    a.nops = v.nops;
    a.cluster = v.cluster;
    a.planes = v.planes;
    a.sg_global = onchip ? 0 : 1;
    a.sg_ws = static_cast<unsigned char *>(base) + kCounterBytes;
    a.fh_ws = static_cast<unsigned char *>(base) + kCounterBytes + (size_t)grid * v.cluster * per_cta;
    a.npc = ef::collide_npc_v(v.d, v.N, v.cluster, v.occ);
    a.out_mode = ef::OUT_COLLIDE;
    a.h = 2.0 * v.L / v.N;
    a.status = v.status;
    a.counter = static_cast<unsigned long long *>(base);
    a.paired = v.paired;
    a.prefetch = v.prefetch;
    e = ef::collide_launch(v.prec, v.d, v.N, a, grid, v.tpb, smem, v.occ, s);
    if (e != cudaSuccess) {
        ef::set_last_error(cudaGetErrorString(e));
        return EF_ERR_CUDA;
    }
    return EF_OK;
}
