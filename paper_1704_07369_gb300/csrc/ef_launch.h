// ef_launch.h -- per-(precision, dimension) kernel entry points defined in the ef_collide_*.cu
// translation units, called by the host plan code.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "ef.h"
#include "ef_internal.h"

namespace ef {

#define EF_DECLARE_VARIANT(SUF)                                                                      \
    bool collide_supported_##SUF(int N);                                                             \
    int collide_maxthreads_##SUF(int N, int occ);                                                    \
    size_t collide_smem_##SUF(int N, int planes, int sg_global, int paired, int occ);                \
    cudaError_t collide_setup_##SUF(int N, size_t smem, int cluster, int tpb, int occ, int *max_clusters); \
    cudaError_t collide_launch_##SUF(int N, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, \
                                     int occ, cudaStream_t s);

// FP32 3D register-accumulator kernels (ef_collide_rg_f32.cu), instantiation v = 1 .. 6 (kernel
// variant occ = 2 + v; 5, 6: two lanes per line): rg_maxthreads_f32 is its launch bound (0: not
// built for N), rg_rows_per_thread its rows per thread or team (0: the gain accumulator in shared
// memory, rows looped).
int rg_maxthreads_f32(int N, int v);
int rg_rows_per_thread(int v);
// lanes per line transform of variant v (2: the team kernel, threads = 2 rows / RPT)
int rg_team(int v);
// the team kernel (ef_collide_tm_f32.cu, variants 5 and 6): launch bound (0: not built for N)
int tm_maxthreads_f32(int N);
cudaError_t tm_setup_f32(int N, int v, size_t smem, int cluster, int tpb, int *max_clusters);
cudaError_t tm_launch_f32(int N, int v, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s);
size_t rg_smem_f32(int N, int planes, int v);
cudaError_t rg_setup_f32(int N, int v, size_t smem, int cluster, int tpb, int *max_clusters);
cudaError_t rg_launch_f32(int N, int v, const CollideArgs &a, int grid_clusters, int tpb, size_t smem, cudaStream_t s);

EF_DECLARE_VARIANT(f32_2d)
EF_DECLARE_VARIANT(f32_3d)
EF_DECLARE_VARIANT(f64_2d)
EF_DECLARE_VARIANT(f64_3d)

#undef EF_DECLARE_VARIANT

// Read-only view of a uniform plan's single size class, for entry points defined outside
// ef_plan.cpp (ef_noalloc.cu).  Returns false for a null or batched plan.
struct PlanView {
    int prec, d, N;
    int cluster, tpb, planes, paired, nops, max_clusters, sg_global, nfeat;   // nfeat: band modes
    int occ;                  // kernel instantiation: 1 or 2 CTAs per SM
    int prefetch;             // 1: L1 prefetch of the next op's multipliers
    int ndir;                 // rows of the multiplier table: n_e directions, n_e partner sums, the loss
    size_t smem;
    double L;
    const void *mult;
    const Op *ops;
    const int *modes;         // device [nfeat][3] band modes (FeatArgs::modes)
    int *status;
    int device;
};
bool plan_view(const struct ef_plan_s *p, PlanView *out);
// uniform plan on the doubled grid 2N with multipliers restricted to the N grid's Galerkin modes
ef_status plan_create_padded(const ef_plan_desc *desc, struct ef_plan_s **out);

// Axis-0 pencils per CTA of a C-CTA cluster (even, so that lane pairs never straddle CTAs) and the
// bytes of one cluster's forward-spectrum workspace (N x NP complex).
inline int collide_npc(int d, int N, int C)
{
    const int NP = (d == 3 ? N : 1) * (N / 2 + 1);
    const int npc = (NP + C - 1) / C;
    return (npc + 1) / 2 * 2;
}
inline size_t collide_fh_bytes(int prec, int d, int N)
{
    return (size_t)N * (d == 3 ? N : 1) * (N / 2 + 1) * (prec == 0 ? 8 : 16);
}
size_t collide_smem(int prec, int d, int N, int planes, int sg_global, int paired, int occ);
// Kernel variants ("occ"): 1 = one CTA per SM, 2 = two CTAs per SM (shared-memory accumulators);
// 3 / 4 / 5 / 6 = FP32 3D kernel that keeps the forward spectrum in shared memory and skips the
// Nyquist column (pencils: N^2 / (2 C) per CTA), with the gain accumulator in registers (one row
// per thread / two / one with at most 200 threads) or (6) in shared memory.
inline int collide_npc_v(int d, int N, int C, int occ)
{
    if (occ >= 3) {
        const int np = N * N / 2;
        return (np % C == 0 && (np / C) % 2 == 0) ? np / C : 0;
    }
    return collide_npc(d, N, C);
}
cudaError_t collide_launch(int prec, int d, int N, const CollideArgs &a, int grid_clusters, int tpb, size_t smem,
                           int occ, cudaStream_t s);
void set_last_error(const char *msg);
// the modified Jackson filter of one axis (eq. JacksonFilter2; sigma(-N/2) = 0), as the plans use it
double jackson_filter(int N, int k, bool enabled);

// low-mode features (ef_features_f32.cu / ef_features_f64.cu): nf = 1 or 2 fields; the grid is
// capped at the CTAs that fit on the device at once (persistent over cells)
bool features_fits(int prec, int d, int N, int nf);
cudaError_t features_launch(int prec, int d, int N, const FeatArgs &a, cudaStream_t s);
#define EF_DECLARE_FEAT(SUF)                                                                          \
    bool features_fits_##SUF(int d, int N, int nf);                                                   \
    cudaError_t features_launch_##SUF(int d, int N, const FeatArgs &a, cudaStream_t s);
EF_DECLARE_FEAT(f32)
EF_DECLARE_FEAT(f64)
#undef EF_DECLARE_FEAT

// out = a x + b y over n values (ef_step.cu); prec 0 = FP32, 1 = FP64
// free transport between the spatial cells of a uniform batch (ef_transport.cu), c = dt h / dx
cudaError_t transport_launch(int prec, int d, int N, const void *Fin, void *Fout, int64_t ncells, double c,
                             cudaStream_t s);
cudaError_t axpby_launch(int prec, void *out, const void *x, const void *y, double a, double b, int64_t n,
                         cudaStream_t s);

// moments / entropy (ef_moments.cu)
cudaError_t moments_launch(int prec, int d, const void *F, const void *Q, const int64_t *cell_off,
                           const int64_t *cell_N, int64_t ncells, int N_uniform, double twoL, double *out,
                           cudaStream_t s);


}  // namespace ef
