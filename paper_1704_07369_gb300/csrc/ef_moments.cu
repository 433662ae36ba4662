// ef_moments.cu -- launcher of the FP64 moments / entropy reduction (ef_moments_entropy).
#include "ef_moments_impl.cuh"
#include "ef_launch.h"

namespace ef {

cudaError_t moments_launch(int prec, int d, const void *F, const void *Q, const int64_t *cell_off,
                           const int64_t *cell_N, int64_t ncells, int N_uniform, double twoL, double *out,
                           cudaStream_t s)
{
    if (ncells <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(ncells < 65535 * 16 ? ncells : 65535 * 16);
    if (prec == 0) {
        if (d == 3)
            moments_kernel<float, 3><<<grid, 256, 0, s>>>((const float *)F, (const float *)Q, cell_off, cell_N,
                                                          ncells, N_uniform, twoL, out);
        else
            moments_kernel<float, 2><<<grid, 256, 0, s>>>((const float *)F, (const float *)Q, cell_off, cell_N,
                                                          ncells, N_uniform, twoL, out);
    } else {
        if (d == 3)
            moments_kernel<double, 3><<<grid, 256, 0, s>>>((const double *)F, (const double *)Q, cell_off, cell_N,
                                                           ncells, N_uniform, twoL, out);
        else
            moments_kernel<double, 2><<<grid, 256, 0, s>>>((const double *)F, (const double *)Q, cell_off, cell_N,
                                                           ncells, N_uniform, twoL, out);
    }
    return cudaGetLastError();
}

}  // namespace ef
