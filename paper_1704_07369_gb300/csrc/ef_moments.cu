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
    const bool q = Q != nullptr;
#define EF_MOM(T, D)                                                                                     \
    do {                                                                                                 \
        if (q) moments_kernel<T, D, true><<<grid, 256, 0, s>>>((const T *)F, (const T *)Q, cell_off, cell_N, \
                                                               ncells, N_uniform, twoL, out);            \
        else moments_kernel<T, D, false><<<grid, 256, 0, s>>>((const T *)F, nullptr, cell_off, cell_N,   \
                                                              ncells, N_uniform, twoL, out);             \
    } while (0)
    if (prec == 0) {
        if (d == 3) EF_MOM(float, 3);
        else EF_MOM(float, 2);
    } else {
        if (d == 3) EF_MOM(double, 3);
        else EF_MOM(double, 2);
    }
#undef EF_MOM
    return cudaGetLastError();
}

}  // namespace ef
