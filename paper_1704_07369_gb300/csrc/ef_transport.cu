// ef_transport.cu -- free transport between spatial cells: the batch's cells are the points x_i of a
// periodic 1D spatial grid (spacing dx), and each velocity point moves along x with velocity
// component v along the first array axis (v = h (j - N/2), h = 2L/N).  One step of
//   dF/dt + v dF/dx = 0
// by first-order upwinding: with the Courant number nu = v dt / dx,
//   F_i <- F_i - nu (F_i - F_{i-1})   (nu > 0),     F_i <- F_i - nu (F_{i+1} - F_i)   (nu < 0),
// i.e. F_i <- (1 - |nu|) F_i + |nu| F_upwind: a convex combination when |nu| <= 1, so it keeps F >= 0.
// The paper leaves the spatially inhomogeneous problem to future work (Sec. 5); the collision step
// between transport steps is the plan's Euler or SSP-RK3 step (operator splitting).
//
// HBM-bound: each point is read once from its own cell and once from its upwind neighbour (an L2
// hit for the neighbour's recent reads in most cases) and written once.  Cells are along grid.y,
// 16-byte vectors of one cell along grid.x; a vector lies in one axis-0 plane (N is a multiple of 4),
// so it has one Courant number.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ef_launch.h"

namespace ef {
namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int W = 2;
};

__device__ __forceinline__ float4 upwind(float4 f, float4 g, float a)
{
    return make_float4(fmaf(-a, f.x - g.x, f.x), fmaf(-a, f.y - g.y, f.y), fmaf(-a, f.z - g.z, f.z),
                       fmaf(-a, f.w - g.w, f.w));
}

__device__ __forceinline__ double2 upwind(double2 f, double2 g, double a)
{
    return make_double2(fma(-a, f.x - g.x, f.x), fma(-a, f.y - g.y, f.y));
}

template <typename T>
__global__ void __launch_bounds__(256) transport_kernel(const T *__restrict__ Fin, T *__restrict__ Fout, int64_t ncells,
                                                        int N, int plane, int nv, T c)
{
    using V = typename Vec16<T>::type;
    constexpr int W = Vec16<T>::W;
    const V *in = reinterpret_cast<const V *>(Fin);
    V *out = reinterpret_cast<V *>(Fout);
    for (int64_t i = blockIdx.y; i < ncells; i += gridDim.y) {
        const int64_t im = i == 0 ? ncells - 1 : i - 1;
        const int64_t ip = i + 1 == ncells ? 0 : i + 1;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
            const int z = (v * W) / plane;                      // axis-0 index of the vector
            const T nu = c * T(z - N / 2);                      // Courant number of the plane
            const V f = in[i * nv + v];
            const V g = in[(nu > T(0) ? im : ip) * nv + v];      // upwind neighbour
            out[i * nv + v] = upwind(f, g, nu > T(0) ? nu : -nu);
        }
    }
}

}  // namespace

cudaError_t transport_launch(int prec, int d, int N, const void *Fin, void *Fout, int64_t ncells, double c,
                             cudaStream_t s)
{
    if (ncells <= 0) return cudaSuccess;
    const int64_t cell = d == 3 ? (int64_t)N * N * N : (int64_t)N * N;
    const int plane = d == 3 ? N * N : N;
    const int W = prec == 0 ? 4 : 2;
    if (cell % W || plane % W) return cudaErrorInvalidValue;
    const int nv = (int)(cell / W);
    const int threads = 256;
    const unsigned gx = (unsigned)std::min<int64_t>((nv + threads - 1) / threads, 1024);
    const unsigned gy = (unsigned)std::min<int64_t>(ncells, 65535);
    const dim3 grid(gx, gy);
    if (prec == 0)
        transport_kernel<float><<<grid, threads, 0, s>>>(static_cast<const float *>(Fin), static_cast<float *>(Fout),
                                                         ncells, N, plane, nv, (float)c);
    else
        transport_kernel<double><<<grid, threads, 0, s>>>(static_cast<const double *>(Fin), static_cast<double *>(Fout),
                                                          ncells, N, plane, nv, c);
    return cudaGetLastError();
}

}  // namespace ef
