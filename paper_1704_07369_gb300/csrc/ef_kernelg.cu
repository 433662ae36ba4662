// ef_kernelg.cu -- the kernel function G^sigma of the plan's discretisation on the GPU.
//
// The DVM form of the method (eq. A_simplified, eq. tildeG) weights the pair (p, q) -> (r, s) by
// G^sigma(y, z) = sum_{i,j in K} B^sigma(i, j) E_i(y) E_j(z).  With the plan's low-rank kernel
// (eq. fastAlg) B^sigma(i, j) = sum_e M_e(i) Gamma_e(j), where M_e are the filtered radial factors of
// the first directions and Gamma_e the weighted sums of their partners (the plan's multiplier tables),
//     G^sigma(y, z) = sum_e m_e(y) g_e(z),  m_e(y) = sum_i M_e(i) E_i(y),  g_e(z) = sum_j Gamma_e(j) E_j(z).
// The tables are real and even in the mode (M(-i) = M(i)), so only the cosine part survives.
// Sec. 3.2.2 shows G^sigma >= 0 for the filtered kernel; without the filter G takes negative values
// (Fig. 1).  This evaluates G by direct sums in FP64 (a diagnostic of the kernel decomposition, not
// part of the collision step): N^d outputs, each a sum over n_e directions and N^d modes.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "ef.h"
#include "ef_launch.h"

namespace {

constexpr double kPiG = 3.14159265358979323846264338327950288;

// value of table row `dir` at mode index (k0, k1, k2) in FFT order (2D: k0 = 0 plane, N1 = 1),
// through the half-spectrum layout [dir][l0][p], p = l1 * H + l2 (3D) or p = l2 (2D), using the
// evenness M(-k) = M(k) for the modes whose last component lies in the other half
template <typename T>
__device__ double table_at(const T *mult, int dir, int d, int N, int k0, int k1, int k2)
{
    const int H = N / 2 + 1, N1 = d == 3 ? N : 1;
    const int64_t per = (int64_t)N * N1 * H;
    if (k2 > N / 2) {                         // mode k2 - N < 0: use -k
        k0 = (N - k0) % N;
        k1 = (N - k1) % N;
        k2 = N - k2;
    }
    const int l0 = d == 3 ? k0 : k1, l1 = d == 3 ? k1 : 0;
    return (double)mult[(int64_t)dir * per + (int64_t)l0 * N1 * H + (int64_t)l1 * H + k2];
}

// cos(2 pi m / N) for the integer phase m (table in shared memory)
template <typename T>
__global__ void kernel_g_kernel(const T *mult, int ne, int d, int N, int64_t zidx, double *G)
{
    extern __shared__ double shg[];
    double *cs = shg;                 // [N] cos(2 pi m / N)
    double *ge = shg + N;             // [ne] g_e(z)
    double *mz = shg + N + ne;        // [ne] m_e(z)
    const int M1 = N, Md = d == 3 ? N * N * N : N * N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) cs[m] = cospi(2.0 * m / N);
    // grid index of z: components j (0 .. N-1 stand for j - N/2)
    int zj[3] = {0, 0, 0};
    {
        int64_t s = zidx;
        for (int a = d - 1; a >= 0; --a) { zj[a] = (int)(s % N) - N / 2; s /= N; }
    }
    __syncthreads();
    // g_e(z) for every direction e: one warp per e, FP64 sum over the modes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < ne; e += nw) {
        double acc = 0.0, accm = 0.0;
        for (int i = lane; i < Md; i += 32) {
            const int k2 = i % M1, k1 = (i / M1) % M1, k0 = d == 3 ? i / (M1 * M1) : 0;
            const int m0 = k0 < N / 2 ? k0 : k0 - N, m1 = k1 < N / 2 ? k1 : k1 - N, m2 = k2 < N / 2 ? k2 : k2 - N;
            const int ph = d == 3 ? m0 * zj[0] + m1 * zj[1] + m2 * zj[2] : m1 * zj[0] + m2 * zj[1];
            const double c = cs[((ph % N) + N) % N];
            acc += table_at<T>(mult, ne + e, d, N, k0, k1, k2) * c;
            accm += table_at<T>(mult, e, d, N, k0, k1, k2) * c;
        }
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            accm += __shfl_xor_sync(0xffffffffu, accm, o);
        }
        if (lane == 0) {
            ge[e] = acc;
            mz[e] = accm;
        }
    }
    __syncthreads();
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < Md; y += (int64_t)gridDim.x * blockDim.x) {
        int yj[3] = {0, 0, 0};
        int64_t s = y;
        for (int a = d - 1; a >= 0; --a) { yj[a] = (int)(s % N) - N / 2; s /= N; }
        double g = 0.0;
        for (int e = 0; e < ne; ++e) {
            double me = 0.0, gy = 0.0;
            for (int i = 0; i < Md; ++i) {
                const int k2 = i % M1, k1 = (i / M1) % M1, k0 = d == 3 ? i / (M1 * M1) : 0;
                const int m0 = k0 < N / 2 ? k0 : k0 - N, m1 = k1 < N / 2 ? k1 : k1 - N, m2 = k2 < N / 2 ? k2 : k2 - N;
                const int ph = d == 3 ? m0 * yj[0] + m1 * yj[1] + m2 * yj[2] : m1 * yj[0] + m2 * yj[1];
                const double c = cs[((ph % N) + N) % N];
                me += table_at<T>(mult, e, d, N, k0, k1, k2) * c;
                gy += table_at<T>(mult, ne + e, d, N, k0, k1, k2) * c;
            }
            g += 0.5 * (me * ge[e] + gy * mz[e]);
        }
        G[y] = g;
    }
}

}  // namespace

extern "C" ef_status ef_kernel_G(ef_plan_t plan, int64_t z_index, double *G_dev, ef_stream_t stream)
{
    ef::PlanView v;
    if (!ef::plan_view(plan, &v)) {
        ef::set_last_error("ef_kernel_G: needs a plan from ef_plan_create / ef_plan_create_ex");
        return EF_ERR_INVALID_ARG;
    }
    const int64_t Md = v.d == 3 ? (int64_t)v.N * v.N * v.N : (int64_t)v.N * v.N;
    if (!G_dev || z_index < 0 || z_index >= Md) {
        ef::set_last_error("ef_kernel_G: null G or z_index outside the grid");
        return EF_ERR_INVALID_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != v.device) {
        ef::set_last_error("ef_kernel_G: the plan's device is not current");
        return EF_ERR_INVALID_ARG;
    }
    const int ne = (v.ndir - 1) / 2;
    const int threads = 256;
    const int blocks = (int)((Md + threads - 1) / threads);
    const size_t smem = (size_t)(v.N + 2 * ne) * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    if (v.prec == EF_PREC_F32)
        kernel_g_kernel<float><<<blocks, threads, smem, s>>>(static_cast<const float *>(v.mult), ne, v.d, v.N, z_index, G_dev);
    else
        kernel_g_kernel<double><<<blocks, threads, smem, s>>>(static_cast<const double *>(v.mult), ne, v.d, v.N, z_index, G_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "ef_kernel_G launch: %s", cudaGetErrorString(e));
        ef::set_last_error(buf);
        return EF_ERR_CUDA;
    }
    return EF_OK;
}
