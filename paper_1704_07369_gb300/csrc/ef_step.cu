// ef_step.cu -- elementwise stage combination of the SSP-RK3 step (ef_rk3_step):
// out = a x + b y over a whole batch (cells back to back), 16-byte vector accesses where the
// pointers and the count allow; out may alias x or y.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ef_launch.h"

namespace {

template <typename T, typename V, int W>
__global__ void axpby_kernel(T *out, const T *x, const T *y, T a, T b, int64_t nvec)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x) {
        const V xv = reinterpret_cast<const V *>(x)[i], yv = reinterpret_cast<const V *>(y)[i];
        V o;
        const T *xs = reinterpret_cast<const T *>(&xv), *ys = reinterpret_cast<const T *>(&yv);
        T *os = reinterpret_cast<T *>(&o);
#pragma unroll
        for (int k = 0; k < W; ++k) os[k] = a * xs[k] + b * ys[k];
        reinterpret_cast<V *>(out)[i] = o;
    }
}

template <typename T, typename V, int W>
cudaError_t launch(void *out, const void *x, const void *y, double a, double b, int64_t n, cudaStream_t s)
{
    const int64_t nvec = n / W;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nvec + 255) / 256, (int64_t)sms * 8));
    if (nvec > 0)
        axpby_kernel<T, V, W><<<grid, 256, 0, s>>>((T *)out, (const T *)x, (const T *)y, (T)a, (T)b, nvec);
    if (n % W) {   // tail (never taken for whole cells: N^d is a multiple of 4)
        const int64_t off = nvec * W;
        axpby_kernel<T, T, 1><<<1, 32, 0, s>>>((T *)out + off, (const T *)x + off, (const T *)y + off, (T)a, (T)b, n - off);
    }
    return cudaGetLastError();
}

}  // namespace

namespace ef {

cudaError_t axpby_launch(int prec, void *out, const void *x, const void *y, double a, double b, int64_t n, cudaStream_t s)
{
    const bool aligned = ((uintptr_t)out | (uintptr_t)x | (uintptr_t)y) % 16 == 0;
    if (prec == 0)
        return aligned ? launch<float, float4, 4>(out, x, y, a, b, n, s) : launch<float, float, 1>(out, x, y, a, b, n, s);
    return aligned ? launch<double, double2, 2>(out, x, y, a, b, n, s) : launch<double, double, 1>(out, x, y, a, b, n, s);
}

}  // namespace ef
