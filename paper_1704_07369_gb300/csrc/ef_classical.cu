// ef_classical.cu -- the entropic Fourier method on the classical form of the collision operator
// (the remark after eq. EFMk), 3D Maxwell molecules (B = 1/(4 pi)), on the GPU in FP64:
//   Qh_k = sum_{l + m = k mod N} (Bs(l, m) - Bs(m, m)) Fh_l Fh_m,   Bs(l, m) = s(l) s(m) B_hat(l, m),
// with s the modified Jackson filter of each axis (eq. JacksonFilter2) and B_hat from
// eq. classical_hatB.  Writing g = r sigma, E_l((g + |g| w)/2) E_m((g - |g| w)/2) splits into
// exp(i c (l+m).g) exp(i c |g| (l-m).w), c = pi / (2T); both sphere integrals are 4 pi sinc, so
//   B_hat(l, m) = 4 pi int_0^R r^2 sinc(c r |l+m|) sinc(c r |l-m|) dr,
// and the radial integral has a closed form (below).  B_hat depends on (l, m) only through the
// integers |l+m|^2 and |l-m|^2 (at most 3 N^2), so it is tabulated over those when the object is
// created (on the device: (3 N^2 + 1)^2 FP64 values, 75 MB at N = 32, 1.2 GB at N = 64, 19 GB at
// N = 128; for one output mode the pairs touch at most 2^3 rows, |l + m| taking at most two
// values per axis, so the lookups stay in L2).  The weight needs the true l + m, not its alias mod N, which is why this path sums mode
// pairs directly (O(N^6) a cell, for the grid sizes of Table 3) instead of the low-rank transforms
// of the Carleman path.
//
// Per cell: F -> Fh by three separable DFT passes (index-origin convention, scaled by N^-3), the pair
// sum (one thread per output mode k, FP64), then three inverse passes and the real part.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "ef.h"
#include "ef_launch.h"

struct ef_classical_s {
    int N = 0;
    double T = 0.0, R = 0.0;
    int device = 0;
    int64_t nn = 0;             // table side: 3 N^2 + 1
    double *d_tab = nullptr;    // [nn][nn]: 4 pi I(c sqrt(s2), c sqrt(d2))
    double *d_sig = nullptr;    // [N^3] filter of each mode
    double *d_bmm = nullptr;    // [N^3] Bs(m, m)
    double2 *d_x = nullptr, *d_y = nullptr;   // [N^3] transform work arrays
};

namespace {

constexpr double kPiC = 3.14159265358979323846264338327950288;

// sin(x R) / x, its limit R at x = 0
__host__ __device__ double sin_over(double x, double R)
{
    const double y = x * R;
    return fabs(y) < 1e-6 ? R * (1.0 - y * y / 6.0) : sin(y) / x;
}

// I(a, b) = int_0^R r^2 sinc(a r) sinc(b r) dr for a, b >= 0, sinc(x) = sin(x) / x:
//   a, b > 0:  (1 / (2ab)) [S(a - b) - S(a + b)],  S(x) = sin(xR) / x  (cos(a-b)r - cos(a+b)r = 2 sin ar sin br)
//   a = 0:     (sin(bR) - bR cos(bR)) / b^3  (series near bR = 0),   a = b = 0:  R^3 / 3
__host__ __device__ double radial_integral(double a, double b, double R)
{
    if (a < b) {
        const double t = a;
        a = b;
        b = t;
    }
    if (a == 0.0) return R * R * R / 3.0;
    if (b == 0.0) {
        const double y = a * R;
        if (y < 1e-2) return R * R * R * (1.0 / 3.0 - y * y / 30.0 + y * y * y * y / 840.0);
        return (sin(y) - y * cos(y)) / (a * a * a);
    }
    return (sin_over(a - b, R) - sin_over(a + b, R)) / (2.0 * a * b);
}

// tab[i][j] = 4 pi I(c sqrt(i), c sqrt(j)) over the integers i, j <= 3 N^2 (built on the device:
// (3 N^2 + 1)^2 entries, 1.2 GB at N = 64)
__global__ void classical_table_kernel(double *tab, int64_t nn, double cc, double R)
{
    const double fourpi = 4.0 * 3.14159265358979323846264338327950288;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn * nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nn, j = t % nn;
        tab[t] = fourpi * radial_integral(cc * sqrt((double)i), cc * sqrt((double)j), R);
    }
}

int mode_at(int N, int i) { return i < N / 2 ? i : i - N; }

ef_status cfail(ef_status s, const std::string &m)
{
    ef::set_last_error(m.c_str());
    return s;
}

ef_status ccuda(cudaError_t e, const char *what)
{
    const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    ef::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

void cfree(ef_classical_s *c)
{
    if (!c) return;
    cudaFree(c->d_tab);
    cudaFree(c->d_sig);
    cudaFree(c->d_bmm);
    cudaFree(c->d_x);
    cudaFree(c->d_y);
    delete c;
}

__global__ void to_complex_kernel(const double *F, double2 *X, int64_t M)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        X[i] = make_double2(F[i], 0.0);
}

__global__ void real_part_kernel(const double2 *X, double *Q, int64_t M)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        Q[i] = X[i].x;
}

// One separable DFT pass along the axis of the given stride: out[..c..] = scale sum_j in[..j..]
// exp(sign 2 pi i c j / N).
__global__ void dft_pass_kernel(const double2 *in, double2 *out, int N, int stride, int sign, double scale, int64_t M)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < M; idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)((idx / stride) % N);
        const int64_t base = idx - (int64_t)c * stride;
        double re = 0.0, im = 0.0;
        int t = 0;                                   // c j mod N
        for (int j = 0; j < N; ++j) {
            double s, co;
            sincospi(2.0 * t / N, &s, &co);
            s *= sign;
            const double2 v = in[base + (int64_t)j * stride];
            re += v.x * co - v.y * s;
            im += v.x * s + v.y * co;
            t += c;
            if (t >= N) t -= N;
        }
        out[idx] = make_double2(scale * re, scale * im);
    }
}

// Qh_k = sum_l (s_l s_m tab[|l+m|^2][|l-m|^2] - bmm_m) Fh_l Fh_m, m = k - l mod N per axis.
__global__ void __launch_bounds__(256) pair_sum_kernel(const double2 *Fh, double2 *Qh, const double *tab,
                                                       const double *sig, const double *bmm, int N, int64_t nn)
{
    const int M = N * N * N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const int k0 = k / (N * N), k1 = (k / N) % N, k2 = k % N;
    const int h = N / 2;
    double re = 0.0, im = 0.0;
    for (int l0 = 0; l0 < N; ++l0) {
        const int m0 = k0 - l0 < 0 ? k0 - l0 + N : k0 - l0;
        const int a0 = l0 < h ? l0 : l0 - N, b0 = m0 < h ? m0 : m0 - N;
        for (int l1 = 0; l1 < N; ++l1) {
            const int m1 = k1 - l1 < 0 ? k1 - l1 + N : k1 - l1;
            const int a1 = l1 < h ? l1 : l1 - N, b1 = m1 < h ? m1 : m1 - N;
            const int s01 = (a0 + b0) * (a0 + b0) + (a1 + b1) * (a1 + b1);
            const int d01 = (a0 - b0) * (a0 - b0) + (a1 - b1) * (a1 - b1);
            const int lrow = (l0 * N + l1) * N, mrow = (m0 * N + m1) * N;
            for (int l2 = 0; l2 < N; ++l2) {
                const int m2 = k2 - l2 < 0 ? k2 - l2 + N : k2 - l2;
                const int a2 = l2 < h ? l2 : l2 - N, b2 = m2 < h ? m2 : m2 - N;
                const int l = lrow + l2, m = mrow + m2;
                const double sl = sig[l], bm = bmm[m];
                if (sl == 0.0 && bm == 0.0) continue;
                const int64_t s2 = s01 + (a2 + b2) * (a2 + b2), d2 = d01 + (a2 - b2) * (a2 - b2);
                const double b = sl * sig[m] * tab[s2 * nn + d2] - bm;
                const double2 fl = Fh[l], fm = Fh[m];
                re += b * (fl.x * fm.x - fl.y * fm.y);
                im += b * (fl.x * fm.y + fl.y * fm.x);
            }
        }
    }
    Qh[k] = make_double2(re, im);
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

extern "C" {

ef_status ef_classical_create(int N, double L, double R_tr, int sigma_enabled, ef_classical_t *out)
{
    if (!out) return cfail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (N < 4 || N % 2 || N > 128) return cfail(EF_ERR_INVALID_ARG, "classical form: N must be even, 4 <= N <= 128");
    if (!(L > 0.0) || !std::isfinite(L)) return cfail(EF_ERR_INVALID_ARG, "L must be > 0");
    const double R = R_tr > 0.0 ? R_tr : 4.0 * L / (3.0 + std::sqrt(2.0));
    if (!std::isfinite(R)) return cfail(EF_ERR_INVALID_ARG, "R_tr must be finite");
    ef_classical_s *c = new (std::nothrow) ef_classical_s();
    if (!c) return cfail(EF_ERR_OOM, "host allocation");
    c->N = N;
    c->T = L;
    c->R = R;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { cfree(c); return ccuda(e, "cudaGetDevice"); }
    const int64_t M = (int64_t)N * N * N;
    c->nn = 3 * (int64_t)N * N + 1;
    const int64_t nn = c->nn;
    const double cc = kPiC / (2.0 * L);
    std::vector<double> s1(N);
    for (int i = 0; i < N; ++i) s1[i] = ef::jackson_filter(N, mode_at(N, i), sigma_enabled != 0);
    std::vector<double> sig((size_t)M), bmm((size_t)M);
    for (int64_t m = 0; m < M; ++m) {
        const int i0 = (int)(m / (N * N)), i1 = (int)((m / N) % N), i2 = (int)(m % N);
        const int a0 = mode_at(N, i0), a1 = mode_at(N, i1), a2 = mode_at(N, i2);
        sig[(size_t)m] = s1[i0] * s1[i1] * s1[i2];
        const int64_t m2 = 4 * ((int64_t)a0 * a0 + (int64_t)a1 * a1 + (int64_t)a2 * a2);
        // B_hat(m, m): |m + m|^2 = 4 |m|^2, |m - m|^2 = 0 (the table's row 4|m|^2, column 0)
        bmm[(size_t)m] = sig[(size_t)m] * sig[(size_t)m] * 4.0 * kPiC * radial_integral(cc * std::sqrt((double)m2), 0.0, R);
    }
    e = cudaMalloc((void **)&c->d_tab, (size_t)(nn * nn) * sizeof(double));
    if (e == cudaSuccess) {
        classical_table_kernel<<<152 * 16, 256>>>(c->d_tab, nn, cc, R);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_sig, (size_t)M * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_bmm, (size_t)M * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_x, (size_t)M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_y, (size_t)M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_sig, sig.data(), sig.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_bmm, bmm.data(), bmm.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cfree(c); return ccuda(e, "classical-form tables"); }
    *out = c;
    return EF_OK;
}

ef_status ef_classical_destroy(ef_classical_t c)
{
    if (!c) return cfail(EF_ERR_INVALID_ARG, "null classical-form object");
    int cur = -1;
    const bool had = cudaGetDevice(&cur) == cudaSuccess;
    const int dev = c->device;
    cudaSetDevice(dev);                 // free on the object's device, then restore the caller's
    cudaDeviceSynchronize();
    cfree(c);
    if (had && cur != dev) cudaSetDevice(cur);
    return EF_OK;
}

ef_status ef_classical_collide(ef_classical_t c, const double *F_dev, double *Q_dev, int64_t ncells, ef_stream_t stream)
{
    if (!c) return cfail(EF_ERR_INVALID_ARG, "null classical-form object");
    if (ncells < 0) return cfail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (ncells == 0) return EF_OK;
    if (!F_dev || !Q_dev) return cfail(EF_ERR_INVALID_ARG, "null F or Q");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != c->device) return cfail(EF_ERR_INVALID_ARG, "the object's device is not current");
    const int N = c->N;
    const int64_t M = (int64_t)N * N * N;
    const uintptr_t bytes = (uintptr_t)(ncells * M * (int64_t)sizeof(double));
    const uintptr_t a = (uintptr_t)F_dev, b = (uintptr_t)Q_dev;
    if (a < b + bytes && b < a + bytes) return cfail(EF_ERR_INVALID_ARG, "Q must not overlap F");
    cudaStream_t s = (cudaStream_t)stream;
    const int strides[3] = {N * N, N, 1};
    const double scale = 1.0 / (double)M;
    for (int64_t cell = 0; cell < ncells; ++cell) {
        const double *F = F_dev + cell * M;
        double *Q = Q_dev + cell * M;
        to_complex_kernel<<<grid_for(M), 256, 0, s>>>(F, c->d_x, M);
        double2 *x = c->d_x, *y = c->d_y;
        for (int ax = 0; ax < 3; ++ax) {
            dft_pass_kernel<<<grid_for(M), 256, 0, s>>>(x, y, N, strides[ax], -1, ax == 0 ? scale : 1.0, M);
            std::swap(x, y);
        }
        pair_sum_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(x, y, c->d_tab, c->d_sig, c->d_bmm, N, c->nn);
        std::swap(x, y);
        for (int ax = 0; ax < 3; ++ax) {
            dft_pass_kernel<<<grid_for(M), 256, 0, s>>>(x, y, N, strides[ax], +1, 1.0, M);
            std::swap(x, y);
        }
        real_part_kernel<<<grid_for(M), 256, 0, s>>>(x, Q, M);
        e = cudaGetLastError();
        if (e != cudaSuccess) return ccuda(e, "classical-form launch");
    }
    return EF_OK;
}

}  // extern "C"
