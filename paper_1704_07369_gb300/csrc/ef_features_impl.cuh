// ef_features_impl.cuh -- low Fourier modes of a cell (the learned surrogate's input and output
// band) in one pass over the cell, optionally with the modes of ln F and the cell's moments.
//
// The band is |k| <= EF_FEATURE_K (K) in the canonical half space; with the library's
// index-origin convention
//   Fh_k = N^-d sum_i F[i] exp(-2 pi i k.i / N)      (i the array index, 0 .. N-1 per axis).
// One CTA per cell (persistent over cells).  For a chunk of PZ axis-0 planes at a time:
//   stage 1  every row along the contiguous axis is transformed (a real row through a half-length
//            complex FFT) and only kx = 0 .. K is kept in shared memory;
//   stage 2  every (plane, kx) column is transformed along axis 1 and ky = -K .. K kept;
// then, with all planes done,
//   stage 3  every band mode sums its N axis-0 values against exp(-2 pi i kz z / N) directly.
// 2D cells are one plane (stage 3 is the identity).  The moments fold each row's sums (in T) into
// FP64, like the fused diagnostics of the collide kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ef.h"
#include "ef_fft.cuh"
#include "ef_internal.h"

namespace ef {


constexpr int kFeatK = EF_FEATURE_K;
constexpr int kFeatKx = kFeatK + 1;          // kx = 0 .. K
constexpr int kFeatKy = 2 * kFeatK + 1;      // ky = -K .. K

// planes per chunk: the largest divisor of N not above the cap
template <int N, int CAP>
constexpr int feat_pz()
{
    int p = CAP < N ? CAP : N;
    while (N % p) --p;
    return p;
}

template <typename T, int D, int N>
struct FeatLayout {
    static constexpr int PZ = (D == 3) ? feat_pz<N, sizeof(T) == 4 ? 8 : 4>() : 1;
    static constexpr int NZ = (D == 3) ? N : 1;
    static constexpr int X1_PLANE = N * kFeatKx + 1;         // odd complex stride per plane
    static constexpr int X1_FIELD = PZ * X1_PLANE;
    static constexpr int X2_PLANE = kFeatKy * kFeatKx;
    static constexpr int X2_FIELD = NZ * X2_PLANE;
    static constexpr size_t bytes(int nf)
    {
        return (size_t)N * sizeof(C2<T>) + (size_t)nf * (X1_FIELD + X2_FIELD) * sizeof(C2<T>) +
               8 * EF_DIAG_STRIDE * sizeof(double);
    }
};

template <typename T>
__device__ __forceinline__ T feat_log(T x);
template <>
__device__ __forceinline__ float feat_log<float>(float x) { return logf(x > 1e-30f ? x : 1e-30f); }
template <>
__device__ __forceinline__ double feat_log<double>(double x) { return log(x > 1e-30 ? x : 1e-30); }

template <typename T, int N>
__device__ __forceinline__ void feat_load_row(const T *src, T (&x)[N])
{
    if constexpr (sizeof(T) == 4 && N % 4 == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = s4[i];
            x[4 * i] = v.x; x[4 * i + 1] = v.y; x[4 * i + 2] = v.z; x[4 * i + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
        const double2 *s2 = reinterpret_cast<const double2 *>(src);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 v = s2[i];
            x[2 * i] = v.x; x[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int n = 0; n < N; ++n) x[n] = src[n];
    }
}

// row sums of one row (T), folded into the FP64 accumulators; the entropy term only with eta
// (otherwise the ln F pass adds it, from the logarithms it computes anyway)
template <typename T, int D, int N>
__device__ __forceinline__ void feat_row_moments(const T (&x)[N], int jz, int jy, double (&s)[EF_DIAG_STRIDE], T &mn,
                                                 bool eta)
{
    T p0 = 0, px = 0, pe = 0, peta = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const T f = x[n];
        const T jx = T(n - N / 2);
        p0 += f;
        px += f * jx;
        pe += f * jx * jx;
        if (eta && f > T(0)) peta += f * feat_log<T>(f);
        mn = f < mn ? f : mn;
    }
    const double m = (double)p0;
    s[0] += m;
    if (D == 3) {
        s[1] += m * jz;
        s[2] += m * jy;
        s[3] += (double)px;
    } else {
        s[1] += m * jy;
        s[2] += (double)px;
    }
    s[4] += (double)pe + m * ((double)jy * jy + (double)jz * jz);
    s[5] += (double)peta;
}

// One real row -> its spectrum at k = 0 .. KX-1 (forward sign, unscaled) through a half-length
// complex transform of z_m = x_2m + i x_2m+1: X_k = E_k + exp(-2 pi i k / N) O_k with
// E_k = (Z_k + conj Z_{M-k}) / 2 and O_k = (Z_k - conj Z_{M-k}) / 2i, M = N / 2.
template <int N, int KX, typename T>
__device__ __forceinline__ void r2c_low(const T (&x)[N], C2<T> (&X)[KX], const C2<T> *tw)
{
    constexpr int M = N / 2;
    static_assert(KX <= M, "band wider than the half-length transform");
    C2<T> z[M];
#pragma unroll
    for (int m = 0; m < M; ++m) z[m] = C2<T>{x[2 * m], x[2 * m + 1]};
    fft<M, -1, N>(z, tw);
#pragma unroll
    for (int k = 0; k < KX; ++k) {
        const C2<T> a = z[k], b = cconj(z[(M - k) % M]);
        const C2<T> e = C2<T>{T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y)};
        const C2<T> o = C2<T>{T(0.5) * (a.y - b.y), T(-0.5) * (a.x - b.x)};
        X[k] = e + cmul(tw[k], o);
    }
}

// CTAs of 4 warps, several per SM (cells in flight overlap their barrier phases): 168 registers
// for N <= 32 (3 CTAs per SM), 255 above (2 per SM)
constexpr int kFeatThreads = 128;
template <int N>
constexpr int feat_min_blocks() { return N <= 32 ? 3 : 2; }

template <typename T, int D, int N>
__global__ void __launch_bounds__(kFeatThreads, feat_min_blocks<N>()) features_kernel(const FeatArgs a)
{
    using Lay = FeatLayout<T, D, N>;
    constexpr int PZ = Lay::PZ, NZ = Lay::NZ;
    constexpr int ROWS = PZ * N;                 // rows along the contiguous axis per chunk
    static_assert(N / 2 > kFeatK, "grid too small for the band");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nf = a.featL ? 2 : 1;
    C2<T> *tw = reinterpret_cast<C2<T> *>(smem_raw);
    C2<T> *X1 = tw + N;
    C2<T> *X2 = X1 + (size_t)nf * Lay::X1_FIELD;
    double *red = reinterpret_cast<double *>(X2 + (size_t)nf * Lay::X2_FIELD);   // [8 warps][EF_DIAG_STRIDE]
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < N; j += nt) {
        T sn, cs;
        if constexpr (sizeof(T) == 4) sincospif(T(2 * j) / T(N), &sn, &cs);
        else sincospi(T(2 * j) / T(N), &sn, &cs);
        tw[j] = C2<T>{cs, -sn};
    }
    __syncthreads();
    const T scale = T(1) / T(D == 3 ? N * N * N : N * N);
    const int64_t ncells = a.dev_ncells ? (int64_t)*a.dev_ncells : a.ncells;
    for (int64_t c = blockIdx.x; c < ncells; c += gridDim.x) {
        const int64_t coff = a.cell_off ? a.cell_off[c] : c * (int64_t)(D == 3 ? N * N * N : N * N);
        const int64_t row = a.cell_id ? a.cell_id[c] : c;
        const T *F = reinterpret_cast<const T *>(a.F) + coff;
        double s[EF_DIAG_STRIDE];
#pragma unroll
        for (int k = 0; k < EF_DIAG_STRIDE; ++k) s[k] = 0.0;
        T mn;
        if constexpr (sizeof(T) == 4) mn = T(3.0e38f);
        else mn = T(1.0e300);

        for (int z0 = 0; z0 < NZ; z0 += PZ) {
            // ---- stage 1: rows -> kx = 0 .. K (field 1 reloads its row: it is in L1 / L2)
            for (int r = tid; r < ROWS; r += nt) {
                const int zl = r / N, y = r % N;
                const T *src = F + ((int64_t)(z0 + zl) * N + y) * N;
                for (int f = 0; f < nf; ++f) {
                    T x[N];
                    feat_load_row<T, N>(src, x);
                    if (f == 0 && a.mom)
                        feat_row_moments<T, D, N>(x, (D == 3) ? z0 + zl - N / 2 : 0, y - N / 2, s, mn, nf == 1);
                    if (f == 1 || a.log_input) {
                        T peta = 0;
#pragma unroll
                        for (int n = 0; n < N; ++n) {
                            const T lf = feat_log<T>(x[n]);
                            if (f == 1 && x[n] > T(0)) peta += x[n] * lf;
                            x[n] = lf;
                        }
                        if (f == 1 && a.mom) s[5] += (double)peta;
                    }
                    C2<T> X[kFeatKx];
                    r2c_low<N, kFeatKx, T>(x, X, tw);
                    C2<T> *d = X1 + (size_t)f * Lay::X1_FIELD + (size_t)zl * Lay::X1_PLANE + y * kFeatKx;
#pragma unroll
                    for (int k = 0; k < kFeatKx; ++k) d[k] = X[k];
                }
            }
            __syncthreads();
            // ---- stage 2: (plane, kx) columns along axis 1 -> ky = -K .. K
            for (int q = tid; q < nf * PZ * kFeatKx; q += nt) {
                const int f = q / (PZ * kFeatKx);
                const int rem = q % (PZ * kFeatKx);
                const int zl = rem / kFeatKx, kx = rem % kFeatKx;
                const C2<T> *col = X1 + (size_t)f * Lay::X1_FIELD + (size_t)zl * Lay::X1_PLANE + kx;
                C2<T> v[N];
#pragma unroll
                for (int y = 0; y < N; ++y) v[y] = col[y * kFeatKx];
                fft<N, -1, N>(v, tw);
                C2<T> *dst = X2 + (size_t)f * Lay::X2_FIELD + (size_t)(z0 + zl) * Lay::X2_PLANE + kx;
#pragma unroll
                for (int ky = -kFeatK; ky <= kFeatK; ++ky) dst[(ky + kFeatK) * kFeatKx] = v[(ky + N) % N];
            }
            __syncthreads();
        }

        // ---- stage 3: axis-0 sums of the band modes, scaled, to the output rows
        for (int q = tid; q < nf * a.nmodes; q += nt) {
            const int f = q / a.nmodes, m = q % a.nmodes;
            const int kz = a.modes[3 * m], ky = a.modes[3 * m + 1], kx = a.modes[3 * m + 2];
            const C2<T> *src = X2 + (size_t)f * Lay::X2_FIELD + (ky + kFeatK) * kFeatKx + kx;
            C2<T> acc{T(0), T(0)};
            if constexpr (D == 3) {
                const int step = ((kz % N) + N) % N;
                int e = 0;
#pragma unroll 8
                for (int z = 0; z < N; ++z) {
                    acc = acc + cmul(src[(size_t)z * Lay::X2_PLANE], tw[e]);
                    e += step;
                    e -= (e >= N) ? N : 0;
                }
            } else {
                acc = src[0];
            }
            float *out = (f == 0 ? a.feat : a.featL) + row * a.fstride;
            out[2 * m] = (float)(acc.x * scale);
            out[2 * m + 1] = (float)(acc.y * scale);
        }

        // ---- moments: CTA reduction
        if (a.mom) {
            s[7] = (double)mn;
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int k = 0; k < EF_DIAG_STRIDE; ++k) {
                double v = s[k];
                for (int sh = 16; sh > 0; sh >>= 1) {
                    const double u = __shfl_xor_sync(0xffffffffu, v, sh);
                    v = (k == 7) ? fmin(v, u) : v + u;
                }
                if (lane == 0) red[warp * EF_DIAG_STRIDE + k] = v;
            }
        }
        __syncthreads();
        if (a.mom && tid < EF_DIAG_STRIDE) {
            const int k = tid;
            double v = red[k];
            for (int w = 1; w < nt / 32; ++w) v = (k == 7) ? fmin(v, red[w * EF_DIAG_STRIDE + k]) : v + red[w * EF_DIAG_STRIDE + k];
            const double h = a.h;
            const double hd = (D == 3) ? h * h * h : h * h;
            if (k == 0 || k == 5) v *= hd;
            else if (k >= 1 && k <= 3) v *= hd * h;
            else if (k == 4) v *= 0.5 * hd * h * h;
            if (k == 6 || k == 8 || k == 9) v = 0.0;
            if (D == 2 && k == 3) v = 0.0;
            a.mom[row * EF_DIAG_STRIDE + k] = v;
        }
        __syncthreads();
    }
}

}  // namespace ef
