// ef_moments_impl.cuh -- the moments / entropy reduction kernel (ef_moments_entropy).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ef_internal.h"

namespace ef {

template <typename T>
__device__ __forceinline__ T moments_log(T x);
template <>
__device__ __forceinline__ float moments_log<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double moments_log<double>(double x) { return log(x); }

// ------------------------------------------------------------------ moments kernel ---------

// One CTA per cell: moments / entropy of F (and entropy production with Q), FP64 across the cell;
// slot 8 holds the positivity error of Sec. 4.2 (the negative part of F, accumulated directly).
// A warp walks rows (lanes along the contiguous axis, coalesced), four rows in flight; each lane
// sums its values in T over runs of at most 32 terms and folds each run into FP64 accumulators, the
// same split as the fused diagnostics of the collide kernel (no per-point FP64 work: the FP64 pipe
// is a small fraction of the FP32 one).
template <typename T, int D>
__global__ void __launch_bounds__(256) moments_kernel(const T *F, const T *Q, const int64_t *cell_off,
                                                      const int64_t *cell_N, int64_t ncells, int N_uniform,
                                                      double h_uniform_times_N, double *out)
{
    __shared__ double red[8][kDiag];
    T big;
    if constexpr (sizeof(T) == 4) big = T(3.0e38f);
    else big = T(1.0e300);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = blockIdx.x; c < ncells; c += gridDim.x) {
        const int N = cell_N ? (int)cell_N[c] : N_uniform;
        const int nrows = (D == 3) ? N * N : N;
        const int64_t coff = cell_off ? cell_off[c] : c * (int64_t)nrows * N;
        const double h = h_uniform_times_N / N;
        double s[kDiag];
        for (int k = 0; k < kDiag; ++k) s[k] = 0.0;
        T mn = big, mq = big;
        T p0 = 0, pz = 0, py = 0, px = 0, pe = 0, peta = 0, pprod = 0, pneg = 0;
        // four rows per warp in flight: their loads are issued before any of them is used
        constexpr int U = 4;
        const int per_row = (N + 31) / 32;                 // values per lane and row (N <= 64)
        const int run_len = 32 / (U * per_row);            // iterations per FP64 fold: <= 32 terms
        int run = 0;
        for (int r0 = warp; r0 < nrows; r0 += U * nw) {
            T fv[U][2], qv[U][2];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * nw;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int x = lane + 32 * e;
                    const bool ok = r < nrows && x < N;
                    fv[u][e] = ok ? F[coff + (int64_t)r * N + x] : T(0);
                    qv[u][e] = (ok && Q) ? Q[coff + (int64_t)r * N + x] : T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * nw;
                if (r >= nrows) break;                      // uniform across the warp
                const T jz = (D == 3) ? T(r / N - N / 2) : T(0);
                const T jy = (D == 3) ? T(r % N - N / 2) : T(r - N / 2);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int x = lane + 32 * e;
                    if (x >= N) continue;
                    const T f = fv[u][e];
                    const T jx = T(x - N / 2);
                    p0 += f;
                    pz += f * jz;
                    py += f * jy;
                    px += f * jx;
                    pe += f * (jx * jx + jy * jy + jz * jz);
                    if (f > T(0)) {
                        const T lf = moments_log<T>(f);
                        peta += f * lf;
                        if (Q) pprod += qv[u][e] * lf;
                    }
                    mn = f < mn ? f : mn;
                    pneg += f < T(0) ? -f : T(0);
                    if (Q) mq = qv[u][e] < mq ? qv[u][e] : mq;
                }
            }
            if (++run >= run_len || r0 + U * nw >= nrows) {
                s[0] += (double)p0;
                if (D == 3) {
                    s[1] += (double)pz;
                    s[2] += (double)py;
                    s[3] += (double)px;
                } else {
                    s[1] += (double)py;
                    s[2] += (double)px;
                }
                s[4] += (double)pe;
                s[5] += (double)peta;
                s[6] += (double)pprod;
                s[8] += (double)pneg;
                p0 = pz = py = px = pe = peta = pprod = pneg = T(0);
                run = 0;
            }
        }
        s[7] = (double)mn;
        s[9] = Q ? (double)mq : 0.0;
        for (int k = 0; k < kDiag; ++k) {
            double v = s[k];
            for (int sh = 16; sh > 0; sh >>= 1) {
                const double u = __shfl_xor_sync(0xffffffffu, v, sh);
                v = (k == 7 || k == 9) ? fmin(v, u) : v + u;
            }
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < kDiag) {
            const int k = threadIdx.x;
            double v = red[0][k];
            for (int w = 1; w < nw; ++w) v = (k == 7 || k == 9) ? fmin(v, red[w][k]) : v + red[w][k];
            const double hd = (D == 3) ? h * h * h : h * h;
            if (k == 0 || k == 5) v *= hd;
            else if (k >= 1 && k <= 3) v *= hd * h;
            else if (k == 4) v *= 0.5 * hd * h * h;
            if (k == 8) {       // positivity error (sum|F| - sum F) / sum|F| = 2 neg / (sum F + 2 neg)
                double m = red[0][0];
                for (int w = 1; w < nw; ++w) m += red[w][0];
                v = (m + 2.0 * v) > 0.0 ? 2.0 * v / (m + 2.0 * v) : 0.0;
            }
            if (D == 2 && k == 3) v = 0.0;
            out[c * kDiag + k] = v;
        }
        __syncthreads();
    }
}

}  // namespace ef
