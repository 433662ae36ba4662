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

// a + b = s + e exactly (Knuth's two-sum, six FP32 operations, no reassociation)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One CTA per cell: moments / entropy of F (and entropy production with Q); slot 8 holds the
// positivity error of Sec. 4.2 (the negative part of F, accumulated directly).
// A warp walks rows (lanes along the contiguous axis, coalesced), four rows in flight; each lane
// sums its values in T over runs of at most 32 terms.  FP64 input folds each run into FP64
// accumulators.  FP32 input folds each run into a compensated FP32 pair (two-sum: the pair holds
// the runs' sum to about FP32 rounding of the total), and a warp adds its lanes' pairs in FP32;
// FP64 is used only for the CTA's sum of its warps, because the FP64 pipe is a small fraction of
// the FP32 one.  FP32 error: at most about (3 + 32 + 8) * 2^-24 of the sum of |terms| (a float4's
// four terms, a run of 32 float4 partials, the pair, the warp); the logarithm is the fast one
// (a few ulp), in the same budget.
// HASQ: Q is given (the FP32 vector path then keeps four float4 of F and four of Q in flight per
// thread; with F alone, eight of F: one cell per CTA leaves few loads in flight otherwise).
template <typename T, int D, bool HASQ>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) moments_kernel(const T *F, const T *Q, const int64_t *cell_off,
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
        const float inv_n = 1.0f / float(N);
        double s[kDiag];
        for (int k = 0; k < kDiag; ++k) s[k] = 0.0;
        float sh_[kDiag], sl_[kDiag];                      // FP32 input: compensated pairs
#pragma unroll
        for (int k = 0; k < kDiag; ++k) sh_[k] = sl_[k] = 0.f;
        T mn = big, mq = big;
        T p0 = 0, pz = 0, py = 0, px = 0, pe = 0, peta = 0, pprod = 0, pneg = 0;
        // FP32 cells with N a multiple of 4: the cell as a flat array of float4, four per thread in
        // flight (the row loop below keeps only 4 KB per CTA in flight, too little to cover HBM
        // latency); each float4 lies in one row, its index split by the rounding-safe FP32 divisions
        const bool vec = sizeof(T) == 4 && (N % 4) == 0;
        if constexpr (sizeof(T) == 4) {
            if (vec) {
                const int nv = (int)((int64_t)nrows * N / 4);
                const float4 *F4 = reinterpret_cast<const float4 *>(F + coff);
                const float4 *Q4 = HASQ ? reinterpret_cast<const float4 *>(Q + coff) : nullptr;
                constexpr int UV = HASQ ? 4 : 8;
                const int bd = blockDim.x;
                const float half = float(N / 2);
                int run = 0;
                for (int v0 = threadIdx.x; v0 < nv; v0 += UV * bd) {
                    float4 fv[UV], qv[HASQ ? UV : 1];
#pragma unroll
                    for (int u = 0; u < UV; ++u) {
                        const int v = v0 + u * bd;
                        const bool ok = v < nv;
                        fv[u] = ok ? F4[v] : make_float4(0.f, 0.f, 0.f, 0.f);
                        if constexpr (HASQ) qv[u] = ok ? Q4[v] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < UV; ++u) {
                        const int v = v0 + u * bd;
                        if (v >= nv) break;
                        // (i + 1/2) / N for i < N^3 <= 2^18: at least 1 / (2N) from an integer, far
                        // more than the FP32 rounding of the product
                        const int i0 = 4 * v;
                        const int q = __float2int_rz((float(i0) + 0.5f) * inv_n);        // row
                        const int x0 = i0 - q * N;
                        int zz = 0, yy = q;
                        if (D == 3) {
                            zz = __float2int_rz((float(q) + 0.5f) * inv_n);
                            yy = q - zz * N;
                        }
                        const float jz = (D == 3) ? float(zz) - half : 0.f, jy = float(yy) - half;
                        const float jx0 = float(x0) - half;
                        const float fa[4] = {fv[u].x, fv[u].y, fv[u].z, fv[u].w};
                        float qa[4] = {0.f, 0.f, 0.f, 0.f};
                        if constexpr (HASQ) {
                            qa[0] = qv[u].x; qa[1] = qv[u].y; qa[2] = qv[u].z; qa[3] = qv[u].w;
                        }
                        float sf = 0.f, sfx = 0.f, sfxx = 0.f, seta = 0.f, sprod = 0.f, sneg = 0.f;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float f = fa[j], jx = jx0 + float(j);
                            sf += f;
                            const float fx = f * jx;
                            sfx += fx;
                            sfxx = fmaf(fx, jx, sfxx);
                            const float lf = __logf(f > 1e-30f ? f : 1e-30f);
                            seta += f > 0.f ? f * lf : 0.f;
                            if constexpr (HASQ) sprod += f > 0.f ? qa[j] * lf : 0.f;
                            mn = fminf(mn, f);
                            sneg += f < 0.f ? -f : 0.f;
                            if constexpr (HASQ) mq = fminf(mq, qa[j]);
                        }
                        p0 += sf;
                        if (D == 3) {
                            pz += sf * jz;
                            py += sf * jy;
                        } else {
                            py += sf * jy;
                        }
                        px += sfx;
                        pe += sfxx + sf * (jy * jy + jz * jz);
                        peta += seta;
                        pprod += sprod;
                        pneg += sneg;
                    }
                    if (++run >= 32 / UV || v0 + UV * bd >= nv) {        // <= 32 float4 partials a run
                        const float v[kDiag] = {p0, D == 3 ? pz : py, D == 3 ? py : px, D == 3 ? px : 0.f, pe,
                                                peta, pprod, 0.f, pneg, 0.f};
#pragma unroll
                        for (int k = 0; k < kDiag; ++k) {
                            if (k == 7 || k == 9 || (D == 2 && k == 3)) continue;
                            float t, e;
                            two_sum(sh_[k], v[k], t, e);
                            sh_[k] = t;
                            sl_[k] += e;
                        }
                        p0 = pz = py = px = pe = peta = pprod = pneg = 0.f;
                        run = 0;
                    }
                }
            }
        }
        if (!vec) {
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
                    // r / N without an integer division: (r + 1/2) / N is at least 1 / (2N) away from
                    // an integer, far more than the FP32 rounding of the product for r < N^2 <= 2^12
                    const int rz = (D == 3) ? __float2int_rz((float(r) + 0.5f) * inv_n) : 0;
                    const T jz = (D == 3) ? T(rz - N / 2) : T(0);
                    const T jy = (D == 3) ? T(r - rz * N - N / 2) : T(r - N / 2);
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
                    T v[kDiag] = {p0, D == 3 ? pz : py, D == 3 ? py : px, D == 3 ? px : T(0), pe, peta, pprod, T(0), pneg, T(0)};
    #pragma unroll
                    for (int k = 0; k < kDiag; ++k) {
                        if (k == 7 || k == 9 || (D == 2 && k == 3)) continue;
                        if constexpr (sizeof(T) == 4) {
                            float t, e;
                            two_sum(sh_[k], (float)v[k], t, e);
                            sh_[k] = t;
                            sl_[k] += e;
                        } else {
                            s[k] += (double)v[k];
                        }
                    }
                    p0 = pz = py = px = pe = peta = pprod = pneg = T(0);
                    run = 0;
                }
            }
        }
        if constexpr (sizeof(T) == 4) {
            float w[kDiag];
#pragma unroll
            for (int k = 0; k < kDiag; ++k) w[k] = sh_[k] + sl_[k];
            w[7] = (float)mn;
            w[9] = Q ? (float)mq : 0.f;
#pragma unroll
            for (int k = 0; k < kDiag; ++k) {
                float x = w[k];
                for (int sh = 16; sh > 0; sh >>= 1) {
                    const float u = __shfl_xor_sync(0xffffffffu, x, sh);
                    x = (k == 7 || k == 9) ? fminf(x, u) : x + u;
                }
                if (lane == 0) red[warp][k] = (double)x;
            }
        } else {
            s[7] = (double)mn;
            s[9] = Q ? (double)mq : 0.0;
            for (int k = 0; k < kDiag; ++k) {
                double x = s[k];
                for (int sh = 16; sh > 0; sh >>= 1) {
                    const double u = __shfl_xor_sync(0xffffffffu, x, sh);
                    x = (k == 7 || k == 9) ? fmin(x, u) : x + u;
                }
                if (lane == 0) red[warp][k] = x;
            }
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
