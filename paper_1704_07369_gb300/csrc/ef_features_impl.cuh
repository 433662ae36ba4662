// ef_features_impl.cuh -- low Fourier modes of a cell (the learned surrogate's input and output
// band) in one pass over the cell, optionally with the modes of ln F and the cell's moments.
//
// The band is |k| <= EF_FEATURE_K (K) in the canonical half space; with the library's
// index-origin convention
//   Fh_k = N^-d sum_i F[i] exp(-2 pi i k.i / N)      (i the array index, 0 .. N-1 per axis).
// One CTA per cell (persistent over cells).  For a chunk of PZ axis-0 planes at a time:
//   stage 1  every row along the contiguous axis gets its kx = 0 .. K spectrum by a folded direct
//            sum with compile-time weights, kept in shared memory;
//   stage 2  every (plane, kx) column gets its ky = -K .. K spectrum along axis 1 the same way;
//   stage 3  every band mode adds the chunk's axis-0 values times exp(-2 pi i kz z / N) to its
//            accumulator (a direct sum over z, one register pair per mode a thread owns);
// after the last chunk the accumulators, scaled, are the output rows.  Only one chunk of planes is
// ever held in shared memory, so FP32 cells up to N = 40 also stage the next chunk's raw planes
// with asynchronous copies while the current one is transformed.
// 2D cells are one plane (stage 3 is the identity).  The moments: each thread sums its rows in T,
// each warp its threads' sums in T, and the CTA the warps' sums in FP64, once per cell.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

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

// band modes |k| <= K in the canonical half space (3D), the most a cell has
constexpr int feat_band_modes()
{
    int n = 0;
    for (int a = -kFeatK; a <= kFeatK; ++a)
        for (int b = -kFeatK; b <= kFeatK; ++b)
            for (int c = 0; c <= kFeatK; ++c)
                if (a * a + b * b + c * c <= kFeatK * kFeatK && (c > 0 || b > 0 || (b == 0 && a >= 0))) ++n;
    return n;
}

// CTAs of 4 warps, several per SM (cells in flight overlap their barrier phases): 168 registers
// for N <= 32 (3 CTAs per SM), 255 above (2 per SM)
constexpr int kFeatThreads = 128;
template <int N>
constexpr int feat_min_blocks() { return N <= 32 ? 3 : 2; }
// accumulators per thread: both fields' band modes over the CTA
constexpr int kFeatQ = (2 * feat_band_modes() + kFeatThreads - 1) / kFeatThreads;

template <typename T, int D, int N>
struct FeatLayout {
    static constexpr int PZ = (D == 3) ? feat_pz<N, sizeof(T) == 4 ? 8 : 4>() : 1;
    static constexpr int NZ = (D == 3) ? N : 1;
    static constexpr int X1_PLANE = N * kFeatKx + 1;         // odd complex stride per plane
    static constexpr int X1_FIELD = PZ * X1_PLANE;
    static constexpr int X2_PLANE = kFeatKy * kFeatKx;
    static constexpr int X2_FIELD = PZ * X2_PLANE;             // the current chunk's planes only
    static constexpr size_t BASE = (size_t)N * sizeof(C2<T>) + 2 * (size_t)(X1_FIELD + X2_FIELD) * sizeof(C2<T>) +
                                   8 * EF_DIAG_STRIDE * sizeof(double);
    // FP32 3D cells whose two-field layout plus one chunk of raw planes still leaves the CTAs per
    // SM of the launch bounds: each chunk of PZ planes is staged in shared memory by asynchronous
    // copies (cp.async, 16 bytes a thread) issued while the previous chunk is being transformed
    static constexpr size_t RB_FULL = (size_t)PZ * N * N * sizeof(T);
    static constexpr bool PF = sizeof(T) == 4 && D == 3 && N % 4 == 0 &&
                               (BASE + RB_FULL + 16 + 1024) * feat_min_blocks<N>() <= 228 * 1024;
    static constexpr size_t RB_BYTES = PF ? RB_FULL : 0;
    static constexpr size_t bytes(int nf)
    {
        return (size_t)N * sizeof(C2<T>) + (size_t)nf * (X1_FIELD + X2_FIELD) * sizeof(C2<T>) +
               8 * EF_DIAG_STRIDE * sizeof(double) + (PF ? RB_BYTES + 16 : 0);
    }
};

// position of 16-byte piece i of staged row r: XOR with the row's low bits when a row has a power
// of two of pieces, else a rotation by the row (consecutive rows start on different banks)
template <int NC>
__device__ __forceinline__ int feat_swz(int i, int r)
{
    if constexpr ((NC & (NC - 1)) == 0) return i ^ (r & (NC < 8 ? NC - 1 : 7));
    else return (i + r) % NC;
}

template <typename T, int N>
__device__ __forceinline__ void feat_load_row_swz(const float4 *RB, int r, T (&x)[N])
{
    constexpr int NC = N / 4;
    const float4 *row = RB + r * NC;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const float4 v = row[feat_swz<NC>(i, r)];
        x[4 * i] = v.x; x[4 * i + 1] = v.y; x[4 * i + 2] = v.z; x[4 * i + 3] = v.w;
    }
}

template <typename T>
__device__ __forceinline__ T feat_log(T x);
template <>
__device__ __forceinline__ float feat_log<float>(float x) { return __logf(x > 1e-30f ? x : 1e-30f); }
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

// row sums of one row, added to the thread's partial sums (T; folded into FP64 once per cell):
// mass, the two or three momentum sums, energy, entropy.  The entropy term only with eta
// (otherwise the ln F pass adds it, from the logarithms it computes anyway)
template <typename T, int D, int N>
__device__ __forceinline__ void feat_row_moments(const T (&x)[N], int jz, int jy, T (&ms)[6], T &mn, bool eta)
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
    ms[0] += p0;
    if (D == 3) {
        ms[1] += p0 * T(jz);
        ms[2] += p0 * T(jy);
        ms[3] += px;
    } else {
        ms[1] += p0 * T(jy);
        ms[2] += px;
    }
    ms[4] += pe + p0 * T(jy * jy + jz * jz);
    ms[5] += peta;
}

// Compile-time cos(2 pi p / q) and sin(2 pi p / q) for integers p, q: the angle is folded by its
// symmetries into |x| <= pi/4 and summed as a Taylor series (terms to x^25: far below FP64 rounding).
constexpr double kCtPi = 3.14159265358979323846;
constexpr double ct_sin_series(double x)
{
    double t = x, s = x;
    for (int i = 1; i <= 12; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
constexpr double ct_cos_series(double x)
{
    double t = 1.0, s = 1.0;
    for (int i = 1; i <= 12; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
constexpr double ct_cos2pi(long p, long q)
{
    long r = ((p % q) + q) % q;                 // angle a = 2 pi r / q in [0, 2 pi)
    if (2 * r > q) r = q - r;                   // cos is even: a in [0, pi]
    if (8 * r <= q) return ct_cos_series(2.0 * kCtPi * r / q);                           // a <= pi / 4
    if (8 * r <= 3 * q) return ct_sin_series(2.0 * kCtPi * (q - 4 * r) / (4.0 * q));     // cos a = sin(pi/2 - a)
    return -ct_cos_series(2.0 * kCtPi * (q - 2 * r) / (2.0 * q));                        // cos a = -cos(pi - a)
}
constexpr double ct_sin2pi(long p, long q) { return ct_cos2pi(4 * p - q, 4 * q); }    // sin x = cos(x - pi/2)

template <long P, long Q>
struct Trig2Pi {
    static constexpr double c = ct_cos2pi(P, Q);
    static constexpr double s = ct_sin2pi(P, Q);
};

// One real row -> its spectrum X_k = sum_n x_n exp(-2 pi i k n / N) at k = 0 .. K (unscaled) by the
// direct sum, folded twice by the symmetries of the kernel: with a_n = x_n + x_{N-n} and
// b_n = x_n - x_{N-n}, Re X_k = x_0 + (-1)^k x_{N/2} + sum_{n<N/2} a_n cos(2 pi k n / N) and
// Im X_k = -sum_{n<N/2} b_n sin(2 pi k n / N); pairing n with N/2 - n then leaves N/4 - 1 terms per
// part, weighted by the compile-time constants (even k: a_n + a_{N/2-n}, b_n - b_{N/2-n}; odd k:
// a_n - a_{N/2-n}, b_n + b_{N/2-n}).  About 2N + 2(K+1)N/4 operations for the whole band.
template <typename T, int N, int k, int... n>
__device__ __forceinline__ C2<T> rdft_mode(const T (&ce)[N / 4], const T (&co)[N / 4], const T (&se)[N / 4],
                                           const T (&so)[N / 4], T e0, T o0, T aq, T bq, std::integer_sequence<int, n...>)
{
    constexpr bool ev = (k % 2) == 0;
    const T(&cc)[N / 4] = ev ? ce : co;
    const T(&ss)[N / 4] = ev ? se : so;
    T re = ev ? e0 : o0;
    if constexpr (k % 4 == 0) re += aq;
    else if constexpr (k % 4 == 2) re -= aq;
    T im = T(0);
    if constexpr (k % 4 == 1) im = bq;
    else if constexpr (k % 4 == 3) im = -bq;
    ((re = fma(cc[n + 1], T(Trig2Pi<(long)k * (n + 1), N>::c), re)), ...);
    if constexpr (k != 0) ((im = fma(ss[n + 1], T(Trig2Pi<(long)k * (n + 1), N>::s), im)), ...);
    return C2<T>{re, -im};
}

template <typename T, int N, int... k>
__device__ __forceinline__ void rdft_band_all(const T (&x)[N], C2<T> (&X)[sizeof...(k)], std::integer_sequence<int, k...>)
{
    static_assert(N % 4 == 0, "the folded direct sum wants N a multiple of 4");
    constexpr int H = N / 2, Q = N / 4;
    T ce[Q], co[Q], se[Q], so[Q];               // [1 .. Q-1] used
#pragma unroll
    for (int n = 1; n < Q; ++n) {
        const T an = x[n] + x[N - n], bn = x[n] - x[N - n];
        const T am = x[H - n] + x[H + n], bm = x[H - n] - x[H + n];
        ce[n] = an + am;
        co[n] = an - am;
        se[n] = bn - bm;
        so[n] = bn + bm;
    }
    ce[0] = co[0] = se[0] = so[0] = T(0);
    const T aq = x[Q] + x[N - Q], bq = x[Q] - x[N - Q];
    const T e0 = x[0] + x[H], o0 = x[0] - x[H];
    ((X[k] = rdft_mode<T, N, k>(ce, co, se, so, e0, o0, aq, bq, std::make_integer_sequence<int, Q - 1>{})), ...);
}

template <typename T, int N, int KX>
__device__ __forceinline__ void rdft_band(const T (&x)[N], C2<T> (&X)[KX])
{
    rdft_band_all<T, N>(x, X, std::make_integer_sequence<int, KX>{});
}

// One complex column -> X_k = sum_n v_n exp(-2 pi i k n / N) at k = -K .. K by the same folded
// direct sum: with p_n = v_n + v_{N-n} and m_n = v_n - v_{N-n},
//   X_{+-k} = C_k -+ i S_k,  C_k = v_0 + (-1)^k v_{N/2} + sum_{n<N/2} p_n cos(2 pi k n / N),
//   S_k = sum_{n<N/2} m_n sin(2 pi k n / N),
// and pairing n with N/2 - n halves both sums again (even k: p_n + p_{N/2-n}, m_n - m_{N/2-n};
// odd k: p_n - p_{N/2-n}, m_n + m_{N/2-n}).  Y[K + k] receives X_k.
template <typename T, int N, int K, int k, int... n>
__device__ __forceinline__ void cdft_mode(const C2<T> (&pe)[N / 4], const C2<T> (&po)[N / 4], const C2<T> (&me)[N / 4],
                                          const C2<T> (&mo)[N / 4], C2<T> e0, C2<T> o0, C2<T> pq, C2<T> mq,
                                          C2<T> (&Y)[2 * K + 1], std::integer_sequence<int, n...>)
{
    constexpr bool ev = (k % 2) == 0;
    const C2<T>(&pp)[N / 4] = ev ? pe : po;
    const C2<T>(&mm)[N / 4] = ev ? me : mo;
    C2<T> c = ev ? e0 : o0;
    if constexpr (k % 4 == 0) c = c + pq;
    else if constexpr (k % 4 == 2) c = c - pq;
    ((c.x = fma(pp[n + 1].x, T(Trig2Pi<(long)k * (n + 1), N>::c), c.x)), ...);
    ((c.y = fma(pp[n + 1].y, T(Trig2Pi<(long)k * (n + 1), N>::c), c.y)), ...);
    if constexpr (k == 0) {
        Y[K] = c;
    } else {
        C2<T> sv{T(0), T(0)};
        if constexpr (k % 4 == 1) sv = mq;
        else if constexpr (k % 4 == 3) sv = C2<T>{-mq.x, -mq.y};
        ((sv.x = fma(mm[n + 1].x, T(Trig2Pi<(long)k * (n + 1), N>::s), sv.x)), ...);
        ((sv.y = fma(mm[n + 1].y, T(Trig2Pi<(long)k * (n + 1), N>::s), sv.y)), ...);
        Y[K + k] = C2<T>{c.x + sv.y, c.y - sv.x};          // C - i S
        Y[K - k] = C2<T>{c.x - sv.y, c.y + sv.x};          // C + i S
    }
}

template <typename T, int N, int K, int... k>
__device__ __forceinline__ void cdft_band_all(const C2<T> (&v)[N], C2<T> (&Y)[2 * K + 1], std::integer_sequence<int, k...>)
{
    static_assert(N % 4 == 0, "the folded direct sum wants N a multiple of 4");
    constexpr int H = N / 2, Q = N / 4;
    C2<T> pe[Q], po[Q], me[Q], mo[Q];           // [1 .. Q-1] used
#pragma unroll
    for (int n = 1; n < Q; ++n) {
        const C2<T> pn = v[n] + v[N - n], mn = v[n] - v[N - n];
        const C2<T> pm = v[H - n] + v[H + n], mm = v[H - n] - v[H + n];
        pe[n] = pn + pm;
        po[n] = pn - pm;
        me[n] = mn - mm;
        mo[n] = mn + mm;
    }
    pe[0] = po[0] = me[0] = mo[0] = C2<T>{T(0), T(0)};
    const C2<T> pq = v[Q] + v[N - Q], mq = v[Q] - v[N - Q];
    const C2<T> e0 = v[0] + v[H], o0 = v[0] - v[H];
    (cdft_mode<T, N, K, k>(pe, po, me, mo, e0, o0, pq, mq, Y, std::make_integer_sequence<int, Q - 1>{}), ...);
}

template <typename T, int N, int K>
__device__ __forceinline__ void cdft_band(const C2<T> (&v)[N], C2<T> (&Y)[2 * K + 1])
{
    cdft_band_all<T, N, K>(v, Y, std::make_integer_sequence<int, K + 1>{});
}

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
    // chunk staging buffer: PZ * N rows of N / 4 float4 pieces, each row's pieces permuted so that
    // one thread per row reads without bank conflicts
    float4 *RB = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(red + 8 * EF_DIAG_STRIDE) + 15) & ~(uintptr_t)15);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < N; j += nt) {
        T sn, cs;
        if constexpr (sizeof(T) == 4) sincospif(T(2 * j) / T(N), &sn, &cs);
        else sincospi(T(2 * j) / T(N), &sn, &cs);
        tw[j] = C2<T>{cs, -sn};
    }
    const T scale = T(1) / T(D == 3 ? N * N * N : N * N);
    const int64_t ncells = a.dev_ncells ? (int64_t)*a.dev_ncells : a.ncells;
    constexpr int64_t CELLSZ = (D == 3) ? (int64_t)N * N * N : (int64_t)N * N;
    // all threads: asynchronous 16-byte copies of planes [zz, zz + PZ) of cell cc into the buffer
    auto rb_issue = [&](int64_t cc, int zz) {
        if constexpr (Lay::PF) {
            constexpr int NC = N / 4;
            const int64_t off = a.cell_off ? a.cell_off[cc] : cc * CELLSZ;
            const float4 *src = reinterpret_cast<const float4 *>(reinterpret_cast<const T *>(a.F) + off + (int64_t)zz * N * N);
            const uint32_t base = (uint32_t)__cvta_generic_to_shared(RB);
            for (int p = tid; p < PZ * N * NC; p += kFeatThreads) {
                const int r = p / NC, i = p % NC;
                const uint32_t dst = base + (uint32_t)(r * NC + feat_swz<NC>(i, r)) * 16u;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + p) : "memory");
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
    };
    if (Lay::PF && (int64_t)blockIdx.x < ncells) {
        rb_issue(blockIdx.x, 0);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();
    for (int64_t c = blockIdx.x; c < ncells; c += gridDim.x) {
        const int64_t coff = a.cell_off ? a.cell_off[c] : c * (int64_t)(D == 3 ? N * N * N : N * N);
        const int64_t row = a.cell_id ? a.cell_id[c] : c;
        const T *F = reinterpret_cast<const T *>(a.F) + coff;
        T ms[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        T mn;
        if constexpr (sizeof(T) == 4) mn = T(3.0e38f);
        else mn = T(1.0e300);
        C2<T> acc[kFeatQ];
#pragma unroll
        for (int j = 0; j < kFeatQ; ++j) acc[j] = C2<T>{T(0), T(0)};

        for (int z0 = 0; z0 < NZ; z0 += PZ) {
            // ---- stage 1: rows -> kx = 0 .. K (field 1 reloads its row: from the staged chunk, or L1 / L2)
            for (int r = tid; r < ROWS; r += nt) {
                const int zl = r / N, y = r % N;
                const T *src = F + ((int64_t)(z0 + zl) * N + y) * N;
                for (int f = 0; f < nf; ++f) {
                    T x[N];
                    if constexpr (Lay::PF) feat_load_row_swz<T, N>(RB, r, x);
                    else feat_load_row<T, N>(src, x);
                    if (f == 0 && a.mom)
                        feat_row_moments<T, D, N>(x, (D == 3) ? z0 + zl - N / 2 : 0, y - N / 2, ms, mn, nf == 1);
                    if (f == 1 || a.log_input) {
                        T peta = 0;
#pragma unroll
                        for (int n = 0; n < N; ++n) {
                            const T lf = feat_log<T>(x[n]);
                            if (f == 1 && x[n] > T(0)) peta += x[n] * lf;
                            x[n] = lf;
                        }
                        if (f == 1 && a.mom) ms[5] += peta;
                    }
                    C2<T> X[kFeatKx];
                    rdft_band<T, N, kFeatKx>(x, X);
                    C2<T> *d = X1 + (size_t)f * Lay::X1_FIELD + (size_t)zl * Lay::X1_PLANE + y * kFeatKx;
#pragma unroll
                    for (int k = 0; k < kFeatKx; ++k) d[k] = X[k];
                }
            }
            __syncthreads();
            if constexpr (Lay::PF) {                  // stage the next chunk (or the next cell's first)
                if (z0 + PZ < NZ) rb_issue(c, z0 + PZ);
                else if (c + (int64_t)gridDim.x < ncells) rb_issue(c + gridDim.x, 0);
            }
            // ---- stage 2: (plane, kx) columns along axis 1 -> ky = -K .. K
            for (int q = tid; q < nf * PZ * kFeatKx; q += nt) {
                const int f = q / (PZ * kFeatKx);
                const int rem = q % (PZ * kFeatKx);
                const int zl = rem / kFeatKx, kx = rem % kFeatKx;
                const C2<T> *col = X1 + (size_t)f * Lay::X1_FIELD + (size_t)zl * Lay::X1_PLANE + kx;
                C2<T> v[N];
#pragma unroll
                for (int y = 0; y < N; ++y) v[y] = col[y * kFeatKx];
                C2<T> Yk[kFeatKy];
                cdft_band<T, N, kFeatK>(v, Yk);
                C2<T> *dst = X2 + (size_t)f * Lay::X2_FIELD + (size_t)zl * Lay::X2_PLANE + kx;
#pragma unroll
                for (int j = 0; j < kFeatKy; ++j) dst[j * kFeatKx] = Yk[j];
            }
            if constexpr (Lay::PF) asm volatile("cp.async.wait_all;\n" ::: "memory");   // the next chunk has landed
            __syncthreads();
            // ---- stage 3: each band mode adds the chunk's planes times exp(-2 pi i kz z / N)
            // (the next chunk's stage 2 rewrites X2 only after its stage-1 barrier)
#pragma unroll
            for (int j = 0; j < kFeatQ; ++j) {
                const int q = tid + j * kFeatThreads;
                if (q < nf * a.nmodes) {
                    const int f = q >= a.nmodes ? 1 : 0, m = q - f * a.nmodes;
                    const int kz = __ldg(a.modes + 3 * m), ky = __ldg(a.modes + 3 * m + 1), kx = __ldg(a.modes + 3 * m + 2);
                    const C2<T> *src = X2 + (size_t)f * Lay::X2_FIELD + (ky + kFeatK) * kFeatKx + kx;
                    if constexpr (D == 3) {
                        const int step = ((kz % N) + N) % N;
                        int e = (step * z0) % N;
#pragma unroll
                        for (int zl = 0; zl < PZ; ++zl) {
                            acc[j] = acc[j] + cmul(src[(size_t)zl * Lay::X2_PLANE], tw[e]);
                            e += step;
                            e -= (e >= N) ? N : 0;
                        }
                    } else {
                        acc[j] = src[0];
                    }
                }
            }
        }

        // ---- the accumulated band modes, scaled, to the output rows
#pragma unroll
        for (int j = 0; j < kFeatQ; ++j) {
            const int q = tid + j * kFeatThreads;
            if (q < nf * a.nmodes) {
                const int f = q >= a.nmodes ? 1 : 0, m = q - f * a.nmodes;
                float *out = (f == 0 ? a.feat : a.featL) + row * a.fstride;
                out[2 * m] = (float)(acc[j].x * scale);
                out[2 * m + 1] = (float)(acc[j].y * scale);
            }
        }

        // ---- moments: CTA reduction
        if (a.mom) {                              // warp sums in T, the CTA's in FP64
            T s[EF_DIAG_STRIDE];
#pragma unroll
            for (int k = 0; k < EF_DIAG_STRIDE; ++k) s[k] = k < 6 ? ms[k] : T(0);
            s[7] = mn;
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int k = 0; k < EF_DIAG_STRIDE; ++k) {
                if (k == 6 || k >= 8) continue;       // zero slots
                T v = s[k];
                for (int sh = 16; sh > 0; sh >>= 1) {
                    const T u = __shfl_xor_sync(0xffffffffu, v, sh);
                    v = (k == 7) ? (u < v ? u : v) : v + u;
                }
                if (lane == 0) red[warp * EF_DIAG_STRIDE + k] = (double)v;
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
