// ef_surrogate.cu -- the learned surrogate path: low Fourier modes of F -> MLP -> low modes of
// Q^sigma, with per-cell gates, a seeded plain-operator audit and device-side fallback.
//
// Normalisation (the operator is quadratic, Q[a F] = a^2 Q[F], and commutes with velocity shifts):
// with m = Fh_0 the zero mode and u the mean velocity (momentum / mass),
//   x_k = (Fh_k e^{i pi k.u/L} / m - mu_k) / s_k,      y_k = (Qh_k e^{i pi k.u/L} / m^2 - nu_k) / t,
// column statistics (mu, s, nu) and one output scale t fitted on the training set.  The prediction sets Qh_0 = 0 (mass
// conservation, Theorem 1).
// Gates, every cell: finite prediction; every normalised input within +-x_max (inside the
// training envelope); band entropy production P = 2 N^3 sum_{k != 0} Re(Qh_k conj(Lh_k)) <= 0 with
// Lh the low modes of ln F (the discrete H-theorem, Theorem 1, restricted to the band).  A
// seeded fraction of cells is also audited against the plain operator.  Gate failures and audited
// cells get the plain operator's band; if more than a set fraction of the audited cells (by default
// none) miss the tolerance, every remaining cell falls back too.  No host synchronisation: counts and lists stay on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "ef.h"
#include "ef_fft.cuh"
#include "ef_launch.h"

namespace {

constexpr int kStride = EF_FEATURE_STRIDE;

ef_status sfail(ef_status s, const std::string &m)
{
    ef::set_last_error(m.c_str());
    return s;
}

ef_status scuda(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    ef::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

int sgrid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// Per-cell scalars of the moments, in FP32 arithmetic (the network's inputs are FP32, and FP64 is a
// narrow pipe): the mean velocity u = momentum / mass, and the kinetic temperature and relative
// entropy to the local Maxwellian (zero at equilibrium):
//   theta = (2E / rho - |u|^2) / d,  KL = eta / rho - ln rho + (d / 2)(ln(2 pi theta) + 1)
__device__ __forceinline__ void cell_velocity(const double *mi, float &ux, float &uy, float &uz)
{
    const float r = 1.0f / (float)mi[0];
    ux = (float)mi[1] * r;
    uy = (float)mi[2] * r;
    uz = (float)mi[3] * r;
}

__device__ __forceinline__ void cell_theta_kl(const double *mi, int d, float &theta, float &kl)
{
    const float rho = (float)mi[0], r = 1.0f / rho;
    float ux, uy, uz;
    cell_velocity(mi, ux, uy, uz);
    theta = (2.0f * (float)mi[4] * r - (ux * ux + uy * uy + uz * uz)) / (float)d;
    kl = (float)mi[5] * r - logf(rho) + 0.5f * (float)d * (logf(6.283185307179586f * theta) + 1.0f);
}

// De-translated, mass-normalised features: with m = Fh_0 and u = momentum / mass the mean velocity,
//   x~_k = Fh_k exp(+i pi k.u / L) / m,     y~_k = Qh_k exp(+i pi k.u / L) / m^2
// (a velocity shift by u multiplies mode k by exp(-i pi k.u / L); the operator commutes with it up
// to aliasing, so the network sees the family without its bulk velocity).  One thread per mode.
__global__ void prep_kernel(const float *featF, const float *featQ, const double *mom, const int *kvec, int64_t n,
                            int nmodes, int idx0, float pi_over_L, int extra, int d, float *Xt, float *Yt)
{
    const int64_t total = n * nmodes;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / nmodes;
        const int j = (int)(q % nmodes);
        const double *mi = mom + i * EF_DIAG_STRIDE;
        if (extra && j == 0) {
            float theta, kl;
            cell_theta_kl(mi, d, theta, kl);
            Xt[i * kStride + 2 * nmodes] = theta;
            Xt[i * kStride + 2 * nmodes + 1] = kl;
        }
        float ux, uy, uz;
        cell_velocity(mi, ux, uy, uz);
        const float ph = pi_over_L * (kvec[3 * j] * ux + kvec[3 * j + 1] * uy + kvec[3 * j + 2] * uz);
        float sn, cs;
        sincosf(ph, &sn, &cs);
        const float m = featF[i * kStride + 2 * idx0];
        const float fr = featF[i * kStride + 2 * j], fi = featF[i * kStride + 2 * j + 1];
        Xt[i * kStride + 2 * j] = (fr * cs - fi * sn) / m;
        Xt[i * kStride + 2 * j + 1] = (fr * sn + fi * cs) / m;
        if (featQ && Yt) {
            const float qr = featQ[i * kStride + 2 * j], qi = featQ[i * kStride + 2 * j + 1];
            Yt[i * kStride + 2 * j] = (qr * cs - qi * sn) / (m * m);
            Yt[i * kStride + 2 * j + 1] = (qr * sn + qi * cs) / (m * m);
        }
    }
}

// Floor of an input column's standard deviation.  Inputs are relative to the mass mode (|x~_0| = 1);
// after de-translation an isotropic cell has real band modes, so imaginary parts (and modes a family
// never excites) vary only at round-off level, and standardising them by their own spread would feed
// the network amplified rounding noise.
constexpr double kSdFloor = 1e-4;

// column mean / std of the prepared inputs and outputs; the output scale is one global RMS
__global__ void stats_kernel(const float *Xt, const float *Yt, int64_t n, int nin, int nf, float *mu, float *sd, float *nu,
                             float *colvar)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nin) return;
    double sx = 0, sxx = 0, sy = 0, syy = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double x = Xt[i * kStride + j], y = j < nf ? Yt[i * kStride + j] : 0.0;
        sx += x;
        sxx += x * x;
        sy += y;
        syy += y * y;
    }
    const double mx = sx / n, my = sy / n;
    const double vx = fmax(sxx / n - mx * mx, 0.0), vy = fmax(syy / n - my * my, 0.0);
    mu[j] = (float)mx;
    nu[j] = (float)my;
    sd[j] = (float)fmax(sqrt(vx), kSdFloor);
    colvar[j] = (float)vy;
}

__global__ void scale_kernel(const float *colvar, int nf, float *td)
{
    double acc = 0.0;
    for (int j = 0; j < nf; ++j) acc += colvar[j];
    const float t = (float)(acc > 0 ? sqrt(acc / nf) : 1.0);
    for (int j = 0; j < kStride; ++j) td[j] = t;
}

// per-sample weights 1 / (|y_b|^2 / nf), then normalised to mean 1 by the caller's second pass
__global__ void rowweight_kernel(const float *Yt, int64_t n, int nf, float *rw)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int j = 0; j < nf; ++j) acc += (double)Yt[i * kStride + j] * Yt[i * kStride + j];
    rw[i] = (float)(1.0 / (acc / nf + 1e-30));
}

__global__ void rowweight_norm_kernel(int64_t n, float *rw)
{
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += rw[i];
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
        if ((int)threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    const float scale = (float)(n / red[0]);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) rw[i] *= scale;
}

// prep_kernel followed by the standardisation (x - mu) / s, (y - nu) / t in one pass: one warp per
// cell, lanes over modes
__global__ void normalize_kernel(const float *featF, const float *featQ, const double *mom, const int *kvec, int64_t n,
                                 int nmodes, int idx0, float pi_over_L, int extra, int d, const float *mu,
                                 const float *sd, const float *nu, const float *td, float *X, float *Y)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const double *mi = mom + i * EF_DIAG_STRIDE;
    float ux, uy, uz;
    cell_velocity(mi, ux, uy, uz);
    const float m = featF[i * kStride + 2 * idx0];
    for (int j = lane; j < nmodes; j += 32) {
        const float ph = pi_over_L * (kvec[3 * j] * ux + kvec[3 * j + 1] * uy + kvec[3 * j + 2] * uz);
        float sn, cs;
        sincosf(ph, &sn, &cs);
        const float fr = featF[i * kStride + 2 * j], fi = featF[i * kStride + 2 * j + 1];
        X[i * kStride + 2 * j] = ((fr * cs - fi * sn) / m - mu[2 * j]) / sd[2 * j];
        X[i * kStride + 2 * j + 1] = ((fr * sn + fi * cs) / m - mu[2 * j + 1]) / sd[2 * j + 1];
        if (featQ && Y) {
            const float qr = featQ[i * kStride + 2 * j], qi = featQ[i * kStride + 2 * j + 1];
            Y[i * kStride + 2 * j] = ((qr * cs - qi * sn) / (m * m) - nu[2 * j]) / td[2 * j];
            Y[i * kStride + 2 * j + 1] = ((qr * sn + qi * cs) / (m * m) - nu[2 * j + 1]) / td[2 * j + 1];
        }
    }
    if (extra && lane == 0) {
        float theta, kl;
        cell_theta_kl(mi, d, theta, kl);
        const int j = 2 * nmodes;
        X[i * kStride + j] = (theta - mu[j]) / sd[j];
        X[i * kStride + j + 1] = (kl - mu[j + 1]) / sd[j + 1];
    }
}

__device__ __forceinline__ float hash_unit(uint64_t seed, int64_t i)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((z >> 40) * (1.0 / 16777216.0));
}

// one warp per cell: decode, gates, audit draw, compaction of the cells that need the plain path
__global__ void decode_gate_kernel(const float *Ypred, int ldy, const float *featF, const float *featL, const double *mom,
                                   const int *kvec, float pi_over_L, int64_t n, int nf, int nin, int idx0, const float *nu,
                                   const float *td, const float *Xn, float xmax, float N3, float audit_frac, uint64_t seed,
                                   float *qfeat, int *flags, unsigned long long *count, int64_t *list_off,
                                   int64_t *list_id, int64_t cell, unsigned *audit, const float *Ycheck, float check_tol,
                                   float *score)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float m = featF[i * kStride + 2 * idx0];
    const double *mi = mom + i * EF_DIAG_STRIDE;
    float ux, uy, uz;
    cell_velocity(mi, ux, uy, uz);
    float prod = 0.f, dnum = 0.f, dden = 0.f;
    bool bad = false;
    for (int jm = lane; jm < nf / 2; jm += 32) {
        float yr = (Ypred[i * ldy + 2 * jm] * td[2 * jm] + nu[2 * jm]) * m * m;
        float yi = (Ypred[i * ldy + 2 * jm + 1] * td[2 * jm + 1] + nu[2 * jm + 1]) * m * m;
        if (Ycheck) {
            // the two networks: their disagreement in the band's own units (the decoded modes
            // differ by the same per-cell phase and scale, which the norms do not see), and their
            // mean as the prediction (an ensemble of two, more accurate than either)
            const float cr = (Ycheck[i * ldy + 2 * jm] * td[2 * jm] + nu[2 * jm]) * m * m;
            const float ci = (Ycheck[i * ldy + 2 * jm + 1] * td[2 * jm + 1] + nu[2 * jm + 1]) * m * m;
            yr = 0.5f * (yr + cr);
            yi = 0.5f * (yi + ci);
            if (jm != idx0) {
                dnum += 4.f * ((yr - cr) * (yr - cr) + (yi - ci) * (yi - ci));
                dden += yr * yr + yi * yi;
            }
        }
        const float ph = pi_over_L * (kvec[3 * jm] * ux + kvec[3 * jm + 1] * uy + kvec[3 * jm + 2] * uz);
        float sn, cs;
        sincosf(ph, &sn, &cs);
        float qr = yr * cs + yi * sn, qi = yi * cs - yr * sn;      // times exp(-i ph)
        if (jm == idx0) qr = qi = 0.f;                             // Qh_0 = 0
        if (!isfinite(qr) || !isfinite(qi)) bad = true;
        if (fabsf(Xn[i * kStride + 2 * jm]) > xmax || fabsf(Xn[i * kStride + 2 * jm + 1]) > xmax) bad = true;
        qfeat[i * kStride + 2 * jm] = qr;
        qfeat[i * kStride + 2 * jm + 1] = qi;
        if (featL) prod += qr * featL[i * kStride + 2 * jm] + qi * featL[i * kStride + 2 * jm + 1];   // Re(q conj(l))
    }
    if (lane == 0)
        for (int j = nf; j < nin; ++j)
            if (fabsf(Xn[i * kStride + j]) > xmax) bad = true;
    for (int o = 16; o > 0; o >>= 1) {
        prod += __shfl_xor_sync(0xffffffffu, prod, o);
        dnum += __shfl_xor_sync(0xffffffffu, dnum, o);
        dden += __shfl_xor_sync(0xffffffffu, dden, o);
        bad |= __shfl_xor_sync(0xffffffffu, (int)bad, o) != 0;
    }
    if (lane == 0) {
        prod *= 2.f * N3;
        int f = 0;
        if (bad || !(prod <= 0.f)) f |= 1;
        const float dis = Ycheck ? sqrtf(dnum / fmaxf(dden, 1e-30f)) : 0.f;
        if (score) score[i] = dis;
        if (Ycheck && !(dis <= check_tol)) f |= 32;          // the checker disagrees: plain operator
        if (hash_unit(seed, i) < audit_frac) {
            f |= 2;
            atomicAdd(&audit[0], 1u);
        }
        flags[i] = f;
        if (f) {
            const unsigned long long k = atomicAdd(count, 1ULL);
            list_off[k] = i * cell;
            list_id[k] = i;
        }
    }
}

// merge the plain band of the listed cells into the output; audited cells compare first
__global__ void merge_kernel(const unsigned long long *count, const int64_t *list_id, const float *qplain, float *qfeat, int nf,
                             float tol, int *flags, unsigned *audit)
{
    const int lane = threadIdx.x & 31;
    const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (k >= *count) return;
    const int64_t i = list_id[k];
    const int f = flags[i];
    float num = 0.f, den = 0.f;
    for (int j = lane; j < nf; j += 32) {
        const float p = qplain[i * kStride + j];
        const float d = qfeat[i * kStride + j] - p;
        num += d * d;
        den += p * p;
        qfeat[i * kStride + j] = p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        int nf2 = f | 8;                                  // plain result used
        if ((f & 2) && num > tol * tol * den) {
            nf2 |= 4;
            atomicAdd(&audit[1], 1u);
        }
        flags[i] = nf2;
    }
}

// second round: when more than max_miss of the audited cells missed the tolerance (any miss when
// max_miss = 0), list every cell that still carries a prediction
__global__ void relist_kernel(const unsigned *audit, float max_miss, int64_t n, int *flags, unsigned long long *count,
                              int64_t *list_off, int64_t *list_id, int64_t cell)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned audited = audit[0], missed = audit[1];
    if (!(missed > 0 && (float)missed > max_miss * (float)audited)) return;
    if (flags[i] & 8) return;
    flags[i] |= 16;                                       // fell back because the batch was untrusted
    const unsigned long long k = atomicAdd(count, 1ULL);
    list_off[k] = i * cell;
    list_id[k] = i;
}

// Q on the grid from the band: Q[i] = sum over the band (both halves) of q_k exp(2 pi i k.i / N), the
// inverse of ef_features' transform on the band (index-origin convention).  Q is real and
// q_{-k} = conj(q_k), so only the half k2 >= 0 of the band enters (the k2 = 0 plane with both of its
// halves), evaluated separably:
//   A[z][k1][k2] = sum_k0 c[k0][k1][k2] exp(2 pi i k0 z / N)          (one shared-memory pass)
//   B_k2(z, y)   = sum_k1 A[z][k1][k2] exp(2 pi i k1 y / N)           (per row, in registers)
//   Q[z][y][x]   = Re B_0 + 2 Re sum_{k2 >= 1} B_k2 exp(2 pi i k2 x / N)  (compile-time twiddles)
// Rows y and N - y share their sums (with P = sum_k1 A cos, R = sum_k1 A sin: B(y) = P + iR,
// B(N - y) = P - iR), and so do the columns x and N - x of a row; one thread takes such a pair of
// rows (y = 0 with y = N/2).  The rows of a chunk of planes are staged in shared memory and written
// out with coalesced 16-byte stores.  One CTA of 256 threads per cell at a time (persistent over
// cells).  Cells whose flags carry 8 (plain operator used) are skipped: the fallback launch wrote
// their Q on the grid itself.  (A three-pass FFT of the zero-padded band has a third of the
// instructions and measured slower: the pass is bound by latency, not by arithmetic.)
constexpr int kBandK = EF_FEATURE_K, kBandW = 2 * EF_FEATURE_K + 1, kBandH = EF_FEATURE_K + 1;

// output planes staged per pass: the largest divisor of N up to 512 / N (about 256 row pairs)
template <int N>
__host__ __device__ constexpr int band_pz()
{
    int p = 512 / N < N ? 512 / N : N;
    while (N % p) --p;
    return p;
}
template <int N>
constexpr size_t band_grid_smem()
{
    return (size_t)band_pz<N>() * N * N * 4 + (size_t)(kBandW * kBandW * kBandH + N * kBandW * kBandH + N) * 8;
}
// position of 16-byte piece j of staged row y: rows of one warp's stores (consecutive y) start on
// different banks (XOR for a power-of-two count of pieces, else a rotation)
template <int N>
__device__ __forceinline__ int band_swz(int j, int y)
{
    constexpr int NC = N / 4;
    if constexpr ((NC & (NC - 1)) == 0) return j ^ (y & (NC < 8 ? NC - 1 : 7));
    else return (j + y) % NC;
}

// one output row from its B_k2, k2 = 0 .. K: out[x] = Re B_0 + 2 Re sum_k2 B_k2 exp(2 pi i k2 x / N),
// into staged row y (float4 pieces, swizzled)
template <int N>
__device__ __forceinline__ void band_row_out(const float2 (&B)[kBandH], float4 *rowbuf, int y)
{
    float out[N];
    float c0 = 0.f, ch = 0.f;                               // x = 0 and x = N/2
#pragma unroll
    for (int k2 = 1; k2 < kBandH; ++k2) {
        c0 += B[k2].x;
        ch += (k2 & 1) ? -B[k2].x : B[k2].x;
    }
    out[0] = B[0].x + 2.f * c0;
    out[N / 2] = B[0].x + 2.f * ch;
#pragma unroll
    for (int x = 1; x < N / 2; ++x) {
        float cs = 0.f, sn = 0.f;
#pragma unroll
        for (int k2 = 1; k2 < kBandH; ++k2) {
            const ef::C2<float> t = ef::tw_value<N, float>((k2 * x) % N);   // (cos, -sin) of 2 pi k2 x / N
            cs += B[k2].x * t.x;
            sn += B[k2].y * t.y;                                             // -b sin
        }
        out[x] = B[0].x + 2.f * (cs + sn);                  // Re(B w) = a cos - b sin
        out[N - x] = B[0].x + 2.f * (cs - sn);
    }
#pragma unroll
    for (int x = 0; x < N; x += 4) rowbuf[band_swz<N>(x / 4, y)] = make_float4(out[x], out[x + 1], out[x + 2], out[x + 3]);
}

template <int N>
__global__ void __launch_bounds__(256) band_to_grid_kernel(const float *qfeat, const int *kvec, int nmodes, const int *flags,
                                                           float *Q, int64_t n)
{
    constexpr int PZ = band_pz<N>(), NC = N / 4;
    extern __shared__ __align__(16) float4 bsm4[];
    float4 *ob = bsm4;                                                                             // [PZ][N rows][N/4]
    float2 *bsm = reinterpret_cast<float2 *>(bsm4 + PZ * N * NC);
    auto cf = reinterpret_cast<float2 (*)[kBandW][kBandH]>(bsm);                                   // [k0][k1][k2 >= 0]
    auto A = reinterpret_cast<float2 (*)[kBandW][kBandH]>(bsm + kBandW * kBandW * kBandH);          // [z][k1][k2]
    float2 *ex = bsm + kBandW * kBandW * kBandH + N * kBandW * kBandH;                             // exp(2 pi i m / N)
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int m = tid; m < N; m += nt) {
        float sn, cs;
        sincospif(2.0f * (float)m / (float)N, &sn, &cs);
        ex[m] = make_float2(cs, sn);
    }
    constexpr int64_t CELL = (int64_t)N * N * N;
    constexpr int NA = N * kBandW * kBandH;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        if (flags && (flags[i] & 8)) continue;             // uniform over the CTA
        __syncthreads();                                    // the previous cell's A and cf reads are done
        for (int t = tid; t < kBandW * kBandW * kBandH; t += nt) (&cf[0][0][0])[t] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int j = tid; j < nmodes; j += nt) {
            const int k0 = kvec[3 * j], k1 = kvec[3 * j + 1], k2 = kvec[3 * j + 2];
            const float re = qfeat[i * kStride + 2 * j], im = qfeat[i * kStride + 2 * j + 1];
            if (k2 > 0) {
                cf[k0 + kBandK][k1 + kBandK][k2] = make_float2(re, im);
            } else if (k2 == 0) {                           // both halves of the k2 = 0 plane
                cf[k0 + kBandK][k1 + kBandK][0] = make_float2(re, im);
                if (k0 || k1) cf[kBandK - k0][kBandK - k1][0] = make_float2(re, -im);
            } else {                                        // a stored mode of the other half: its conjugate
                cf[kBandK - k0][kBandK - k1][-k2] = make_float2(re, -im);
            }
        }
        __syncthreads();
        for (int o = tid; o < NA; o += nt) {
            const int z = o / (kBandW * kBandH), r = o % (kBandW * kBandH);
            const int k1 = r / kBandH, k2 = r % kBandH;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k0 = 0; k0 < kBandW; ++k0) {
                const float2 c = cf[k0][k1][k2];
                const float2 e = ex[(((k0 - kBandK) * z) % N + N) % N];
                acc.x += c.x * e.x - c.y * e.y;
                acc.y += c.x * e.y + c.y * e.x;
            }
            A[z][k1][k2] = acc;
        }
        __syncthreads();
        float4 *Qi = reinterpret_cast<float4 *>(Q + i * CELL);
        for (int z0 = 0; z0 < N; z0 += PZ) {
            for (int item = tid; item < PZ * (N / 2); item += nt) {
                const int zl = item / (N / 2), p = item % (N / 2), z = z0 + zl;
                float4 *pl = ob + zl * N * NC;
                float2 P[kBandH], R[kBandH];
#pragma unroll
                for (int k2 = 0; k2 < kBandH; ++k2) {
                    P[k2] = A[z][kBandK][k2];
                    R[k2] = make_float2(0.f, 0.f);
                }
                if (p == 0) {
                    // rows y = 0 (every exp = 1) and y = N/2 (exp = (-1)^k1): R = 0 for both
                    float2 Ph[kBandH];
#pragma unroll
                    for (int k2 = 0; k2 < kBandH; ++k2) Ph[k2] = P[k2];
#pragma unroll
                    for (int m = 1; m <= kBandK; ++m) {
#pragma unroll
                        for (int k2 = 0; k2 < kBandH; ++k2) {
                            const float2 u = A[z][kBandK + m][k2], v = A[z][kBandK - m][k2];
                            const float sx = u.x + v.x, sy = u.y + v.y;
                            P[k2].x += sx;
                            P[k2].y += sy;
                            Ph[k2].x += (m & 1) ? -sx : sx;
                            Ph[k2].y += (m & 1) ? -sy : sy;
                        }
                    }
                    band_row_out<N>(P, pl, 0);
                    band_row_out<N>(Ph, pl + (N / 2) * NC, N / 2);
                } else {
                    const float2 w = ex[p];
                    float2 e = w;                           // exp(2 pi i m p / N), m = 1 .. K
#pragma unroll
                    for (int m = 1; m <= kBandK; ++m) {
#pragma unroll
                        for (int k2 = 0; k2 < kBandH; ++k2) {
                            const float2 u = A[z][kBandK + m][k2], v = A[z][kBandK - m][k2];
                            P[k2].x += (u.x + v.x) * e.x;
                            P[k2].y += (u.y + v.y) * e.x;
                            R[k2].x += (u.x - v.x) * e.y;
                            R[k2].y += (u.y - v.y) * e.y;
                        }
                        e = make_float2(e.x * w.x - e.y * w.y, e.x * w.y + e.y * w.x);
                    }
                    float2 B[kBandH];
#pragma unroll
                    for (int k2 = 0; k2 < kBandH; ++k2) B[k2] = make_float2(P[k2].x - R[k2].y, P[k2].y + R[k2].x);   // P + iR
                    band_row_out<N>(B, pl + p * NC, p);
#pragma unroll
                    for (int k2 = 0; k2 < kBandH; ++k2) B[k2] = make_float2(P[k2].x + R[k2].y, P[k2].y - R[k2].x);   // P - iR
                    band_row_out<N>(B, pl + (N - p) * NC, N - p);
                }
            }
            __syncthreads();
            // the chunk's planes, contiguous in Q: coalesced 16-byte stores
            for (int c = tid; c < PZ * N * NC; c += nt) {
                const int row = c / NC, j = c % NC;
                Qi[(int64_t)z0 * N * NC + c] = ob[row * NC + band_swz<N>(j, row % N)];
            }
            __syncthreads();
        }
    }
}

template <int N>
cudaError_t band_to_grid_n(const float *qfeat, const int *kvec, int nmodes, const int *flags, float *Q, int64_t n,
                           cudaStream_t st)
{
    // per device: the shared-memory attribute and the persistent grid (resident CTAs on every SM)
    static int grid_of[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int full = dev < 64 ? grid_of[dev] : 0;
    if (full == 0) {
        cudaError_t e = cudaFuncSetAttribute(band_to_grid_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)band_grid_smem<N>());
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, band_to_grid_kernel<N>, 256, band_grid_smem<N>());
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        full = std::max(1, per_sm) * sms;
        if (dev < 64) grid_of[dev] = full;
    }
    const int grid = (int)std::min<int64_t>(n, full);
    band_to_grid_kernel<N><<<grid, 256, band_grid_smem<N>(), st>>>(qfeat, kvec, nmodes, flags, Q, n);
    return cudaGetLastError();
}

cudaError_t band_to_grid(int N, const float *qfeat, const int *kvec, int nmodes, const int *flags, float *Q, int64_t n,
                         cudaStream_t st)
{
    switch (N) {
    case 16: return band_to_grid_n<16>(qfeat, kvec, nmodes, flags, Q, n, st);
    case 24: return band_to_grid_n<24>(qfeat, kvec, nmodes, flags, Q, n, st);
    case 32: return band_to_grid_n<32>(qfeat, kvec, nmodes, flags, Q, n, st);
    case 40: return band_to_grid_n<40>(qfeat, kvec, nmodes, flags, Q, n, st);
    case 48: return band_to_grid_n<48>(qfeat, kvec, nmodes, flags, Q, n, st);
    case 64: return band_to_grid_n<64>(qfeat, kvec, nmodes, flags, Q, n, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

struct ef_surrogate_s {
    ef_plan_t plan;
    ef_mlp_t mlp;
    int64_t max_batch;
    int nf, nin, idx0, noutp, d;        // nin = nf, or nf + 2 with the two moment features
    float *mu = nullptr, *sd = nullptr, *nu = nullptr, *td = nullptr, *colvar = nullptr;
    int *kvec = nullptr;
    double *mom = nullptr;
    float pi_over_L = 0.f;
    float *featF = nullptr, *featL = nullptr, *X = nullptr, *Y = nullptr, *qplain = nullptr;
    void *Qs = nullptr;
    void *fh = nullptr;                   // forward-spectrum workspace of the fallback collide launches
    unsigned *audit = nullptr;            // [0] audited cells, [1] audited misses (this call)
    unsigned long long *count = nullptr;
    int64_t *list_off = nullptr, *list_id = nullptr;
    float xmax = 8.f;
    float max_miss = 0.f;
    ef_mlp_t checker = nullptr;           // second network; its disagreement gates cells (nullable)
    float check_tol = 0.f;
    float *Yc = nullptr;                  // checker outputs (max_batch rows)
    bool entropy_gate = true;             // the band entropy-production gate (needs the band of ln F)
};

namespace {

void sur_free(ef_surrogate_s *s)
{
    if (!s) return;
    cudaFree(s->mu);
    cudaFree(s->sd);
    cudaFree(s->nu);
    cudaFree(s->td);
    cudaFree(s->colvar);
    cudaFree(s->kvec);
    cudaFree(s->mom);
    cudaFree(s->featF);
    cudaFree(s->featL);
    cudaFree(s->X);
    cudaFree(s->Y);
    cudaFree(s->qplain);
    cudaFree(s->Qs);
    cudaFree(s->Yc);
    cudaFree(s->fh);
    cudaFree(s->audit);
    cudaFree(s->count);
    cudaFree(s->list_off);
    cudaFree(s->list_id);
    delete s;
}

// the feature modes in ef_features order (canonical half, K = EF_FEATURE_K); returns the slot of 0
int mode_list(int d, std::vector<int> &kv)
{
    const int K = EF_FEATURE_K;
    int zero = -1;
    kv.clear();
    for (int k0 = -K; k0 <= K; ++k0)
        for (int k1 = -K; k1 <= K; ++k1)
            for (int k2 = 0; k2 <= K; ++k2) {
                if (k0 * k0 + k1 * k1 + k2 * k2 > K * K) continue;
                if (!(k2 > 0 || (k2 == 0 && (k1 > 0 || (k1 == 0 && k0 >= 0))))) continue;
                if (d == 2 && (k2 != 0 || k1 < 0)) continue;
                if (k0 == 0 && k1 == 0 && k2 == 0) zero = (int)kv.size() / 3;
                kv.push_back(k0);
                kv.push_back(k1);
                kv.push_back(k2);
            }
    return zero;
}

}  // namespace

extern "C" {

ef_status ef_surrogate_create(ef_plan_t plan, ef_mlp_t mlp, int64_t max_batch, ef_surrogate_t *out)
{
    if (!out) return sfail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    ef::PlanView v;
    if (!ef::plan_view(plan, &v)) return sfail(EF_ERR_INVALID_ARG, "surrogate needs a uniform plan");
    if (!mlp) return sfail(EF_ERR_INVALID_ARG, "null mlp");
    if (v.nfeat == 0) return sfail(EF_ERR_UNSUPPORTED, "N too small for the feature band");
    if (v.sg_global) return sfail(EF_ERR_UNSUPPORTED, "surrogate fallback needs a shared-memory accumulator shape");
    int64_t info[8];
    ef_status st = ef_mlp_info(mlp, info);
    if (st != EF_OK) return st;
    const int nf = 2 * v.nfeat;
    if ((info[0] != nf && info[0] != nf + 2) || info[3] != nf)
        return sfail(EF_ERR_INVALID_ARG, "mlp widths: input 2 x feature modes (+ 2 moment features), output 2 x feature modes");
    if (max_batch < 64 || max_batch % 64 || max_batch > info[7])
        return sfail(EF_ERR_INVALID_ARG, "max_batch: multiple of 64, at most the mlp's max batch");
    ef_surrogate_s *s = new ef_surrogate_s();
    s->plan = plan;
    s->mlp = mlp;
    s->max_batch = max_batch;
    s->nf = nf;
    s->nin = (int)info[0];
    s->d = v.d;
    s->noutp = (int)info[6];
    std::vector<int> kv;
    s->idx0 = mode_list(v.d, kv);
    s->pi_over_L = (float)(3.14159265358979323846 / v.L);
    const int64_t cell = v.d == 3 ? (int64_t)v.N * v.N * v.N : (int64_t)v.N * v.N;
    const size_t el = v.prec == EF_PREC_F32 ? 4 : 8;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(p, b);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, b);
    };
    alloc((void **)&s->mu, kStride * 4);
    alloc((void **)&s->sd, kStride * 4);
    alloc((void **)&s->nu, kStride * 4);
    alloc((void **)&s->td, kStride * 4);
    alloc((void **)&s->colvar, kStride * 4);
    alloc((void **)&s->kvec, kv.size() * 4);
    alloc((void **)&s->mom, (size_t)max_batch * EF_DIAG_STRIDE * 8);
    alloc((void **)&s->featF, (size_t)max_batch * kStride * 4);
    alloc((void **)&s->featL, (size_t)max_batch * kStride * 4);
    alloc((void **)&s->X, (size_t)max_batch * kStride * 4);
    alloc((void **)&s->Y, (size_t)max_batch * s->noutp * 4);
    alloc((void **)&s->qplain, (size_t)max_batch * kStride * 4);
    alloc((void **)&s->Qs, (size_t)max_batch * cell * el);
    alloc((void **)&s->fh, (size_t)v.max_clusters * ef::collide_fh_bytes(v.prec, v.d, v.N));
    alloc((void **)&s->audit, 8);
    alloc((void **)&s->count, 8);
    alloc((void **)&s->list_off, (size_t)max_batch * 8);
    alloc((void **)&s->list_id, (size_t)max_batch * 8);
    if (e != cudaSuccess) {
        sur_free(s);
        return scuda(e, "surrogate allocation");
    }
    if (e == cudaSuccess) e = cudaMemcpy(s->kvec, kv.data(), kv.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        sur_free(s);
        return scuda(e, "surrogate mode table");
    }
    // identity normalisation until fitted
    std::vector<float> one(kStride, 1.f);
    cudaMemcpy(s->sd, one.data(), kStride * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(s->td, one.data(), kStride * 4, cudaMemcpyHostToDevice);
    *out = s;
    return EF_OK;
}

ef_status ef_surrogate_destroy(ef_surrogate_t s)
{
    if (!s) return sfail(EF_ERR_INVALID_ARG, "null surrogate");
    sur_free(s);
    return EF_OK;
}

ef_status ef_surrogate_fit_stats(ef_surrogate_t s, const float *featF, const float *featQ, const double *mom, float *Xt,
                                 float *Yt, float *rowweight, int64_t n, ef_stream_t stream)
{
    if (!s || !featF || !featQ || !mom || !Xt || !Yt || n <= 0) return sfail(EF_ERR_INVALID_ARG, "bad surrogate statistics arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int nm = s->nf / 2;
    prep_kernel<<<sgrid(n * nm), 256, 0, st>>>(featF, featQ, mom, s->kvec, n, nm, s->idx0, s->pi_over_L, s->nin > s->nf,
                                               s->d, Xt, Yt);
    stats_kernel<<<(s->nin + 127) / 128, 128, 0, st>>>(Xt, Yt, n, s->nin, s->nf, s->mu, s->sd, s->nu, s->colvar);
    scale_kernel<<<1, 1, 0, st>>>(s->colvar, s->nf, s->td);
    if (rowweight) {
        rowweight_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Yt, n, s->nf, rowweight);
        rowweight_norm_kernel<<<1, 256, 0, st>>>(n, rowweight);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : scuda(e, "stats");
}

ef_status ef_surrogate_normalize(ef_surrogate_t s, const float *featF, const float *featQ, const double *mom, float *X,
                                 float *Y, int64_t n, ef_stream_t stream)
{
    if (!s || !featF || !mom || !X || n < 0) return sfail(EF_ERR_INVALID_ARG, "bad normalisation arguments");
    if (n == 0) return EF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int nm = s->nf / 2;
    const bool withY = featQ && Y;
    normalize_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(featF, withY ? featQ : nullptr, mom, s->kvec, n, nm, s->idx0,
                                                              s->pi_over_L, s->nin > s->nf, s->d, s->mu, s->sd, s->nu,
                                                              s->td, X, withY ? Y : nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : scuda(e, "normalise");
}

ef_status ef_surrogate_stats(ef_surrogate_t s, float *host4, int set)
{
    if (!s || !host4) return sfail(EF_ERR_INVALID_ARG, "null surrogate or buffer");
    float *d[4] = {s->mu, s->sd, s->nu, s->td};
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = set ? cudaMemcpy(d[k], host4 + k * kStride, kStride * 4, cudaMemcpyHostToDevice)
                            : cudaMemcpy(host4 + k * kStride, d[k], kStride * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return scuda(e, "surrogate stats copy");
    }
    return EF_OK;
}

ef_status ef_surrogate_set_policy(ef_surrogate_t s, float max_miss_fraction, float xmax)
{
    if (!s) return sfail(EF_ERR_INVALID_ARG, "null surrogate");
    if (!(max_miss_fraction >= 0.f && max_miss_fraction <= 1.f)) return sfail(EF_ERR_INVALID_ARG, "max_miss_fraction in [0, 1]");
    if (!(xmax > 0.f)) return sfail(EF_ERR_INVALID_ARG, "xmax > 0");
    s->max_miss = max_miss_fraction;
    s->xmax = xmax;
    return EF_OK;
}

ef_status ef_surrogate_set_entropy_gate(ef_surrogate_t s, int on)
{
    if (!s) return sfail(EF_ERR_INVALID_ARG, "null surrogate");
    s->entropy_gate = on != 0;
    return EF_OK;
}

ef_status ef_features_inverse(ef_plan_t plan, const float *feat, float *Q_dev, int64_t ncells, ef_stream_t stream)
{
    ef::PlanView v;
    if (!ef::plan_view(plan, &v)) return sfail(EF_ERR_INVALID_ARG, "ef_features_inverse: needs a uniform plan");
    if (v.prec != EF_PREC_F32 || v.d != 3 || v.nfeat == 0) return sfail(EF_ERR_UNSUPPORTED, "ef_features_inverse: FP32 3D plans with a band");
    if (ncells < 0) return sfail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (ncells == 0) return EF_OK;
    if (!feat || !Q_dev || (uintptr_t)Q_dev % 16) return sfail(EF_ERR_INVALID_ARG, "null feat or Q, or Q not 16-byte aligned");
    const cudaError_t e = band_to_grid(v.N, feat, v.modes, v.nfeat, nullptr, Q_dev, ncells, (cudaStream_t)stream);
    return e == cudaSuccess ? EF_OK : scuda(e, "ef_features_inverse");
}

ef_status ef_surrogate_set_checker(ef_surrogate_t s, ef_mlp_t checker, float tol)
{
    if (!s) return sfail(EF_ERR_INVALID_ARG, "null surrogate");
    if (checker) {
        int64_t a[8], b[8];
        ef_status st = ef_mlp_info(s->mlp, a);
        if (st == EF_OK) st = ef_mlp_info(checker, b);
        if (st != EF_OK) return st;
        if (a[0] != b[0] || a[3] != b[3] || b[7] < s->max_batch)
            return sfail(EF_ERR_INVALID_ARG, "checker: same inputs and outputs as the surrogate's network, max batch >= the surrogate's");
        if (!(tol > 0.f)) return sfail(EF_ERR_INVALID_ARG, "checker tolerance must be > 0");
        if (!s->Yc) {
            cudaError_t e = cudaMalloc((void **)&s->Yc, (size_t)s->max_batch * s->noutp * 4);
            if (e != cudaSuccess) { s->Yc = nullptr; return scuda(e, "checker outputs"); }
        }
    }
    s->checker = checker;
    s->check_tol = tol;
    return EF_OK;
}

ef_status ef_surrogate_infer(ef_surrogate_t s, const void *F, float *qfeat, int *flags, int64_t ncells, float audit_fraction,
                             uint64_t seed, float tol, ef_stream_t stream)
{
    return ef_surrogate_infer_ex(s, F, qfeat, flags, nullptr, nullptr, ncells, audit_fraction, seed, tol, stream);
}

ef_status ef_surrogate_infer_ex(ef_surrogate_t s, const void *F, float *qfeat, int *flags, float *score, float *Q,
                                int64_t ncells, float audit_fraction, uint64_t seed, float tol, ef_stream_t stream)
{
    if (!s || !F || !qfeat || !flags) return sfail(EF_ERR_INVALID_ARG, "null argument");
    if (ncells < 0 || ncells > s->max_batch || ncells % 64) return sfail(EF_ERR_INVALID_ARG, "ncells: multiple of 64, <= max_batch");
    if (ncells == 0) return EF_OK;
    if (!(audit_fraction >= 0.f && audit_fraction <= 1.f) || !(tol > 0.f)) return sfail(EF_ERR_INVALID_ARG, "bad audit fraction or tolerance");
    ef::PlanView v;
    if (!ef::plan_view(s->plan, &v)) return sfail(EF_ERR_INVALID_ARG, "bad plan");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t cell = v.d == 3 ? (int64_t)v.N * v.N * v.N : (int64_t)v.N * v.N;
    if ((uintptr_t)F % 16) return sfail(EF_ERR_INVALID_ARG, "F must be 16-byte aligned");
    // one pass over the cells: band modes of F (and of ln F for the entropy gate), and the moments of F
    ef::FeatArgs fa{};
    fa.F = F;
    fa.ncells = ncells;
    fa.feat = s->featF;
    fa.featL = s->entropy_gate ? s->featL : nullptr;
    fa.fstride = kStride;
    fa.mom = s->mom;
    fa.h = 2.0 * v.L / v.N;
    fa.modes = v.modes;
    fa.nmodes = v.nfeat;
    cudaError_t e = ef::features_launch(v.prec, v.d, v.N, fa, st);
    if (e != cudaSuccess) return scuda(e, "surrogate features");
    ef_status r = ef_surrogate_normalize(s, s->featF, nullptr, s->mom, s->X, nullptr, ncells, stream);
    if (r != EF_OK) return r;
    r = ef_mlp_forward(s->mlp, s->X, kStride, s->Y, s->noutp, ncells, stream);
    if (r != EF_OK) return r;
    if (s->checker) {
        r = ef_mlp_forward(s->checker, s->X, kStride, s->Yc, s->noutp, ncells, stream);
        if (r != EF_OK) return r;
    }
    if (Q && (v.prec != EF_PREC_F32 || v.d != 3 || (uintptr_t)Q % 16)) return sfail(EF_ERR_UNSUPPORTED, "Q on the grid: FP32 3D plans, 16-byte aligned Q");
    e = cudaMemsetAsync(s->count, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->audit, 0, 8, st);
    if (e != cudaSuccess) return scuda(e, "surrogate reset");
    decode_gate_kernel<<<(unsigned)((ncells * 32 + 255) / 256), 256, 0, st>>>(
        s->Y, s->noutp, s->featF, s->entropy_gate ? s->featL : nullptr, s->mom, s->kvec, s->pi_over_L, ncells, s->nf, s->nin, s->idx0, s->nu, s->td, s->X,
        s->xmax, (float)cell,
        audit_fraction, seed, qfeat, flags, s->count, s->list_off, s->list_id, cell, s->audit,
        s->checker ? s->Yc : nullptr, s->check_tol, score);
    for (int round = 0; round < 2; ++round) {
        // plain operator on the listed cells (count read on the device), then their band; with Q on
        // the grid requested the plain operator writes the listed cells' Q there directly
        ef::CollideArgs a{};
        a.F = F;
        a.Q = Q ? static_cast<void *>(Q) : s->Qs;
        a.cell_off = s->list_off;
        a.cell_id = s->list_id;
        a.ncells = ncells;
        a.dev_ncells = reinterpret_cast<const long long *>(s->count);
        a.mult = v.mult;
        a.ops = v.ops;
        a.nops = v.nops;
        a.cluster = v.cluster;
        a.planes = v.planes;
        a.paired = v.paired;
        a.fh_ws = s->fh;
        a.npc = ef::collide_npc_v(v.d, v.N, v.cluster, v.occ);
        a.out_mode = ef::OUT_COLLIDE;
        a.h = 2.0 * v.L / v.N;
        a.status = v.status;
        const int grid = (int)std::min<int64_t>(ncells, v.max_clusters);
        e = ef::collide_launch(v.prec, v.d, v.N, a, grid, v.tpb, v.smem, v.occ, st);
        if (e != cudaSuccess) return scuda(e, "fallback collide");
        ef::FeatArgs qa{};
        qa.F = a.Q;
        qa.cell_off = s->list_off;
        qa.cell_id = s->list_id;
        qa.ncells = ncells;
        qa.dev_ncells = s->count;
        qa.feat = s->qplain;
        qa.fstride = kStride;
        qa.h = 2.0 * v.L / v.N;
        qa.modes = v.modes;
        qa.nmodes = v.nfeat;
        e = ef::features_launch(v.prec, v.d, v.N, qa, st);
        if (e != cudaSuccess) return scuda(e, "fallback features");
        merge_kernel<<<(unsigned)((ncells * 32 + 255) / 256), 256, 0, st>>>(s->count, s->list_id, s->qplain, qfeat, s->nf,
                                                                            tol, flags, s->audit);
        if (round == 0) {
            e = cudaMemsetAsync(s->count, 0, 8, st);
            if (e != cudaSuccess) return scuda(e, "surrogate reset");
            relist_kernel<<<(unsigned)((ncells + 255) / 256), 256, 0, st>>>(s->audit, s->max_miss, ncells, flags,
                                                                            s->count, s->list_off, s->list_id, cell);
        }
    }
    if (Q) {
        e = band_to_grid(v.N, qfeat, s->kvec, s->nf / 2, flags, Q, ncells, st);
        if (e != cudaSuccess) return scuda(e, "band to grid");
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : scuda(e, "surrogate infer");
}

}  // extern "C"
