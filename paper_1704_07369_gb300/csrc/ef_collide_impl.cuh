// ef_collide_impl.cuh -- the fused EFM collision kernel (one thread-block cluster per cell).
//
// Per cell (Sec. 4.1, eq. fastAlg; the DVM form eq. Qsr evaluated by collocation, Sec. 3.1):
//   F1  each CTA of the cluster owns N/C planes of axis 0; it transforms its planes along the
//       last axis (real -> half complex) and, in 3D, along axis 1, into its shared-memory slab.
//   F2  CTA r owns the axis-0 pencils (spectral columns p) [r npc, (r + 1) npc); a thread per
//       pencil gathers it from the slabs of all CTAs through distributed shared memory, finishes
//       the forward transform along axis 0 and stores Fhat[:, p] to the cluster's L2-resident
//       workspace (registers stay free for the transforms).
//   for each op (one spectral direction u, or the loss; paired ops two directions):
//     A  a thread per (direction, pencil): Fhat[:, p] * M_u[:, p] (filter and radial kernel
//        factor, L2-resident table), inverse transform along axis 0, scatter the result to the
//        owning CTAs' slabs (DSMEM stores).
//     B  each CTA finishes the inverse transform of its planes (axis 1, then half complex ->
//        real along the last axis, two rows per thread) and folds the real-space values into the
//        S / G accumulators, or, for the loss op, forms Q = G - F nu and writes the output
//        (Q, or F + dt Q for an Euler step) with FP64 diagnostics.
// Two cluster barriers per op separate the scatter (A) from the local passes (B).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ef_fft.cuh"
#include "ef_internal.h"

namespace ef {

namespace cg = cooperative_groups;

// Threads per CTA the kernel is compiled for.  Registers are shared per SM sub-partition: 8 warps
// allow 255 per thread, 10 warps (3 on some sub-partition) 168.  The output pass (Q or F + dt Q
// with the FP64 diagnostics) holds three rows of N values; FP32 N >= 40 and FP64 keep 8 warps so
// that it does not spill (the plan-time autotuner picks smaller CTAs in any case).
template <typename T, int N>
__host__ __device__ constexpr int max_threads() { return (sizeof(T) == 8 || N >= 40) ? 256 : 320; }

// Second instantiation for two co-resident CTAs per SM (of different cells, whose barrier phases
// then overlap): at most 6 warps per CTA, so 12 per SM and 168 registers per thread.  Built for
// the FP32 3D sizes of the batched workload; the autotuner chooses between the two.
constexpr int kOcc2Threads = 192;
template <typename T, int D, int N>
__host__ __device__ constexpr bool occ2_built()
{
    return sizeof(T) == 4 && D == 3 && (N == 24 || N == 32 || N == 40 || N == 48);
}

// ln f of the diagnostic sums (entropy F ln F and production Q ln F, f > 0).  FP32: the hardware
// log2 approximation times ln 2 (__logf, a few instructions instead of the accurate logf's
// sequence), whose error (about 2e-7 absolute on ln f) is far below the FP32 path's parity bar of
// 2e-5 max|Q| sum |ln F| on the production sum.
template <typename T>
__device__ __forceinline__ T log_t(T x);
template <>
__device__ __forceinline__ float log_t<float>(float x) { return __logf(x); }
template <>
__device__ __forceinline__ double log_t<double>(double x) { return log(x); }

// Cluster barriers.  full(): release/acquire, publishes prior (distributed) shared-memory writes.
// war(): relaxed arrive, for write-after-read protection only (every value loaded before it has
// already been consumed).  A one-CTA cluster uses the CTA barrier.
struct Sync {
    cg::cluster_group cl;
    int C;
    __device__ __forceinline__ void full()
    {
        if (C == 1) __syncthreads();
        else cl.sync();
    }
    __device__ __forceinline__ void war()
    {
        if (C == 1) {
            __syncthreads();
        } else {
            asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
            asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
        }
    }
};

__device__ __forceinline__ void record_status(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// Two Hermitian half rows R0, R1 (k = 0 .. N/2, in shared memory) -> the complex row
// z = IFFT(R0) + i IFFT(R1) (unscaled, inverse sign): the two-for-one inverse of c2r_pair, built
// straight from shared memory so that no half-spectrum copy lives in registers.
template <int N, typename T>
__device__ __forceinline__ void c2r_rows_from(const C2<T> *R0, const C2<T> *R1, C2<T> (&z)[N])
{
    z[0] = C2<T>{R0[0].x, R1[0].x};
#pragma unroll
    for (int k = 1; k < N / 2; ++k) {
        const C2<T> x0 = R0[k], x1 = R1[k];
        z[k] = C2<T>{x0.x - x1.y, x0.y + x1.x};
        z[N - k] = C2<T>{x0.x + x1.y, x1.x - x0.y};
    }
    z[N / 2] = C2<T>{R0[N / 2].x, R1[N / 2].x};
    fft<N, 1, N>(z);
}

// Row stride (complex values) of one axis-0 plane in a spectral slab.  The FP32 paired pencil
// scatter stores 16 bytes per lane, even lanes into plane z and odd lanes into plane z + 1: a
// plane stride of 8 mod 16 complex values puts the two halves of a quarter warp on different
// banks (a multiple of 16 would make every store a two-way bank conflict).
template <typename T, int D, int N>
__host__ __device__ constexpr int slab_stride()
{
    constexpr int NP = ((D == 3) ? N : 1) * (N / 2 + 1);
    if constexpr (sizeof(T) == 4 && NP % 2 == 0) return NP + ((8 - NP % 16) + 16) % 16;
    else return NP;
}

// shared-memory bytes of one CTA (must match the carve-up in the kernel).  Paired mode holds two
// spectral slabs and G; single mode one slab and S, G.
template <typename T, int D, int N>
__host__ __device__ constexpr size_t smem_bytes_for(int planes, int sg_global, int paired)
{
    constexpr int N1 = (D == 3) ? N : 1;
    size_t is = (size_t)(paired ? 2 : 1) * planes * slab_stride<T, D, N>() * sizeof(C2<T>);
    size_t sg = sg_global ? 0 : (size_t)(paired ? 1 : 2) * planes * N1 * N * sizeof(T);
    sg = (sg + 15) / 16 * 16;
    size_t part = (32 + 1) * kDiag * sizeof(double);
    return is + sg + part + 16;             // + the cluster's current cell index and a flag
}

// Per-cell diagnostics of one thread (FP64 sums of per-row FP32/FP64 partial sums).
struct Diag {
    double sum[kDiag];
    double min_f, max_nu, min_out;
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int k = 0; k < kDiag; ++k) sum[k] = 0.0;
        min_f = 1e300;
        max_nu = -1e300;
        min_out = 1e300;
    }
    // one row's partial sums (row index jz along axis 0, jy along axis 1); moments in array-axis
    // order: [1] axis 0, [2] axis 1, [3] axis 2 (2D: [1] axis 0, [2] axis 1)
    template <int D, typename T>
    __device__ __forceinline__ void add_row(T s_m, T s_mx, T s_e2, T s_eta, T s_prod, int jz, int jy, T mn_f, T mn_out)
    {
        const double m = (double)s_m;
        sum[0] += m;
        if (D == 3) {
            sum[1] += m * jz;
            sum[2] += m * jy;
            sum[3] += (double)s_mx;
        } else {
            sum[1] += m * jz;
            sum[2] += (double)s_mx;
        }
        sum[4] += (double)s_e2 + m * ((double)jy * jy + (double)jz * jz);
        sum[5] += (double)s_eta;
        sum[6] += (double)s_prod;
        min_f = fmin(min_f, (double)mn_f);
        min_out = fmin(min_out, (double)mn_out);
    }
};

// Float-float accumulation (an unevaluated sum hi + lo of two FP32 values): Knuth's TwoSum gives
// the exact rounding error of an FP32 addition, an FMA the exact error of a product (Dekker's
// TwoProduct), so a running sum keeps about 48 significant bits in FP32 arithmetic.  The FP32 3D
// kernels accumulate their per-cell diagnostics this way and convert to FP64 once per cell: on
// GB300 the FP64 pipe runs at a small fraction of the FP32 rate.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void ff_add(FF &x, float b)
{
    float s, e;
    ff_two_sum(x.hi, b, s, e);
    x.hi = s;
    x.lo += e;
}
// x += a b with the product's rounding error kept
__device__ __forceinline__ void ff_add_prod(FF &x, float a, float b)
{
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    ff_add(x, p);
    x.lo += pe;
}
__device__ __forceinline__ FF ff_merge(FF a, FF b)
{
    float s, e;
    ff_two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    const float h = s + e;                  // renormalise (|s| >= |e|)
    return FF{h, e - (h - s)};
}
__device__ __forceinline__ double ff_value(FF x) { return (double)x.hi + (double)x.lo; }

struct DiagF {
    FF sum[7];                              // the seven sums of Diag (slots 0 - 6)
    float min_f, max_nu, min_out;
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int k = 0; k < 7; ++k) sum[k] = FF{0.f, 0.f};
        min_f = 3.0e38f;
        max_nu = -3.0e38f;
        min_out = 3.0e38f;
    }
    template <int D, typename T>
    __device__ __forceinline__ void add_row(float s_m, float s_mx, float s_e2, float s_eta, float s_prod, int jz, int jy,
                                            float mn_f, float mn_out)
    {
        static_assert(D == 3, "the float-float diagnostics serve the 3D kernels");
        ff_add(sum[0], s_m);
        ff_add_prod(sum[1], s_m, (float)jz);
        ff_add_prod(sum[2], s_m, (float)jy);
        ff_add(sum[3], s_mx);
        ff_add(sum[4], s_e2);
        ff_add_prod(sum[4], s_m, (float)(jy * jy + jz * jz));
        ff_add(sum[5], s_eta);
        ff_add(sum[6], s_prod);
        min_f = fminf(min_f, mn_f);
        min_out = fminf(min_out, mn_out);
    }
};

// Global row I/O: a row is N contiguous values starting on a 16-byte boundary (the caller's
// buffers are 16-byte aligned and every cell and row offset is a multiple of 4 values), moved with
// 16-byte vector accesses.
template <typename T, int N>
__device__ __forceinline__ void load_row(const T *src, T (&x)[N])
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

template <typename T, int N>
__device__ __forceinline__ void store_row(T *dst, const T (&x)[N])
{
    if constexpr (sizeof(T) == 4 && N % 4 == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int i = 0; i < N / 4; ++i) d4[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
    } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
        double2 *d2 = reinterpret_cast<double2 *>(dst);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) d2[i] = make_double2(x[2 * i], x[2 * i + 1]);
    } else {
#pragma unroll
        for (int n = 0; n < N; ++n) dst[n] = x[n];
    }
}

// Final output of one real row: Q = q, written as Q (collide) or F + dt Q (Euler), with the
// non-finite / positivity status checks and the diagnostic sums of the row.  nu (nullable) gives
// the point-wise collision frequency for the positivity test; otherwise nu_big says whether
// dt nu > 1 anywhere in this CTA's rows.
template <typename T, int D, int N, typename DG>
__device__ __forceinline__ void emit_row(const CollideArgs &a, const T (&fr)[N], T *Orow, T (&q)[N], const T *nu,
                                         bool nu_big, int64_t grow, DG &dg)
{
    constexpr int N1 = (D == 3) ? N : 1;
    const int jz = (int)(grow / N1) - N / 2;
    const int jy = (D == 3) ? (int)(grow % N1) - N / 2 : 0;
    T s_m = 0, s_mx = 0, s_e2 = 0, s_eta = 0, s_prod = 0;
    T mn_f = fr[0], mn_out = T(3.0e38);
    bool bad = false, neg = false;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const T f = fr[n];
        const T qv = q[n];
        T outv;
        if (a.out_mode == OUT_EULER) {
            outv = f + T(a.dt) * qv;
            const bool big = nu ? (T(a.dt) * nu[n] > T(1)) : nu_big;
            if (outv < T(0) && big) neg = true;
        } else {
            outv = qv;
        }
        q[n] = outv;
        if (!isfinite(outv)) bad = true;
        if (a.diag) {
            const T jx = T(n - N / 2);
            s_m += f;
            s_mx += f * jx;
            s_e2 += f * jx * jx;
            if (f > T(0)) {
                const T lf = log_t<T>(f);
                s_eta += f * lf;
                s_prod += qv * lf;
            }
            mn_f = f < mn_f ? f : mn_f;
            mn_out = outv < mn_out ? outv : mn_out;
        }
    }
    store_row<T, N>(Orow, q);
    if (bad) record_status(a.status, 7);     // EF_ERR_NOT_FINITE
    if (neg) record_status(a.status, 6);     // EF_ERR_POSITIVITY
    if (a.diag) dg.template add_row<D, T>(s_m, s_mx, s_e2, s_eta, s_prod, jz, jy, mn_f, mn_out);
}

// Distributed shared memory through explicit shared::cluster addresses: mapa turns this CTA's
// shared-memory address into the same offset in CTA `rank` of the cluster, and the loads / stores
// name the state space, so that they take the shared-memory path rather than the generic one.
__device__ __forceinline__ uint32_t smem_u32addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, int rank)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, C2<float> v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, C2<double> v)
{
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void ld_cluster(uint32_t a, C2<float> &v)
{
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
}
__device__ __forceinline__ void ld_cluster(uint32_t a, C2<double> &v)
{
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
}

// Stage-A scatter of one inverse-transformed axis-0 pencil into the owners' slabs.  For FP32,
// lanes 2j and 2j+1 hold the adjacent pencils p, p+1 (p even); one shuffle per z pair lets each
// lane write both pencils of one z as a single 16-byte store, halving the number of (mostly
// remote, distributed shared memory) store transactions.
// owner CTA of axis-0 index z for P planes per CTA: floor(z / P) = floor(z pm / 2^32) with the 64-bit
// multiplier pm = ceil(2^32 / P) (pm = 2^32 for P = 1), exact for 0 <= z < 2^16 and P < 2^16
__device__ __forceinline__ int plane_owner(int z, unsigned long long pm)
{
    return (int)(((unsigned long long)(unsigned)z * pm) >> 32);
}

template <typename T, int N, bool WIDE>
__device__ __forceinline__ void scatter_pencil(const C2<T> (&v)[N], C2<T> *slab, int P, unsigned long long pm, int NP, int pencil,
                                               unsigned mask)
{
    const uint32_t base = smem_u32addr(slab);
    if constexpr (WIDE) {
        const bool odd = pencil & 1;
        const int pbase = pencil & ~1;
#pragma unroll
        for (int z0 = 0; z0 < N; z0 += 2) {
            const C2<T> send = odd ? v[z0] : v[z0 + 1];
            C2<T> recv;
            recv.x = __shfl_xor_sync(mask, send.x, 1);
            recv.y = __shfl_xor_sync(mask, send.y, 1);
            const int z = odd ? z0 + 1 : z0;
            const C2<T> lo = odd ? recv : v[z0];
            const C2<T> hi = odd ? v[z0 + 1] : recv;
            const int owner = plane_owner(z, pm), zl = z - owner * P;
            const uint32_t dst = cluster_map(base + (uint32_t)((zl * NP + pbase) * sizeof(C2<T>)), owner);
            st_cluster(dst, make_float4(lo.x, lo.y, hi.x, hi.y));
        }
    } else {
#pragma unroll
        for (int z = 0; z < N; ++z) {
            const int owner = plane_owner(z, pm), zl = z - owner * P;
            st_cluster(cluster_map(base + (uint32_t)((zl * NP + pencil) * sizeof(C2<T>)), owner), v[z]);
        }
    }
}

// The matching gather (forward pass F2): 16-byte loads of both pencils of one z, one shuffle.
template <typename T, int N, bool WIDE>
__device__ __forceinline__ void gather_pencil(C2<T> (&v)[N], C2<T> *slab, int P, unsigned long long pm, int NP, int pencil,
                                              unsigned mask)
{
    const uint32_t base = smem_u32addr(slab);
    if constexpr (WIDE) {
        const bool odd = pencil & 1;
        const int pbase = pencil & ~1;
#pragma unroll
        for (int z0 = 0; z0 < N; z0 += 2) {
            const int z = odd ? z0 + 1 : z0;
            const int owner = plane_owner(z, pm), zl = z - owner * P;
            const float4 w = ld_cluster_f4(cluster_map(base + (uint32_t)((zl * NP + pbase) * sizeof(C2<T>)), owner));
            const C2<T> lo = C2<T>{w.x, w.y}, hi = C2<T>{w.z, w.w};
            const C2<T> send = odd ? lo : hi;
            C2<T> recv;
            recv.x = __shfl_xor_sync(mask, send.x, 1);
            recv.y = __shfl_xor_sync(mask, send.y, 1);
            v[z0] = odd ? recv : lo;
            v[z0 + 1] = odd ? hi : recv;
        }
    } else {
#pragma unroll
        for (int z = 0; z < N; ++z) {
            const int owner = plane_owner(z, pm), zl = z - owner * P;
            ld_cluster(cluster_map(base + (uint32_t)((zl * NP + pencil) * sizeof(C2<T>)), owner), v[z]);
        }
    }
}

template <typename T, int D, int N, int OCC = 1>
__global__ void __launch_bounds__(OCC == 1 ? max_threads<T, N>() : kOcc2Threads, OCC) collide_kernel(const CollideArgs a)
{
    constexpr int H = N / 2 + 1;
    constexpr int N1 = (D == 3) ? N : 1;
    constexpr int NP = N1 * H;         // spectral columns of one axis-0 plane = pencils
    constexpr int NPP = slab_stride<T, D, N>();   // plane stride of the slabs (padded NP)
    constexpr int64_t CELL = (int64_t)N * N1 * N;
    // 16-byte paired pencil stores need FP32 and an even pencil count (so that every slab row
    // starts on a 16-byte boundary and lane pairs hold pencil pairs)
    constexpr bool WIDE = sizeof(T) == 4 && NP % 2 == 0;

    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int P = a.planes;
    const int tid = threadIdx.x, nt = blockDim.x;
    Sync bar{cl, C};
    const int rows = P * N1;           // real rows owned by this CTA
    const int npairs = rows / 2;
    const int nbuf = a.paired ? 2 : 1;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2<T> *Is0 = reinterpret_cast<C2<T> *>(smem_raw);
    C2<T> *Is1 = Is0 + (size_t)P * NPP;                 // paired mode only
    size_t off = (size_t)nbuf * P * NPP * sizeof(C2<T>);
    T *Sb = nullptr, *Gb;
    if (a.sg_global) {
        const int64_t slot = blockIdx.x;
        T *base = reinterpret_cast<T *>(a.sg_ws) + slot * (int64_t)2 * rows * N;
        Sb = base;
        Gb = base + (int64_t)rows * N;
    } else {
        if (!a.paired) {
            Sb = reinterpret_cast<T *>(smem_raw + off);
            off += (size_t)rows * N * sizeof(T);
        }
        Gb = reinterpret_cast<T *>(smem_raw + off);
        off += (size_t)rows * N * sizeof(T);
        off = (off + 15) / 16 * 16;
    }
    double *part = reinterpret_cast<double *>(smem_raw + off);      // [32 warps + 1][kDiag]
    off += (32 + 1) * kDiag * sizeof(double);
    long long *s_cell = reinterpret_cast<long long *>(smem_raw + off);
    int *s_nubig = reinterpret_cast<int *>(smem_raw + off + 8);

    const unsigned long long pm = (0x100000000ull + (unsigned)P - 1u) / (unsigned)P;   // plane_owner's multiplier

    const int64_t nclusters = gridDim.x / C;
    const int64_t cid = blockIdx.x / C;
    const int lane = tid & 31;
    const int NPC = a.npc;                          // pencils per CTA (even, so pairs never split)
    C2<T> *Fh = reinterpret_cast<C2<T> *>(a.fh_ws) + cid * (int64_t)N * NP;   // this cluster's spectrum
    const T scale = T(1) / T(CELL);
    const T *Mbase = reinterpret_cast<const T *>(a.mult);

    const int64_t ncells = a.dev_ncells ? (int64_t)*a.dev_ncells : a.ncells;
    int64_t c = cid - nclusters;
    for (;;) {
        if (a.counter) {            // dynamic: the cluster takes the next unclaimed cell
            if (rank == 0 && tid == 0) *s_cell = (long long)atomicAdd(a.counter, 1ULL);
            bar.full();
            c = *cl.map_shared_rank(s_cell, 0);
        } else {
            c += nclusters;
        }
        if (c >= ncells) break;
        const int64_t coff = a.cell_off ? a.cell_off[c] : c * CELL;
        const int64_t cglob = a.cell_id ? a.cell_id[c] : c;
        const T *F = reinterpret_cast<const T *>(a.F) + coff;
        T *Out = reinterpret_cast<T *>(a.Q) + coff;
        if (tid == 0) *s_nubig = 0;

        // ---------------- F1: own planes, last axis real -> half complex (two rows per thread)
        // rows q and q + rows/2 per thread: consecutive threads touch consecutive rows, so the
        // odd row stride (H complex) keeps shared-memory accesses conflict free
        for (int q = tid; q < npairs; q += nt) {
            const int r0 = q, r1 = q + npairs;
            const T *src0 = F + ((int64_t)rank * rows + r0) * N;
            const T *src1 = F + ((int64_t)rank * rows + r1) * N;
            T x0[N], x1[N];
            load_row<T, N>(src0, x0);
            load_row<T, N>(src1, x1);
            C2<T> X0[H], X1[H];
            r2c_pair<N, T>(x0, x1, X0, X1);
#pragma unroll
            for (int k = 0; k < H; ++k) {
                Is0[(r0 / N1) * NPP + (r0 % N1) * H + k] = X0[k];
                Is0[(r1 / N1) * NPP + (r1 % N1) * H + k] = X1[k];
            }
        }
        if constexpr (D == 3) {
            __syncthreads();
            for (int q = tid; q < P * H; q += nt) {            // axis 1, forward
                const int zl = q / H, lx = q % H;
                C2<T> *col = Is0 + (size_t)zl * NPP + lx;
                C2<T> v[N];
#pragma unroll
                for (int y = 0; y < N; ++y) v[y] = col[y * H];
                fft<N, -1, N>(v);
#pragma unroll
                for (int y = 0; y < N; ++y) col[y * H] = v[y];
            }
        }
        bar.full();

        // ---------------- F2: gather the axis-0 pencils and finish the forward transform
        // (warp-uniform trip count: lane pairs shuffle inside gather_pencil)
        for (int q0 = tid - lane; q0 < NPC; q0 += nt) {
            const int pencil = rank * NPC + q0 + lane;
            const bool has = q0 + lane < NPC && pencil < NP;
            const unsigned mask = __ballot_sync(0xffffffffu, has);
            if (has) {
                C2<T> v[N];
                gather_pencil<T, N, WIDE>(v, Is0, P, pm, NPP, pencil, mask);
                fft<N, -1, N>(v);
#pragma unroll
                for (int z = 0; z < N; ++z) Fh[(size_t)z * NP + pencil] = cscale(v[z], scale);
            }
        }
        // publishes Fh to the CTA (stage A reads pencils other threads stored) and keeps every
        // CTA's slab intact until all gathers are done
        bar.full();

        Diag dg;
        dg.reset();

        for (int o = 0; o < a.nops; ++o) {
            const Op op = a.ops[o];
            const bool pair = op.kind >= OP_PAIR;
            // ---------------- A: multiply, inverse along axis 0, scatter to the owners' slabs;
            // one (direction, pencil) item per thread, warp-uniform trip count
            const int nitems = (pair ? 2 : 1) * NPC;
            for (int q0 = tid - lane; q0 < nitems; q0 += nt) {
                const int q = q0 + lane;
                const int b = q >= NPC;
                const int pencil = rank * NPC + (q - b * NPC);
                const bool has = q < nitems && pencil < NP;
                const unsigned mask = __ballot_sync(0xffffffffu, has);
                if (has) {
                    const int dir = b ? op.dir2 : op.dir;
                    const T *M = Mbase + (size_t)dir * N * NP + pencil;
                    C2<T> v[N];
#pragma unroll
                    for (int z = 0; z < N; ++z) v[z] = cscale(Fh[(size_t)z * NP + pencil], __ldg(M + (size_t)z * NP));
                    fft<N, 1, N>(v);
                    scatter_pencil<T, N, WIDE>(v, b ? Is1 : Is0, P, pm, NPP, pencil, mask);
                    if (a.prefetch && o + 1 < a.nops) {   // pull the next op's multipliers towards L1
                        const Op nx = a.ops[o + 1];
                        const T *Mn = Mbase + (size_t)(b ? nx.dir2 : nx.dir) * N * NP + pencil;
#pragma unroll
                        for (int z = 0; z < N; ++z) asm volatile("prefetch.global.L1 [%0];" ::"l"(Mn + (size_t)z * NP));
                    }
                }
            }
            bar.full();

            // ---------------- B: local inverse passes and accumulation
            if constexpr (D == 3) {
                const int ncol = (pair ? 2 : 1) * P * H;
                for (int q = tid; q < ncol; q += nt) {          // axis 1, inverse
                    const int b = q >= P * H;
                    const int rem = q - b * P * H;
                    const int zl = rem / H, lx = rem % H;
                    C2<T> *col = (b ? Is1 : Is0) + (size_t)zl * NPP + lx;
                    C2<T> v[N];
#pragma unroll
                    for (int y = 0; y < N; ++y) v[y] = col[y * H];
                    fft<N, 1, N>(v);
#pragma unroll
                    for (int y = 0; y < N; ++y) col[y * H] = v[y];
                }
                __syncthreads();
            }
            if (pair) {
                // one row per thread, both directions at once: a_e (slab 0) and S_e (slab 1)
                // come out of a single complex transform; G (column-major) += a_e S_e
                const bool last = op.kind == OP_PAIR_LAST;
                const bool big = *s_nubig != 0;
                for (int r = tid; r < rows; r += nt) {
                    // two Hermitian half rows -> one complex row z (a_e + i S_e), built straight
                    // from shared memory (the two-for-one inverse of c2r_pair)
                    C2<T> z[N];
                    const int ro = (r / N1) * NPP + (r % N1) * H;
                    c2r_rows_from<N, T>(Is0 + ro, Is1 + ro, z);
                    T *Gr = Gb + r;
                    if (!last) {
#pragma unroll
                        for (int n = 0; n < N; ++n) Gr[n * rows] += z[n].x * z[n].y;
                    } else {
                        T qv[N];
#pragma unroll
                        for (int n = 0; n < N; ++n) qv[n] = Gr[n * rows] + z[n].x * z[n].y;
                        const int64_t grow = (int64_t)rank * rows + r;
                        T fr[N];
                        load_row<T, N>(F + grow * N, fr);
                        emit_row<T, D, N>(a, fr, Out + grow * N, qv, nullptr, big, grow, dg);
                    }
                }
            } else {
                for (int q = tid; q < npairs; q += nt) {
                    const int r0 = q, r1 = q + npairs;
                    C2<T> z[N];                      // z[n] = (row r0, row r1) at x = n
                    c2r_rows_from<N, T>(Is0 + (r0 / N1) * NPP + (r0 % N1) * H, Is0 + (r1 / N1) * NPP + (r1 % N1) * H, z);
                    // S and G are stored column-major ([x][row]): consecutive threads own
                    // consecutive rows, so every access below is conflict free without padding
                    T *S0 = Sb + r0, *S1 = Sb + r1;
                    T *G0 = Gb + r0, *G1 = Gb + r1;
                    const T w = T(op.w);
                    switch (op.kind) {
                    case OP_S_SET:
#pragma unroll
                        for (int n = 0; n < N; ++n) { S0[n * rows] = w * z[n].x; S1[n * rows] = w * z[n].y; }
                        break;
                    case OP_S_ADD:
#pragma unroll
                        for (int n = 0; n < N; ++n) { S0[n * rows] += w * z[n].x; S1[n * rows] += w * z[n].y; }
                        break;
                    case OP_G_SET:
#pragma unroll
                        for (int n = 0; n < N; ++n) { G0[n * rows] = z[n].x * S0[n * rows]; G1[n * rows] = z[n].y * S1[n * rows]; }
                        break;
                    case OP_G_ADD:
#pragma unroll
                        for (int n = 0; n < N; ++n) { G0[n * rows] += z[n].x * S0[n * rows]; G1[n * rows] += z[n].y * S1[n * rows]; }
                        break;
                    case OP_NU_INIT: {          // paired mode, first pass: G = -F nu
                        bool big = false;
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const int r = half ? r1 : r0;
                            T fr[N];
                            load_row<T, N>(F + ((int64_t)rank * rows + r) * N, fr);
                            T *Gr = Gb + r;
                            T mx = half ? z[0].y : z[0].x;
#pragma unroll
                            for (int n = 0; n < N; ++n) {
                                const T nu = half ? z[n].y : z[n].x;
                                Gr[n * rows] = -fr[n] * nu;
                                mx = nu > mx ? nu : mx;
                                if (T(a.dt) * nu > T(1)) big = true;
                            }
                            dg.max_nu = fmax(dg.max_nu, (double)mx);
                        }
                        if (big && a.out_mode == OUT_EULER) *s_nubig = 1;
                    } break;
                    default: {  // OP_LOSS (single mode, last): Q = G - F nu; output; diagnostics
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const int r = half ? r1 : r0;
                            const int64_t grow = (int64_t)rank * rows + r;
                            T fr[N], nu[N];
                            load_row<T, N>(F + grow * N, fr);
                            T *Gr = Gb + r;
                            T qv[N];
#pragma unroll
                            for (int n = 0; n < N; ++n) nu[n] = half ? z[n].y : z[n].x;
                            T mx = nu[0];
#pragma unroll
                            for (int n = 0; n < N; ++n) {
                                qv[n] = Gr[n * rows] - fr[n] * nu[n];
                                mx = nu[n] > mx ? nu[n] : mx;
                            }
                            dg.max_nu = fmax(dg.max_nu, (double)mx);
                            emit_row<T, D, N>(a, fr, Out + grow * N, qv, nu, false, grow, dg);
                        }
                    } break;
                    }
                }
            }
            bar.war();
        }

        // ---------------- per-cell FP64 reduction of the diagnostics
        if (a.diag) {
            dg.sum[7] = dg.min_f;
            dg.sum[8] = dg.max_nu;
            dg.sum[9] = dg.min_out;
            const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
#pragma unroll
            for (int k = 0; k < kDiag; ++k) {
                double v = dg.sum[k];
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const double u = __shfl_xor_sync(0xffffffffu, v, s);
                    v = (k == 7 || k == 9) ? fmin(v, u) : (k == 8 ? fmax(v, u) : v + u);
                }
                if (lane == 0) part[warp * kDiag + k] = v;
            }
            __syncthreads();
            if (tid < kDiag) {
                const int k = tid;
                double v = part[k];
                for (int w2 = 1; w2 < nw; ++w2) {
                    const double u = part[w2 * kDiag + k];
                    v = (k == 7 || k == 9) ? fmin(v, u) : (k == 8 ? fmax(v, u) : v + u);
                }
                part[32 * kDiag + k] = v;
            }
            bar.full();
            if (rank == 0 && tid < kDiag) {
                const int k = tid;
                double v = part[32 * kDiag + k];
                for (int r = 1; r < C; ++r) {
                    const double *rp = cl.map_shared_rank(part, r);
                    const double u = rp[32 * kDiag + k];
                    v = (k == 7 || k == 9) ? fmin(v, u) : (k == 8 ? fmax(v, u) : v + u);
                }
                const double hd = (D == 3) ? a.h * a.h * a.h : a.h * a.h;
                if (k == 0 || k == 5) v *= hd;
                else if (k >= 1 && k <= 3) v *= hd * a.h;
                else if (k == 4) v *= 0.5 * hd * a.h * a.h;
                if (D == 2 && k == 3) v = 0.0;
                a.diag[cglob * kDiag + k] = v;
            }
            bar.war();
        }
    }
    bar.war();   // no CTA leaves while a peer may still read its shared memory
}

}  // namespace ef
