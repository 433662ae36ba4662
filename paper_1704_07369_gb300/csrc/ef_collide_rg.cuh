// ef_collide_rg.cuh -- the FP32 3D collision kernel with the gain accumulator in registers and
// the forward spectrum in shared memory (one thread-block cluster per cell).
//
// Same arithmetic as collide_kernel (Sec. 4.1, eq. fastAlg, paired op list: G = -F nu, then
// G += a_e S_e for every first direction e, where S_e is the inverse transform of the weighted sum
// of e's partner multipliers; the last pass writes Q or F + dt Q with the FP64 diagnostics), laid
// out for sm_103a:
//   * every thread owns RPT fixed real rows for the whole cell, so G lives in its registers: the
//     accumulate pass touches no shared memory for G, and the shared memory this frees holds the
//     CTA's axis-0 pencils of the forward spectrum, so stage A reads Fhat from shared memory
//     instead of L2;
//   * the multiplier of every op vanishes on the modes with a component -N/2 (sigma_N(-N/2) = 0,
//     Sec. 4.1), so the Nyquist column k_x = -N/2 is neither stored nor transformed: the axis-0
//     pencils (k_y, k_x < N/2) number N^2/2, the axis-1 columns of a plane N/2, and each stage has
//     exactly one work item per real row (N^2 / C per CTA for a paired op), which matches the
//     thread count rows / RPT with no partial rounds;
//   * slab rows of N/2 + 2 complex values (an odd count of 16-byte pairs) and float4 row access
//     keep the row passes free of bank conflicts; a plane stride of 8 mod 16 complex values does
//     the same for the paired 16-byte pencil stores of stage A.
// Per cell: F1 (own planes: real -> half complex along the last axis, axis 1 forward), F2 (own
// pencils: gather through distributed shared memory, axis 0 forward, keep in shared memory), then
// per op: A (multiply, axis 0 inverse, scatter to the owners' slabs), B (axis 1 inverse, then the
// two-for-one half complex -> real row transform and the accumulate / output).
#pragma once

#include "ef_collide_impl.cuh"

namespace ef {

// Slab layout of one axis-0 plane: N rows (k_y) of N/2 stored k_x values (complex).  Where a row
// holds a multiple of 4 16-byte pairs (N = 16, 32, 48, 64) the pairs of row y are stored in the
// order pair ^ s(y), an XOR swizzle inside aligned groups of pairs: s(y) = y & 7 when a row holds a
// multiple of 8 pairs (its rows all start on the same bank), (y >> 1) & 3 when it holds 4 mod 8
// (consecutive rows start 64 bytes apart).  Otherwise each row is padded to N/2 + 2 values (an odd
// number of pairs).  Either way 16-byte accesses to pair j of eight consecutive rows, and 8-byte
// accesses to a k_x range of one row, fall on distinct banks.
template <int N>
__host__ __device__ constexpr bool rg_swizzled() { return (N / 4) % 4 == 0; }
template <int N>
__host__ __device__ constexpr int rg_row_stride() { return rg_swizzled<N>() ? N / 2 : N / 2 + 2; }
template <int N>
__device__ __forceinline__ int rg_swz(int y)
{
    if constexpr (!rg_swizzled<N>()) return 0;
    else if constexpr ((N / 4) % 8 == 0) return y & 7;
    else return (y >> 1) & 3;
}
// offset (complex values) of (k_y = y, k_x) inside a plane; the pair (k_x even, k_x + 1) stays adjacent
template <int N>
__device__ __forceinline__ int rg_at(int y, int kx)
{
    if constexpr (rg_swizzled<N>()) return y * (N / 2) + ((((kx >> 1) ^ rg_swz<N>(y)) << 1) | (kx & 1));
    else return y * rg_row_stride<N>() + kx;
}
// plane stride: N rows, padded to r mod 16 complex values (16 values = 128 bytes, one bank line).
// Swizzled rows: r = 8, so that the two lanes of a scatter pair (planes z and z + 1, same pencil
// offset) store to opposite halves of a line.  Padded rows: r = N/2 mod 16, so that column q =
// plane * N/2 + k_x of a column pass sits at bank slot q + const (mod 16) and the warps of the
// axis-1 passes, which straddle planes, touch every 8-byte slot exactly twice.
template <int N>
__host__ __device__ constexpr int rg_plane_stride()
{
    constexpr int s = N * rg_row_stride<N>();
    constexpr int r = rg_swizzled<N>() ? 8 : (N / 2) % 16;
    return s + ((r - s % 16) % 16 + 16) % 16;
}
// Instantiations ("variants", one CTA per SM each): 1 = the gain accumulator G in registers, one
// row per thread, the size's widest launch bound; 2 = G in registers, two rows per thread; 3 = G in
// registers, one row per thread, at most 200 threads (N = 40, 48: 7 warps keep 255 registers where
// the widest bound leaves 168); 4 = G in shared memory (any thread count up to the bound: for the
// sizes where a row in registers besides a length-N transform would spill).  rg_bound is the
// launch bound (0: not built).
template <int N, int V>
__host__ __device__ constexpr int rg_bound()
{
    if (V == 1) return N == 40 ? 320 : (N == 32 || N == 64) ? 256 : 288;
    if (V == 2) return N == 16 ? 128 : N == 24 ? 288 : N == 32 ? 256 : N == 40 ? 200 : N == 48 ? 192 : 128;
    if (V == 3) return (N == 40 || N == 48) ? 200 : 0;
    if (V == 4) return N == 40 ? 320 : (N == 48 || N == 24) ? 288 : 256;
    return 0;
}
template <int V>
__host__ __device__ constexpr int rg_rpt() { return V == 2 ? 2 : 1; }
template <int N>
__host__ __device__ constexpr bool rg_built() { return N == 16 || N == 24 || N == 32 || N == 40 || N == 48 || N == 64; }

// pencils (k_y, k_x < N/2) per CTA of a C-CTA cluster; 0 if the split is not even
__host__ __device__ inline int rg_npc(int N, int C)
{
    const int np = N * N / 2;
    return (np % C == 0 && (np / C) % 2 == 0) ? np / C : 0;
}

template <int N>
__host__ __device__ constexpr size_t rg_smem_bytes(int planes, int npc, bool g_shared)
{
    return (size_t)2 * planes * rg_plane_stride<N>() * 8 + (size_t)N * npc * 8 + (g_shared ? (size_t)planes * N * N * 4 : 0) +
           (32 + 1) * kDiag * sizeof(double) + 16 + 32 * sizeof(float);
}

// lanes of the calling thread's warp that exist: a block whose size is not a multiple of 32 has a
// partial last warp, and warp-synchronous operations name only these lanes
__device__ __forceinline__ unsigned warp_lanes(int nt, int tid)
{
    const int n = nt - (tid & ~31);
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// in-plane offset of the even pencil of a lane pair: pencil q (even) -> (k_y, k_x) = (q / (N/2), q % (N/2))
template <int N>
__device__ __forceinline__ int rg_poff(int q) { return rg_at<N>(q / (N / 2), q % (N / 2)); }

// stage-A scatter of one pencil (lane pairs hold pencils q, q + 1 of one slab row; one shuffle per
// z pair so that each lane issues 16-byte stores; owner CTA of z by multiply-high)
template <int N>
__device__ __forceinline__ void rg_scatter(const C2<float> (&v)[N], uint32_t slab_base, int P, unsigned long long pm,
                                           int poff, bool odd, unsigned mask)
{
    constexpr int NPP = rg_plane_stride<N>();
#pragma unroll
    for (int z0 = 0; z0 < N; z0 += 2) {
        const C2<float> send = odd ? v[z0] : v[z0 + 1];
        C2<float> recv;
        recv.x = __shfl_xor_sync(mask, send.x, 1);
        recv.y = __shfl_xor_sync(mask, send.y, 1);
        const int z = odd ? z0 + 1 : z0;
        const C2<float> lo = odd ? recv : v[z0];
        const C2<float> hi = odd ? v[z0 + 1] : recv;
        const int owner = plane_owner(z, pm), zl = z - owner * P;
        st_cluster(cluster_map(slab_base + (uint32_t)((zl * NPP + poff) * 8), owner), make_float4(lo.x, lo.y, hi.x, hi.y));
    }
}

template <int N>
__device__ __forceinline__ void rg_gather(C2<float> (&v)[N], uint32_t slab_base, int P, unsigned long long pm, int poff,
                                          bool odd, unsigned mask)
{
    constexpr int NPP = rg_plane_stride<N>();
#pragma unroll
    for (int z0 = 0; z0 < N; z0 += 2) {
        const int z = odd ? z0 + 1 : z0;
        const int owner = plane_owner(z, pm), zl = z - owner * P;
        const float4 w = ld_cluster_f4(cluster_map(slab_base + (uint32_t)((zl * NPP + poff) * 8), owner));
        const C2<float> lo = C2<float>{w.x, w.y}, hi = C2<float>{w.z, w.w};
        const C2<float> send = odd ? lo : hi;
        C2<float> recv;
        recv.x = __shfl_xor_sync(mask, send.x, 1);
        recv.y = __shfl_xor_sync(mask, send.y, 1);
        v[z0] = odd ? recv : lo;
        v[z0 + 1] = odd ? hi : recv;
    }
}

// two Hermitian half rows (k < N/2; the k = N/2 entry is zero for every op) -> z = IFFT(R0) + i
// IFFT(R1), read as 16-byte pairs; R0, R1 point at the start of rows y0, y1 of their planes
template <int N>
__device__ __forceinline__ void rg_c2r_rows(const C2<float> *R0, int y0, const C2<float> *R1, int y1, C2<float> (&z)[N])
{
    const float4 *A = reinterpret_cast<const float4 *>(R0);
    const float4 *B = reinterpret_cast<const float4 *>(R1);
    const int sw0 = rg_swz<N>(y0);
    const int sw1 = rg_swz<N>(y1);
#pragma unroll
    for (int k2 = 0; k2 < N / 2; k2 += 2) {
        const float4 a = A[(k2 / 2) ^ sw0], b = B[(k2 / 2) ^ sw1];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k2 + h;
            const C2<float> x0 = h ? C2<float>{a.z, a.w} : C2<float>{a.x, a.y};
            const C2<float> x1 = h ? C2<float>{b.z, b.w} : C2<float>{b.x, b.y};
            if (k == 0) {
                z[0] = C2<float>{x0.x, x1.x};
            } else {
                z[k] = C2<float>{x0.x - x1.y, x0.y + x1.x};
                z[N - k] = C2<float>{x0.x + x1.y, x1.x - x0.y};
            }
        }
    }
    z[N / 2] = C2<float>{0.f, 0.f};
    fft<N, 1, N>(z);
}

// Per-cell reduction of the FP32 3D kernels' diagnostics, FP32 until the last step: float-float
// sums and FP32 minima / maxima across each warp (shuffles), across the CTA's warps (kDiag threads)
// and across the cluster's CTAs (rank 0, distributed shared memory), then one conversion to FP64
// and the cell's scale factors.  part (33 * kDiag doubles of shared memory) holds float-float
// pairs here: [warp][k][hi, lo], [32][k][hi, lo] the CTA's.  Slot 8 (max nu) comes from the loss
// op's per-warp maxima.  (GB300's FP64 pipe runs at a small fraction of the FP32 rate, so the
// sums stay on the FP32 pipe; float-float keeps about 48 significant bits.)
template <typename SYNC>
__device__ __forceinline__ void diag_reduce_cell(const CollideArgs &a, const DiagF &dg, const float *s_maxnu, double *part,
                                                 unsigned wmask, int lane, int tid, int nt, int rank, int C, SYNC &bar,
                                                 cg::cluster_group &cl, int64_t cglob)
{
    float *pf = reinterpret_cast<float *>(part);
    const int warp = tid >> 5, nw = (nt + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        FF v = dg.sum[k];
#pragma unroll
        for (int sh2 = 16; sh2 > 0; sh2 >>= 1) {
            FF u;
            u.hi = __shfl_xor_sync(wmask, v.hi, sh2);
            u.lo = __shfl_xor_sync(wmask, v.lo, sh2);
            if ((wmask >> (lane ^ sh2)) & 1u) v = ff_merge(v, u);
        }
        if (lane == 0) {
            pf[(warp * kDiag + k) * 2] = v.hi;
            pf[(warp * kDiag + k) * 2 + 1] = v.lo;
        }
    }
    float mnf = dg.min_f, mno = dg.min_out;
#pragma unroll
    for (int sh2 = 16; sh2 > 0; sh2 >>= 1) {
        const float u1 = __shfl_xor_sync(wmask, mnf, sh2), u2 = __shfl_xor_sync(wmask, mno, sh2);
        if ((wmask >> (lane ^ sh2)) & 1u) {
            mnf = fminf(mnf, u1);
            mno = fminf(mno, u2);
        }
    }
    if (lane == 0) {
        pf[(warp * kDiag + 7) * 2] = mnf;
        pf[(warp * kDiag + 8) * 2] = s_maxnu[warp];
        pf[(warp * kDiag + 9) * 2] = mno;
    }
    __syncthreads();
    if (tid < kDiag) {
        const int k = tid;
        FF v{pf[k * 2], pf[k * 2 + 1]};
        for (int w2 = 1; w2 < nw; ++w2) {
            const FF u{pf[(w2 * kDiag + k) * 2], pf[(w2 * kDiag + k) * 2 + 1]};
            if (k == 7 || k == 9) v.hi = fminf(v.hi, u.hi);
            else if (k == 8) v.hi = fmaxf(v.hi, u.hi);
            else v = ff_merge(v, u);
        }
        pf[(32 * kDiag + k) * 2] = v.hi;
        pf[(32 * kDiag + k) * 2 + 1] = (k >= 7) ? 0.f : v.lo;
    }
    bar.full();
    if (rank == 0 && tid < kDiag) {
        // the other CTAs' values, all loads issued before the first use
        const int k = tid;
        float2 u[16];
#pragma unroll
        for (int r = 1; r < 16; ++r)
            if (r < C) u[r] = *reinterpret_cast<const float2 *>(cl.map_shared_rank(pf, r) + (32 * kDiag + k) * 2);
        FF v{pf[(32 * kDiag + k) * 2], pf[(32 * kDiag + k) * 2 + 1]};
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            if (r >= C) continue;
            if (k == 7 || k == 9) v.hi = fminf(v.hi, u[r].x);
            else if (k == 8) v.hi = fmaxf(v.hi, u[r].x);
            else v = ff_merge(v, FF{u[r].x, u[r].y});
        }
        double d = ff_value(v);
        const double hd = a.h * a.h * a.h;
        if (k == 0 || k == 5) d *= hd;
        else if (k >= 1 && k <= 3) d *= hd * a.h;
        else if (k == 4) d *= 0.5 * hd * a.h * a.h;
        a.diag[cglob * kDiag + k] = d;
    }
    // no barrier here: part[] is written again only in the next cell's reduction, after cluster
    // barriers that rank 0 reaches only once these reads are done (the kernel's closing barrier
    // covers the last cell)
}

// GS = false: G of this thread's RPT rows in registers (nt * RPT = rows); GS = true: G in shared
// memory, column-major ([x][row], so consecutive threads touch consecutive banks), rows looped.
template <int D, int N, int RPT, int LB, bool GS>
__global__ void __launch_bounds__(LB, 1) collide_kernel_rg(const CollideArgs a)
{
    static_assert(D == 3, "3D only");
    using T = float;
    constexpr int NPP = rg_plane_stride<N>();
    constexpr int NH = N / 2;              // stored k_x values per row
    constexpr int64_t CELL = (int64_t)N * N * N;

    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int P = a.planes;
    const int tid = threadIdx.x, nt = blockDim.x;
    Sync bar{cl, C};
    const int rows = P * N;
    const int NPC = a.npc;                 // pencils per CTA = N^2 / (2 C), even
    // the launch shape this layout needs (the same for every CTA, so all return together):
    // RPT rows per thread exactly (G in registers), an even pencil split over the cluster
    if ((!GS && nt * RPT != rows) || P * C != N || 2 * NPC * C != N * N || NPC % 2) {
        if (tid == 0) record_status(a.status, 2);       // EF_ERR_UNSUPPORTED
        return;
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2<T> *Is0 = reinterpret_cast<C2<T> *>(smem_raw);
    C2<T> *Is1 = Is0 + (size_t)P * NPP;
    C2<T> *Fs = Is1 + (size_t)P * NPP;                       // [z][local pencil] forward spectrum
    T *Gs = reinterpret_cast<T *>(Fs + (size_t)N * NPC);      // GS: [x][row]
    double *part = reinterpret_cast<double *>(Gs + (GS ? (size_t)rows * N : 0));   // [32 warps + 1][kDiag]
    long long *s_cell = reinterpret_cast<long long *>(part + (32 + 1) * kDiag);
    int *s_nubig = reinterpret_cast<int *>(s_cell + 1);
    float *s_maxnu = reinterpret_cast<float *>(s_cell + 2);          // [32 warps] max nu of the loss op
    const uint32_t base0 = smem_u32addr(Is0), base1 = smem_u32addr(Is1);

    const unsigned long long pm = (0x100000000ull + (unsigned)P - 1u) / (unsigned)P;
    const int64_t nclusters = gridDim.x / C;
    const int64_t cid = blockIdx.x / C;
    const int lane = tid & 31;
    const unsigned wmask = warp_lanes(nt, tid);
    const T scale = T(1) / T(CELL);
    const T *Mbase = reinterpret_cast<const T *>(a.mult);
    constexpr int H = N / 2 + 1;
    constexpr int NPT = N * H;             // multiplier table: [dir][k_z][k_y * H + k_x]

    const int64_t ncells = a.dev_ncells ? (int64_t)*a.dev_ncells : a.ncells;
    int64_t c = cid - nclusters;
    for (;;) {
        if (a.counter) {
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

        // ---------------- F1: own rows real -> half complex (k_x < N/2 kept), two rows per item
        for (int q = tid; q < rows / 2; q += nt) {
            const int r0 = q, r1 = q + rows / 2;
            T x0[N], x1[N];
            load_row<T, N>(F + ((int64_t)rank * rows + r0) * N, x0);
            load_row<T, N>(F + ((int64_t)rank * rows + r1) * N, x1);
            C2<T> X0[H], X1[H];
            r2c_pair<N, T>(x0, x1, X0, X1);
            C2<T> *d0 = Is0 + (r0 / N) * NPP, *d1 = Is0 + (r1 / N) * NPP;
            const int y0 = r0 % N, y1 = r1 % N;
#pragma unroll
            for (int k = 0; k < NH; k += 2) {
                *reinterpret_cast<float4 *>(d0 + rg_at<N>(y0, k)) = make_float4(X0[k].x, X0[k].y, X0[k + 1].x, X0[k + 1].y);
                *reinterpret_cast<float4 *>(d1 + rg_at<N>(y1, k)) = make_float4(X1[k].x, X1[k].y, X1[k + 1].x, X1[k + 1].y);
            }
        }
        __syncthreads();
        for (int q = tid; q < P * NH; q += nt) {            // axis 1 forward, k_x < N/2
            const int zl = q / NH, lx = q % NH;
            C2<T> *pl = Is0 + (size_t)zl * NPP;
            C2<T> v[N];
#pragma unroll
            for (int y = 0; y < N; ++y) v[y] = pl[rg_at<N>(y, lx)];
            fft<N, -1, N>(v);
#pragma unroll
            for (int y = 0; y < N; ++y) pl[rg_at<N>(y, lx)] = v[y];
        }
        bar.full();

        // ---------------- F2: own pencils, gathered, axis 0 forward, kept in shared memory
        for (int q0 = tid - lane; q0 < NPC; q0 += nt) {
            const int ql = q0 + lane;
            const bool has = ql < NPC;
            const unsigned mask = __ballot_sync(wmask, has);
            if (has) {
                const int q = rank * NPC + ql;
                C2<T> v[N];
                rg_gather<N>(v, base0, P, pm, rg_poff<N>(q & ~1), q & 1, mask);
                fft<N, -1, N>(v);
#pragma unroll
                for (int z = 0; z < N; ++z) Fs[(size_t)z * NPC + ql] = cscale(v[z], scale);
            }
        }
        bar.full();                        // Fs complete; every slab free again

        // the diagnostics accumulate only in the last op (reset there), so they hold no registers
        // through the earlier ops; the loss op's max nu goes to shared memory per warp
        DiagF dg;
        T g[GS ? 1 : RPT][N];              // G in registers: this thread's rows tid + j nt

        for (int o = 0; o < a.nops; ++o) {
            const Op op = a.ops[o];
            const bool pair = op.kind >= OP_PAIR;
            // ---------------- A: multiply, axis 0 inverse, scatter (one (direction, pencil) item
            // per thread; lanes of a pair share the direction since NPC is even)
            const int nitems = (pair ? 2 : 1) * NPC;
            for (int q0 = tid - lane; q0 < nitems; q0 += nt) {
                const int qi = q0 + lane;
                const bool has = qi < nitems;
                const unsigned mask = __ballot_sync(wmask, has);
                if (has) {
                    const int b = qi >= NPC;
                    const int ql = qi - b * NPC;
                    const int q = rank * NPC + ql;
                    const int ky = q / NH, kx = q % NH;
                    const T *M = Mbase + (size_t)(b ? op.dir2 : op.dir) * N * NPT + ky * H + kx;
                    C2<T> v[N];
#pragma unroll
                    for (int z = 0; z < N; ++z) v[z] = cscale(Fs[(size_t)z * NPC + ql], __ldg(M + (size_t)z * NPT));
                    fft<N, 1, N>(v);
                    rg_scatter<N>(v, b ? base1 : base0, P, pm, rg_poff<N>(q & ~1), q & 1, mask);
                    if (a.prefetch && o + 1 < a.nops) {
                        // pull the next op's multipliers of this item towards L1 while the local
                        // passes run (the next op has the same item split: both directions or, after
                        // the loss, two); a hint only, every address is inside the table
                        const Op nx = a.ops[o + 1];
                        const T *Mn = Mbase + (size_t)(b ? nx.dir2 : nx.dir) * N * NPT + ky * H + kx;
#pragma unroll
                        for (int z = 0; z < N; ++z) asm volatile("prefetch.global.L1 [%0];" ::"l"(Mn + (size_t)z * NPT));
                    }
                }
            }
            bar.full();

            // ---------------- B: axis 1 inverse on the stored k_x < N/2 columns of each slab
            const int ncol = (pair ? 2 : 1) * P * NH;
            for (int q = tid; q < ncol; q += nt) {
                const int b = q >= P * NH;
                const int rem = q - b * P * NH;
                const int zl = rem / NH, lx = rem % NH;
                C2<T> *pl = (b ? Is1 : Is0) + (size_t)zl * NPP;
                C2<T> v[N];
#pragma unroll
                for (int y = 0; y < N; ++y) v[y] = pl[rg_at<N>(y, lx)];
                fft<N, 1, N>(v);
#pragma unroll
                for (int y = 0; y < N; ++y) pl[rg_at<N>(y, lx)] = v[y];
            }
            __syncthreads();

            // ---------------- rows: half complex -> real, accumulate / output
            if (pair) {
                const bool last = op.kind == OP_PAIR_LAST;
                const bool big = *s_nubig != 0;
                if (last) dg.reset();
                if constexpr (GS) {
                    for (int r = tid; r < rows; r += nt) {
                        const int rb = (r / N) * NPP + (r % N) * rg_row_stride<N>();
                        C2<T> z[N];
                        rg_c2r_rows<N>(Is0 + rb, r % N, Is1 + rb, r % N, z);
                        T *Gr = Gs + r;
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
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        const int r = tid + j * nt;
                        const int rb = (r / N) * NPP + (r % N) * rg_row_stride<N>();
                        C2<T> z[N];
                        rg_c2r_rows<N>(Is0 + rb, r % N, Is1 + rb, r % N, z);
                        if (!last) {
#pragma unroll
                            for (int n = 0; n < N; ++n) g[j][n] += z[n].x * z[n].y;
                        } else {
                            T qv[N];
#pragma unroll
                            for (int n = 0; n < N; ++n) qv[n] = g[j][n] + z[n].x * z[n].y;
                            const int64_t grow = (int64_t)rank * rows + r;
                            T fr[N];
                            load_row<T, N>(F + grow * N, fr);
                            emit_row<T, D, N>(a, fr, Out + grow * N, qv, nullptr, big, grow, dg);
                        }
                    }
                }
            } else {
                // the loss (first op): nu of the rows, G = -F nu; two rows share one complex
                // transform (with G in registers and one row per thread, the second input is zero)
                bool bigt = false;
                T mxt = T(-3.0e38);
                if constexpr (GS || RPT == 2) {
                    // rows r0 and r1 = r0 + rows / 2 (G in shared memory: looped; two rows per
                    // thread in registers: tid and tid + nt = tid + rows / 2)
                    for (int q = tid; q < rows / 2; q += nt) {
                        const int r0 = q, r1 = q + rows / 2;
                        const int rb0 = (r0 / N) * NPP + (r0 % N) * rg_row_stride<N>();
                        const int rb1 = (r1 / N) * NPP + (r1 % N) * rg_row_stride<N>();
                        C2<T> z[N];
                        rg_c2r_rows<N>(Is0 + rb0, r0 % N, Is0 + rb1, r1 % N, z);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int r = j ? r1 : r0;
                            T fr[N];
                            load_row<T, N>(F + ((int64_t)rank * rows + r) * N, fr);
                            T mx = j ? z[0].y : z[0].x;
#pragma unroll
                            for (int n = 0; n < N; ++n) {
                                const T nu = j ? z[n].y : z[n].x;
                                const T gv = -fr[n] * nu;
                                if constexpr (GS) Gs[n * rows + r] = gv;
                                else g[j][n] = gv;
                                mx = nu > mx ? nu : mx;
                                if (T(a.dt) * nu > T(1)) bigt = true;
                            }
                            mxt = mx > mxt ? mx : mxt;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        const int r = tid + j * nt;
                        const C2<T> *R0 = Is0 + (r / N) * NPP;
                        const int y = r % N;
                        // real row from one half spectrum: z = IFFT(R0) (the second input zero)
                        C2<T> z[N];
#pragma unroll
                        for (int k = 1; k < NH; ++k) {
                            const C2<T> w = R0[rg_at<N>(y, k)];
                            z[k] = w;
                            z[N - k] = cconj(w);
                        }
                        z[0] = C2<T>{R0[rg_at<N>(y, 0)].x, 0.f};
                        z[NH] = C2<T>{0.f, 0.f};
                        fft<N, 1, N>(z);
                        T fr[N];
                        load_row<T, N>(F + ((int64_t)rank * rows + r) * N, fr);
                        T mx = z[0].x;
#pragma unroll
                        for (int n = 0; n < N; ++n) {
                            const T nu = z[n].x;
                            g[j][n] = -fr[n] * nu;
                            mx = nu > mx ? nu : mx;
                            if (T(a.dt) * nu > T(1)) bigt = true;
                        }
                        mxt = mx > mxt ? mx : mxt;
                    }
                }
                if (bigt && a.out_mode == OUT_EULER) *s_nubig = 1;
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1) {
                    const T u = __shfl_xor_sync(wmask, mxt, o2);
                    if ((wmask >> (lane ^ o2)) & 1u) mxt = u > mxt ? u : mxt;
                }
                if (lane == 0) s_maxnu[tid >> 5] = mxt;
            }
            bar.war();
        }

        // ---------------- per-cell reduction of the diagnostics
        if (a.diag) diag_reduce_cell(a, dg, s_maxnu, part, wmask, lane, tid, nt, rank, C, bar, cl, cglob);
    }
    bar.war();   // no CTA leaves while a peer may still read its shared memory
}

}  // namespace ef
