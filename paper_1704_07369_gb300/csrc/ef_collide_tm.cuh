// ef_collide_tm.cuh -- the FP32 3D register-accumulator collision kernel with every line transform
// split over a team of two lanes.
//
// Same arithmetic, op list, data layout and stage order as collide_kernel_rg (Sec. 4.1, eq.
// fastAlg): F1, F2 once per cell, then per op A (multiply, axis-0 inverse, scatter), B (axis-1
// inverse), the row pass with the accumulate / output.  The difference is the work item: lanes
// 2t and 2t + 1 of a warp share one length-N line.  Lane s holds the samples n = 2m + s (m < N/2),
// transforms them locally (length N/2) and the two halves are combined by one radix-2 step across
// the pair (one shuffle per value); afterwards lane s holds the outputs s N/2 .. s N/2 + N/2 - 1.
// Every thread therefore keeps half a line and half of its rows' gain accumulator in registers, so
// a CTA runs twice the threads of collide_kernel_rg for the same shared memory: the latency of the
// shared-memory, L2 and distributed-shared-memory accesses of one warp is hidden behind twice as
// many others.  The paired 16-byte pencil stores of stage A pair the two teams of a lane quad.
#pragma once

#include "ef_collide_rg.cuh"

namespace ef {

// Lanes 2t, 2t + 1 (s = lane & 1) hold x[2m + s], m < N/2, in h[m]; afterwards h[k] =
// X[s N/2 + k] with X[k] = sum_n x[n] exp(SIGN 2 pi i n k / N): a length-N/2 transform per lane,
// then X[k] = E0[k] + w^k E1[k], X[k + N/2] = E0[k] - w^k E1[k] (w = exp(SIGN 2 pi i / N)) across
// the pair, the odd lane multiplying by w^k before the exchange.
template <int N, int SIGN>
__device__ __forceinline__ void fft_team(C2<float> (&h)[N / 2], int s, unsigned mask)
{
    fft<N / 2, SIGN, N>(h);
    const float sg = s ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        C2<float> t = h[k];
        if (k > 0) {
            C2<float> w;
            if (4 * k == N) {
                w = C2<float>{0.f, SIGN > 0 ? 1.f : -1.f};
            } else {
                w = tw_value<N, float>(k);                  // exp(-2 pi i k / N)
                if (SIGN > 0) w.y = -w.y;
            }
            t = cmul(t, s ? w : C2<float>{1.f, 0.f});
        }
        C2<float> r;
        r.x = __shfl_xor_sync(mask, t.x, 1);
        r.y = __shfl_xor_sync(mask, t.y, 1);
        h[k] = C2<float>{r.x + sg * t.x, r.y + sg * t.y};
    }
}

// Stage-A scatter of a team's half pencil: lane quads hold pencils q (lanes 0, 1 of the quad, q
// even) and q + 1 (lanes 2, 3) with the same z values z = s N/2 + k; one shuffle across the quad
// per pair of k so that each lane stores a 16-byte (pencil q, pencil q + 1) pair.
template <int N>
__device__ __forceinline__ void tm_scatter(const C2<float> (&v)[N / 2], uint32_t slab_base, int P, unsigned long long pm,
                                           int poff, int s, bool odd, unsigned mask)
{
    constexpr int NPP = rg_plane_stride<N>();
#pragma unroll
    for (int k0 = 0; k0 < N / 2; k0 += 2) {
        const C2<float> send = odd ? v[k0] : v[k0 + 1];
        C2<float> recv;
        recv.x = __shfl_xor_sync(mask, send.x, 2);
        recv.y = __shfl_xor_sync(mask, send.y, 2);
        const int z = s * (N / 2) + (odd ? k0 + 1 : k0);
        const C2<float> lo = odd ? recv : v[k0];
        const C2<float> hi = odd ? v[k0 + 1] : recv;
        const int owner = plane_owner(z, pm), zl = z - owner * P;
        st_cluster(cluster_map(slab_base + (uint32_t)((zl * NPP + poff) * 8), owner), make_float4(lo.x, lo.y, hi.x, hi.y));
    }
}

// A team's half of the complex row z = IFFT(R0) + i IFFT(R1) built from two stored half rows (k_x
// < N/2; the Nyquist value is zero): lane s gets z[n] for n = 2m + s.  For n < N/2 the value comes
// from k = n, for n > N/2 from k = N - n (conjugated); n = 0 ignores the imaginary parts of the
// k = 0 values, n = N/2 is zero.  TWO = false: R1 = 0 (one real row).
template <int N, bool TWO>
__device__ __forceinline__ void tm_c2r_load(const C2<float> *R0, int y0, const C2<float> *R1, int y1, int s,
                                            C2<float> (&h)[N / 2])
{
    constexpr int NH = N / 2;
#pragma unroll
    for (int m = 0; m < NH; ++m) {
        if (m < NH / 2) {
            const int k = 2 * m + s;
            const C2<float> a = R0[rg_at<N>(y0, k)];
            const C2<float> b = TWO ? R1[rg_at<N>(y1, k)] : C2<float>{0.f, 0.f};
            if (m == 0 && s == 0) h[m] = C2<float>{a.x, b.x};
            else h[m] = C2<float>{a.x - b.y, a.y + b.x};
        } else {
            const int n = 2 * m + s;
            if (n == NH) {
                h[m] = C2<float>{0.f, 0.f};
            } else {
                const int k = N - n;
                const C2<float> a = R0[rg_at<N>(y0, k)];
                const C2<float> b = TWO ? R1[rg_at<N>(y1, k)] : C2<float>{0.f, 0.f};
                h[m] = C2<float>{a.x + b.y, b.x - a.y};
            }
        }
    }
}

// Output of one half row [x0, x0 + N/2): Q = q, written as Q (collide) or F + dt Q (Euler), with
// the status checks and the half row's share of the diagnostic sums (the same sums as emit_row).
template <int N>
__device__ __forceinline__ void tm_emit_half(const CollideArgs &a, const float (&fr)[N / 2], float *Ohalf, float (&q)[N / 2],
                                             bool nu_big, int64_t grow, int x0, DiagF &dg)
{
    constexpr int NH = N / 2;
    const int jz = (int)(grow / N) - N / 2;
    const int jy = (int)(grow % N) - N / 2;
    float s_m = 0, s_mx = 0, s_e2 = 0, s_eta = 0, s_prod = 0;
    float mn_f = fr[0], mn_out = 3.0e38f;
    bool bad = false, neg = false;
#pragma unroll
    for (int n = 0; n < NH; ++n) {
        const float f = fr[n];
        const float qv = q[n];
        float outv;
        if (a.out_mode == OUT_EULER) {
            outv = f + float(a.dt) * qv;
            if (outv < 0.f && nu_big) neg = true;
        } else {
            outv = qv;
        }
        q[n] = outv;
        if (!isfinite(outv)) bad = true;
        if (a.diag) {
            const float jx = float(x0 + n - N / 2);
            s_m += f;
            s_mx += f * jx;
            s_e2 += f * jx * jx;
            if (f > 0.f) {
                const float lf = log_t<float>(f);
                s_eta += f * lf;
                s_prod += qv * lf;
            }
            mn_f = f < mn_f ? f : mn_f;
            mn_out = outv < mn_out ? outv : mn_out;
        }
    }
    store_row<float, NH>(Ohalf, q);
    if (bad) record_status(a.status, 7);     // EF_ERR_NOT_FINITE
    if (neg) record_status(a.status, 6);     // EF_ERR_POSITIVITY
    if (a.diag) dg.template add_row<3, float>(s_m, s_mx, s_e2, s_eta, s_prod, jz, jy, mn_f, mn_out);
}

// RPT: rows per team (G of RPT half rows per lane in registers; teams = rows / RPT, threads = 2
// teams); LB, MINB: launch bounds.
template <int D, int N, int RPT, int LB, int MINB>
__global__ void __launch_bounds__(LB, MINB) collide_kernel_tm(const CollideArgs a)
{
    static_assert(D == 3, "3D only");
    static_assert(N % 8 == 0, "team transforms pair k values of a half line");
    using T = float;
    constexpr int NPP = rg_plane_stride<N>();
    constexpr int NH = N / 2;               // stored k_x values per row; half a line per lane
    constexpr int64_t CELL = (int64_t)N * N * N;

    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int P = a.planes;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, s = tid & 1, tm = tid >> 1, nteam = nt >> 1;
    const int wteam = (tid - lane) >> 1;    // the warp's first team
    const unsigned wmask = warp_lanes(nt, tid);
    Sync bar{cl, C};
    const int rows = P * N;
    const int NPC = a.npc;                  // pencils per CTA = N^2 / (2 C), even
    // the launch shape this layout needs (the same for every CTA, so all return together): RPT
    // rows per team exactly, an even split of the pencils over the cluster
    if ((nt & 1) || nteam * RPT != rows || P * C != N || 2 * NPC * C != N * N || NPC % 2) {
        if (tid == 0) record_status(a.status, 2);       // EF_ERR_UNSUPPORTED
        return;
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2<T> *Is0 = reinterpret_cast<C2<T> *>(smem_raw);
    C2<T> *Is1 = Is0 + (size_t)P * NPP;
    C2<T> *Fs = Is1 + (size_t)P * NPP;                       // [z][local pencil] forward spectrum
    double *part = reinterpret_cast<double *>(Fs + (size_t)N * NPC);   // [32 warps + 1][kDiag]
    long long *s_cell = reinterpret_cast<long long *>(part + (32 + 1) * kDiag);
    int *s_nubig = reinterpret_cast<int *>(s_cell + 1);
    float *s_maxnu = reinterpret_cast<float *>(s_cell + 2);          // [32 warps] max nu of the loss op
    const uint32_t base0 = smem_u32addr(Is0), base1 = smem_u32addr(Is1);

    const unsigned long long pm = (0x100000000ull + (unsigned)P - 1u) / (unsigned)P;
    const int64_t nclusters = gridDim.x / C;
    const int64_t cid = blockIdx.x / C;
    const T scale = T(1) / T(CELL);
    const T *Mbase = reinterpret_cast<const T *>(a.mult);
    constexpr int H = N / 2 + 1;
    constexpr int NPT = N * H;              // multiplier table: [dir][k_z][k_y * H + k_x]

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

        // ---------------- F1: own rows real -> half complex, two rows per team transform
        for (int i0 = wteam; i0 < rows / 2; i0 += nteam) {
            const int it = i0 + (lane >> 1);
            const bool has = it < rows / 2;
            const unsigned mask = __ballot_sync(wmask, has);
            if (has) {
                const int r0 = it, r1 = it + rows / 2;
                const T *src0 = F + ((int64_t)rank * rows + r0) * N, *src1 = F + ((int64_t)rank * rows + r1) * N;
                C2<T> h[NH];
#pragma unroll
                for (int m = 0; m < NH; ++m) h[m] = C2<T>{__ldg(src0 + 2 * m + s), __ldg(src1 + 2 * m + s)};
                fft_team<N, -1>(h, s, mask);
                // lane 0 holds Z[k], lane 1 Z[N/2 + k]; X0[k] = (Z[k] + conj Z[N-k]) / 2 goes to row
                // r0 (lane 0), X1[k] = (Z[k] - conj Z[N-k]) / 2i to row r1 (lane 1)
                C2<T> *dst = (s ? Is0 + (r1 / N) * NPP : Is0 + (r0 / N) * NPP);
                const int y = s ? r1 % N : r0 % N;
                C2<T> prev;
                {
                    const float z0y = __shfl_xor_sync(mask, h[0].y, 1);      // lane 1 needs Im Z[0]
                    prev = C2<T>{s ? z0y : h[0].x, 0.f};
                }
                // the k values in pairs, stored as soon as a pair is complete (the exchange of
                // k reads h[k] and h[N/2 - k], which later k still need: nothing is overwritten)
#pragma unroll
                for (int k = 1; k < NH; ++k) {
                    const C2<T> send = s ? h[NH - k] : h[k];
                    C2<T> recv;
                    recv.x = __shfl_xor_sync(mask, send.x, 1);
                    recv.y = __shfl_xor_sync(mask, send.y, 1);
                    const C2<T> za = s ? recv : h[k];              // Z[k]
                    const C2<T> zb = s ? h[NH - k] : recv;         // Z[N - k]
                    const C2<T> xk = s ? C2<T>{T(0.5) * (za.y + zb.y), T(0.5) * (zb.x - za.x)}
                                       : C2<T>{T(0.5) * (za.x + zb.x), T(0.5) * (za.y - zb.y)};
                    if (k & 1)
                        *reinterpret_cast<float4 *>(dst + rg_at<N>(y, k - 1)) = make_float4(prev.x, prev.y, xk.x, xk.y);
                    else
                        prev = xk;
                }
            }
        }
        __syncthreads();
        for (int i0 = wteam; i0 < P * NH; i0 += nteam) {     // axis 1 forward, k_x < N/2
            const int it = i0 + (lane >> 1);
            const bool has = it < P * NH;
            const unsigned mask = __ballot_sync(wmask, has);
            if (has) {
                const int zl = it / NH, lx = it % NH;
                C2<T> *pl = Is0 + (size_t)zl * NPP;
                C2<T> h[NH];
#pragma unroll
                for (int m = 0; m < NH; ++m) h[m] = pl[rg_at<N>(2 * m + s, lx)];
                fft_team<N, -1>(h, s, mask);
#pragma unroll
                for (int k = 0; k < NH; ++k) pl[rg_at<N>(s * NH + k, lx)] = h[k];
            }
        }
        bar.full();

        // ---------------- F2: own pencils, gathered, axis 0 forward, kept in shared memory
        for (int i0 = wteam; i0 < NPC; i0 += nteam) {
            const int it = i0 + (lane >> 1);
            const bool has = it < NPC;
            const unsigned mask = __ballot_sync(wmask, has);
            if (has) {
                const int q = rank * NPC + it;
                const int poff = rg_poff<N>(q);
                C2<T> h[NH];
#pragma unroll
                for (int m = 0; m < NH; ++m) {
                    const int z = 2 * m + s;
                    const int owner = plane_owner(z, pm), zl = z - owner * P;
                    ld_cluster(cluster_map(base0 + (uint32_t)((zl * NPP + poff) * 8), owner), h[m]);
                }
                fft_team<N, -1>(h, s, mask);
#pragma unroll
                for (int k = 0; k < NH; ++k) Fs[(size_t)(s * NH + k) * NPC + it] = cscale(h[k], scale);
            }
        }
        bar.full();                        // Fs complete; every slab free again

        DiagF dg;
        T g[RPT][NH];                      // G of this lane's half of rows tm + j teams

        for (int o = 0; o < a.nops; ++o) {
            const Op op = a.ops[o];
            const bool pair = op.kind >= OP_PAIR;
            // ---------------- A: multiply, axis 0 inverse, scatter (one (direction, pencil) item
            // per team; the two teams of a lane quad hold adjacent pencils of one direction)
            const int nitems = (pair ? 2 : 1) * NPC;
            for (int i0 = wteam; i0 < nitems; i0 += nteam) {
                const int it = i0 + (lane >> 1);
                const bool has = it < nitems;
                const unsigned mask = __ballot_sync(wmask, has);
                if (has) {
                    const int b = it >= NPC;
                    const int ql = it - b * NPC;
                    const int q = rank * NPC + ql;
                    const int ky = q / NH, kx = q % NH;
                    const T *M = Mbase + (size_t)(b ? op.dir2 : op.dir) * N * NPT + ky * H + kx;
                    C2<T> h[NH];
#pragma unroll
                    for (int m = 0; m < NH; ++m) {
                        const int z = 2 * m + s;
                        h[m] = cscale(Fs[(size_t)z * NPC + ql], __ldg(M + (size_t)z * NPT));
                    }
                    fft_team<N, 1>(h, s, mask);
                    tm_scatter<N>(h, b ? base1 : base0, P, pm, rg_poff<N>(q & ~1), s, (lane >> 1) & 1, mask);
                }
            }
            bar.full();

            // ---------------- B: axis 1 inverse on the stored k_x < N/2 columns of each slab
            const int ncol = (pair ? 2 : 1) * P * NH;
            for (int i0 = wteam; i0 < ncol; i0 += nteam) {
                const int it = i0 + (lane >> 1);
                const bool has = it < ncol;
                const unsigned mask = __ballot_sync(wmask, has);
                if (has) {
                    const int b = it >= P * NH;
                    const int rem = it - b * P * NH;
                    const int zl = rem / NH, lx = rem % NH;
                    C2<T> *pl = (b ? Is1 : Is0) + (size_t)zl * NPP;
                    C2<T> h[NH];
#pragma unroll
                    for (int m = 0; m < NH; ++m) h[m] = pl[rg_at<N>(2 * m + s, lx)];
                    fft_team<N, 1>(h, s, mask);
#pragma unroll
                    for (int k = 0; k < NH; ++k) pl[rg_at<N>(s * NH + k, lx)] = h[k];
                }
            }
            __syncthreads();

            // ---------------- rows: half complex -> real, accumulate / output (every team has
            // exactly RPT rows, so every existing lane of a warp takes part)
            const unsigned full = wmask;
            if (pair) {
                const bool last = op.kind == OP_PAIR_LAST;
                const bool big = *s_nubig != 0;
                if (last) dg.reset();
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int r = tm + j * nteam;
                    const int rb = (r / N) * NPP;
                    C2<T> h[NH];
                    tm_c2r_load<N, true>(Is0 + rb, r % N, Is1 + rb, r % N, s, h);
                    fft_team<N, 1>(h, s, full);
                    if (!last) {
#pragma unroll
                        for (int n = 0; n < NH; ++n) g[j][n] += h[n].x * h[n].y;
                    } else {
                        T qv[NH];
#pragma unroll
                        for (int n = 0; n < NH; ++n) qv[n] = g[j][n] + h[n].x * h[n].y;
                        const int64_t grow = (int64_t)rank * rows + r;
                        T fr[NH];
                        load_row<T, NH>(F + grow * N + s * NH, fr);
                        tm_emit_half<N>(a, fr, Out + grow * N + s * NH, qv, big, grow, s * NH, dg);
                    }
                }
            } else {
                // the loss (first op): nu of the rows, G = -F nu; with two rows per team both share
                // one complex transform, with one the second input is zero
                bool bigt = false;
                T mxt = T(-3.0e38);
                C2<T> h[NH];
                int r0 = tm, r1 = tm;
                if constexpr (RPT == 2) {
                    r1 = tm + nteam;
                    tm_c2r_load<N, true>(Is0 + (r0 / N) * NPP, r0 % N, Is0 + (r1 / N) * NPP, r1 % N, s, h);
                } else {
                    tm_c2r_load<N, false>(Is0 + (r0 / N) * NPP, r0 % N, Is0, 0, s, h);
                }
                fft_team<N, 1>(h, s, full);
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int r = j ? r1 : r0;
                    T fr[NH];
                    load_row<T, NH>(F + ((int64_t)rank * rows + r) * N + s * NH, fr);
                    T mx = j ? h[0].y : h[0].x;
#pragma unroll
                    for (int n = 0; n < NH; ++n) {
                        const T nu = j ? h[n].y : h[n].x;
                        g[j][n] = -fr[n] * nu;
                        mx = nu > mx ? nu : mx;
                        if (T(a.dt) * nu > T(1)) bigt = true;
                    }
                    mxt = mx > mxt ? mx : mxt;
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
