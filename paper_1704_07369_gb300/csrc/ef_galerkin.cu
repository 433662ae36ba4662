// ef_galerkin.cu -- the Fourier Galerkin method (FGM) on the GPU, the comparison method of the
// paper's Fig. 2 (Sec. 1.2, eq. FGM_Q; fast form eq. fastFGM with zero padding).
//
// FGM keeps the mode set K = {-(N/2 - 1), ..., N/2 - 1}^d of the N grid and sums the quadratic
// form without aliasing: Qh^G_k = sum_{l + m = k} (B(l,m) - B(m,m)) Fh_l Fh_m over l, m in K.  The
// fast algorithm evaluates it by zero padding: on the grid of 2N points per axis the products of
// functions band-limited to K never wrap (|l + m| <= N - 2 < N), so
//   1. F is interpolated from the N grid to the 2N grid (the trigonometric interpolant on K);
//   2. the collision kernel of the 2N grid runs with multiplier tables restricted to K (gain and
//      loss as products on the 2N grid, the same kernels as ef_collide);
//   3. the result is projected back onto K and evaluated on the N grid.
// Steps 1 and 3 are separable: one small real matrix per axis (2N x N and N x 2N), applied by a
// direct-sum kernel.  The initial data are the grid values (the interpolation "I" of Fig. 2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "ef.h"
#include "ef_launch.h"

struct ef_galerkin_s {
    ef_plan_t plan2 = nullptr;     // the 2N-grid plan with restricted multipliers
    int d = 3, N = 0, prec = 0;
    int64_t max_cells = 0;
    size_t el = 4;
    void *A = nullptr, *B = nullptr, *C = nullptr;   // scratch: max_cells (2N)^d values each
    void *Sup = nullptr, *Sdn = nullptr;             // [2N][N] and [N][2N] in the plan's precision
    int device = 0;
};

namespace {

ef_status gfail(ef_status s, const std::string &m)
{
    ef::set_last_error(m.c_str());
    return s;
}

ef_status gcuda(cudaError_t e, const char *what)
{
    const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    ef::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

void gfree(ef_galerkin_s *g)
{
    if (!g) return;
    if (g->plan2) ef_plan_destroy(g->plan2);
    cudaFree(g->A);
    cudaFree(g->B);
    cudaFree(g->C);
    cudaFree(g->Sup);
    cudaFree(g->Sdn);
    delete g;
}

// out[c][..., i, ...] = sum_j S[i][j] in[c][..., j, ...] along `axis` of a per-cell array whose
// dimensions are dims_in (the output has dims_in[axis] replaced by mo)
template <typename T>
__global__ void apply_axis_kernel(const T *in, T *out, const T *S, int64_t ncells, int d, int axis, int n0, int n1,
                                  int n2, int mo)
{
    const int din[3] = {n0, n1, n2};
    int dout[3] = {n0, n1, n2};
    dout[axis] = mo;
    const int mi = din[axis];
    const int64_t per_out = (int64_t)dout[0] * dout[1] * (d == 3 ? dout[2] : 1);
    const int64_t per_in = (int64_t)din[0] * din[1] * (d == 3 ? din[2] : 1);
    const int64_t total = ncells * per_out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / per_out;
        int64_t r = t % per_out;
        int idx[3] = {0, 0, 0};
        for (int a = d - 1; a >= 0; --a) {
            idx[a] = (int)(r % dout[a]);
            r /= dout[a];
        }
        const int io = idx[axis];
        int64_t base = 0, stride = 1;
        for (int a = d - 1; a >= 0; --a) {
            if (a == axis) {
                stride = 1;
                for (int b = d - 1; b > a; --b) stride *= din[b];
            } else {
                int64_t s = 1;
                for (int b = d - 1; b > a; --b) s *= din[b];
                base += (int64_t)idx[a] * s;
            }
        }
        const T *src = in + c * per_in + base;
        const T *row = S + (int64_t)io * mi;
        T acc = T(0);
        for (int j = 0; j < mi; ++j) acc += row[j] * src[(int64_t)j * stride];
        out[t] = acc;
    }
}

template <typename T>
cudaError_t apply_axes(const ef_galerkin_s *g, const void *in, void *out, void *tmp0, void *tmp1, int64_t ncells,
                       bool up, cudaStream_t s)
{
    const int N = g->N, d = g->d;
    int dims[3] = {N, N, d == 3 ? N : 1};
    if (d == 2) dims[2] = 1;
    const int from = up ? N : 2 * N, to = up ? 2 * N : N;
    for (int a = 0; a < d; ++a) dims[a] = from;
    const T *S = static_cast<const T *>(up ? g->Sup : g->Sdn);
    const void *src = in;
    for (int a = d - 1; a >= 0; --a) {
        void *dst = (a == 0) ? out : ((a % 2) ? tmp0 : tmp1);
        int64_t per = 1;
        for (int b = 0; b < d; ++b) per *= (b == a ? to : dims[b]);
        const int64_t total = ncells * per;
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
        apply_axis_kernel<T><<<blocks, threads, 0, s>>>(static_cast<const T *>(src), static_cast<T *>(dst), S, ncells, d, a,
                                                        dims[0], dims[1], d == 3 ? dims[2] : 1, to);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dims[a] = to;
        src = dst;
    }
    return cudaSuccess;
}

// S_up[i'][j] = (1/N) sum_{k in K_1} exp(i pi k (x'_i' - x_j) / T): interpolation from the N grid
// (x_j = (j - N/2) 2T/N) to the 2N grid (x'_i' = (i' - N) T/N) on the modes |k| <= N/2 - 1;
// S_dn[j][i'] = S_up[i'][j] / 2 is the projection back (the 2N-grid DFT restricted to K_1).
void make_matrices(int N, std::vector<double> &up, std::vector<double> &dn)
{
    const double pi = 3.14159265358979323846264338327950288;
    const int n = N / 2 - 1;
    up.assign((size_t)2 * N * N, 0.0);
    dn.assign((size_t)2 * N * N, 0.0);
    for (int ip = 0; ip < 2 * N; ++ip)
        for (int j = 0; j < N; ++j) {
            // pi k (x' - x) / T = 2 pi k (ip - N - 2 (j - N/2)) / (2N) = pi k (ip - 2 j) / N
            double v = 1.0;
            for (int k = 1; k <= n; ++k) v += 2.0 * std::cos(pi * k * (double)(ip - 2 * j) / N);
            up[(size_t)ip * N + j] = v / N;
            dn[(size_t)j * 2 * N + ip] = v / (2.0 * N);
        }
}

}  // namespace

extern "C" {

ef_status ef_galerkin_create(const ef_plan_desc *desc, int64_t max_cells, ef_galerkin_t *out)
{
    if (!out) return gfail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (!desc || max_cells < 1) return gfail(EF_ERR_INVALID_ARG, "need a plan description and max_cells >= 1");
    ef_galerkin_s *g = new ef_galerkin_s();
    g->d = desc->d;
    g->N = desc->N;
    g->prec = desc->prec;
    g->max_cells = max_cells;
    g->el = desc->prec == EF_PREC_F32 ? 4 : 8;
    cudaGetDevice(&g->device);
    ef_status st = ef::plan_create_padded(desc, &g->plan2);
    if (st != EF_OK) { gfree(g); return st; }
    const int64_t per = g->d == 3 ? (int64_t)8 * g->N * g->N * g->N : (int64_t)4 * g->N * g->N;
    cudaError_t e = cudaMalloc(&g->A, (size_t)max_cells * per * g->el);
    if (e == cudaSuccess) e = cudaMalloc(&g->B, (size_t)max_cells * per * g->el);
    if (e == cudaSuccess) e = cudaMalloc(&g->C, (size_t)max_cells * per * g->el);
    std::vector<double> up, dn;
    make_matrices(g->N, up, dn);
    if (e == cudaSuccess) e = cudaMalloc(&g->Sup, up.size() * g->el);
    if (e == cudaSuccess) e = cudaMalloc(&g->Sdn, dn.size() * g->el);
    if (e == cudaSuccess) {
        if (g->el == 8) {
            e = cudaMemcpy(g->Sup, up.data(), up.size() * 8, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(g->Sdn, dn.data(), dn.size() * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> uf(up.begin(), up.end()), df(dn.begin(), dn.end());
            e = cudaMemcpy(g->Sup, uf.data(), uf.size() * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(g->Sdn, df.data(), df.size() * 4, cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) { gfree(g); return gcuda(e, "galerkin buffers"); }
    *out = g;
    return EF_OK;
}

ef_status ef_galerkin_collide(ef_galerkin_t g, const void *F_dev, void *Q_dev, int64_t ncells, ef_stream_t stream)
{
    if (!g) return gfail(EF_ERR_INVALID_ARG, "null galerkin object");
    if (ncells < 0 || ncells > g->max_cells) return gfail(EF_ERR_INVALID_ARG, "ncells outside [0, max_cells]");
    if (ncells == 0) return EF_OK;
    if (!F_dev || !Q_dev) return gfail(EF_ERR_INVALID_ARG, "null F or Q");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) return gfail(EF_ERR_INVALID_ARG, "the object's device is not current");
    cudaStream_t s = (cudaStream_t)stream;
    // F (N grid) -> A (2N grid); collide A -> C; C -> Q (N grid); B and the free buffer are scratch
    cudaError_t e = g->el == 8 ? apply_axes<double>(g, F_dev, g->A, g->B, g->C, ncells, true, s)
                               : apply_axes<float>(g, F_dev, g->A, g->B, g->C, ncells, true, s);
    if (e != cudaSuccess) return gcuda(e, "galerkin interpolation");
    ef_status st = ef_collide(g->plan2, g->A, g->C, ncells, stream);
    if (st != EF_OK) return st;
    e = g->el == 8 ? apply_axes<double>(g, g->C, Q_dev, g->A, g->B, ncells, false, s)
                   : apply_axes<float>(g, g->C, Q_dev, g->A, g->B, ncells, false, s);
    if (e != cudaSuccess) return gcuda(e, "galerkin projection");
    return EF_OK;
}

ef_status ef_galerkin_status(ef_galerkin_t g, int sync, int reset)
{
    if (!g) return gfail(EF_ERR_INVALID_ARG, "null galerkin object");
    return ef_plan_status(g->plan2, sync, reset);
}

ef_status ef_galerkin_destroy(ef_galerkin_t g)
{
    if (!g) return gfail(EF_ERR_INVALID_ARG, "null galerkin object");
    gfree(g);
    return EF_OK;
}

}  // extern "C"
