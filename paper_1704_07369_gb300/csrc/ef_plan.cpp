// ef_plan.cpp -- host side of the C ABI in include/ef.h: plan construction (filter, angular
// quadrature, radial kernel factors, multiplier tables, op lists), cluster / block shape choice,
// argument checks and kernel launches.
//
// The multiplier table of spectral direction u holds M_u(l) = sigma_N(l) Phi_u(l . e_u) for every
// mode l of the half spectrum (FP64 on the host, stored in the plan's precision), where Phi_u is
// the radial factor of the low-rank kernel decomposition (Sec. 4.1, eq. fastAlg):
//   2D Maxwell      psi_R(x) = 2 R sinc(pi R x / T)                        (eq. discrete_hatB)
//   3D hard sphere  phi(x)   = R^2 [2 sinc(pi R x/T) - sinc^2(pi R x/(2T))]
//   3D Maxwell      phi_j(x) = 2 int_0^R rho exp(-u_j^2 rho^2) cos(pi rho x / T) d rho
// The gain is sum over pairs (u, u*) of w a_u a_u*, a_u = IFFT(M_u Fhat); the loss table is
// L(m) = sum_pairs w M_u(m) M_u*(m) = sigma(m)^2 B_fast(m, m) (eq. def_A).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "ef.h"
#include "ef_internal.h"
#include "ef_launch.h"

namespace {

thread_local std::string g_last_error;

ef_status fail(ef_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

ef_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- plan math ---------------

// Modified Jackson filter (eq. JacksonFilter2) with n = N/2 for even N; sigma(-N/2) = 0 (Sec. 4.1).
double jackson(int N, int k, bool enabled)
{
    if (k == -N / 2) return 0.0;
    if (!enabled) return 1.0;
    const int n = N / 2;
    const int b = std::abs(k);
    if (b >= n) return 0.0;
    const double np1 = n + 1.0;
    const double t = kPi * b / np1, c = kPi / np1;
    return ((np1 - b) * std::cos(t) + std::sin(t) * std::cos(c) / std::sin(c)) / np1;
}

double sinc(double y) { return std::fabs(y) < 1e-8 ? 1.0 - y * y / 6.0 : std::sin(y) / y; }

// Gauss-Legendre nodes / weights on [-1, 1] (Newton on the three-term recurrence).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

template <class Fn>
void parallel_for(int64_t n, Fn fn)
{
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 4096) nt = 1;
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        for (;;) {
            const int64_t b = next.fetch_add(1024);
            if (b >= n) break;
            const int64_t e = std::min(n, b + 1024);
            for (int64_t i = b; i < e; ++i) fn(i);
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(worker);
    worker();
    for (auto &t : th) t.join();
}

// Radial profile of one direction.
struct Profile {
    int type;        // 0: 2D psi, 1: 3D hard sphere phi, 2: 3D Maxwell Gaussian-damped phi
    double u;        // Gaussian rate (type 2)
};

struct Dir {
    double e[3];
    Profile prof;
};

struct Pair {
    int de, ds;      // gain term w * a_de * a_ds
    double w;
};

struct Desc {
    int d, N, R, nmu, nphi, nc, J, sigma;
    double L, T, Rtr;
    ef_kernel kernel;
    ef_precision prec;
    int gal_N = 0;      // > 0: a zero-padded Galerkin plan (grid N = 2 gal_N) whose multipliers keep
                        // only the modes of the gal_N grid's set K (|k_a| <= gal_N/2 - 1)
};

// Directions and gain pairs of the low-rank kernel (independent of N).
void build_directions(const Desc &ds, std::vector<Dir> &dirs, std::vector<Pair> &pairs)
{
    dirs.clear();
    pairs.clear();
    if (ds.d == 2) {
        // theta_t = t pi / R over [0, pi); e_t^perp = e_{t + R/2}; weight (1/pi)(pi/R) per term,
        // each unordered pair appearing twice in sum_t.
        for (int t = 0; t < ds.R; ++t) {
            const double th = kPi * t / ds.R;
            dirs.push_back(Dir{{std::cos(th), std::sin(th), 0.0}, Profile{0, 0.0}});
        }
        for (int t = 0; t < ds.R / 2; ++t) pairs.push_back(Pair{t, t + ds.R / 2, 2.0 / ds.R});
        return;
    }
    // 3D: e on the half sphere (Gauss-Legendre in mu = cos(polar) on [0,1], uniform azimuth),
    // e* on the half circle orthogonal to e; weight (1/pi) w_mu (2 pi / n_phi) (pi / n_c).
    std::vector<double> gx, gw;
    gauss_legendre(ds.nmu, gx, gw);
    std::vector<double> uj, cj;
    if (ds.kernel == EF_KERNEL_MAXWELL) {
        // 1/sqrt(s) = (2/sqrt(pi)) int_0^inf exp(-u^2 s) du; u = exp(tau), tau in
        // [ln(0.4/R), ln(35/R)] by (J-1)-point Gauss-Legendre, plus one u = 0 term for the rest.
        const int n = ds.J - 1;
        std::vector<double> tx, tw;
        if (n > 0) gauss_legendre(n, tx, tw);
        const double ta = std::log(0.4 / ds.Rtr), tb = std::log(35.0 / ds.Rtr);
        uj.push_back(0.0);
        cj.push_back(2.0 / std::sqrt(kPi) * std::exp(ta));
        for (int j = 0; j < n; ++j) {
            const double tau = ta + 0.5 * (tx[j] + 1.0) * (tb - ta);
            uj.push_back(std::exp(tau));
            cj.push_back(2.0 / std::sqrt(kPi) * 0.5 * (tb - ta) * tw[j] * std::exp(tau));
        }
    } else {
        uj.push_back(0.0);
        cj.push_back(1.0);
    }
    for (size_t j = 0; j < uj.size(); ++j) {
        const Profile pr{ds.kernel == EF_KERNEL_MAXWELL ? 2 : 1, uj[j]};
        for (int a = 0; a < ds.nmu; ++a) {
            const double mu = 0.5 * (gx[a] + 1.0), wmu = 0.5 * gw[a];
            const double st = std::sqrt(1.0 - mu * mu);
            for (int b = 0; b < ds.nphi; ++b) {
                const double al = 2.0 * kPi * b / ds.nphi;
                const double ev[3] = {st * std::cos(al), st * std::sin(al), mu};
                const double uv[3] = {mu * std::cos(al), mu * std::sin(al), -st};
                const double vv[3] = {-std::sin(al), std::cos(al), 0.0};
                const int de = (int)dirs.size();
                dirs.push_back(Dir{{ev[0], ev[1], ev[2]}, pr});
                for (int c = 0; c < ds.nc; ++c) {
                    const double ph = kPi * c / ds.nc;
                    Dir es{{std::cos(ph) * uv[0] + std::sin(ph) * vv[0], std::cos(ph) * uv[1] + std::sin(ph) * vv[1],
                            std::cos(ph) * uv[2] + std::sin(ph) * vv[2]},
                           pr};
                    const int dsi = (int)dirs.size();
                    dirs.push_back(es);
                    const double w = (1.0 / kPi) * wmu * (2.0 * kPi / ds.nphi) * (kPi / ds.nc) * cj[j];
                    pairs.push_back(Pair{de, dsi, w});
                }
            }
        }
    }
}

// radial factor Phi(x), x = l . e
struct RadialEval {
    double T, Rtr;
    std::vector<double> rho, wr;   // composite Gauss-Legendre on [0, R]: 16 panels x 8 nodes
    RadialEval(double T_, double R_) : T(T_), Rtr(R_)
    {
        std::vector<double> gx, gw;
        gauss_legendre(8, gx, gw);
        const double hp = Rtr / 16.0;
        for (int p = 0; p < 16; ++p)
            for (int i = 0; i < 8; ++i) {
                rho.push_back(hp * (p + 0.5 * (gx[i] + 1.0)));
                wr.push_back(0.5 * hp * gw[i]);
            }
    }
    double operator()(const Profile &pr, double x) const
    {
        if (pr.type == 0) return 2.0 * Rtr * sinc(kPi * Rtr * x / T);
        if (pr.type == 1) {
            const double a = kPi * x / T, s2 = sinc(0.5 * a * Rtr);
            return Rtr * Rtr * (2.0 * sinc(a * Rtr) - s2 * s2);
        }
        const double a = kPi * x / T;
        double acc = 0.0;
        for (size_t i = 0; i < rho.size(); ++i)
            acc += wr[i] * rho[i] * std::exp(-pr.u * pr.u * rho[i] * rho[i]) * std::cos(a * rho[i]);
        return 2.0 * acc;
    }
};

int mode_of(int N, int i) { return i < N / 2 ? i : i - N; }

// ---------------------------------------------------------------- plan objects -------------

struct ClassPlan {
    int N = 0;
    int64_t ncells = 0;                 // batched: cells of this size; uniform plan: 0
    int cluster = 1, tpb = 32, planes = 0, sg_global = 0, prefetch = 1, paired = 0, occ = 1;
    double tuned_ms = 0.0;              // autotuner's best time (0 when not tuned)
    size_t smem = 0;
    int max_clusters = 0;
    int ndir = 0, nops = 0;              // op count of the active mode
    int nfeat = 0;                       // complex feature modes
    int nops_single = 0, nops_paired = 0;
    void *d_mult = nullptr;
    ef::Op *d_ops = nullptr;             // active op list (points into one of the two below)
    ef::Op *d_ops_single = nullptr, *d_ops_paired = nullptr;
    int *d_modes = nullptr;              // band modes [nfeat][3] (|k| <= EF_FEATURE_K), feature slot order
    int64_t *d_cell_off = nullptr, *d_cell_id = nullptr;
    void *d_sg = nullptr;
    int64_t sg_slots = 0;
    void *d_fh = nullptr;                // forward-spectrum workspace, fh_slots clusters
    int64_t fh_slots = 0;
};

}  // namespace

struct ef_plan_s {
    Desc desc;
    // concurrent size classes: one internal stream, event and cell counter per class
    std::vector<cudaStream_t> cstreams;
    std::vector<cudaEvent_t> cevents;
    cudaEvent_t fork = nullptr;
    unsigned long long *d_counters = nullptr;
    int device = 0;
    bool batched = false;
    int64_t ncells = 0;
    std::vector<ClassPlan> classes;
    int64_t *d_all_off = nullptr, *d_all_N = nullptr;
    int *d_status = nullptr;
    int h_status = 0;
    bool use_graph = false;
    // graph cache: one captured step per (mode, F, Q, ncells, dt, diag, stream)
    cudaGraphExec_t gexec = nullptr;
    const void *g_F = nullptr;
    void *g_Q = nullptr;
    int64_t g_n = -1;
    int g_mode = -1;
    double g_dt = 0.0;
    double *g_diag = nullptr;
    cudaStream_t g_stream = nullptr;
    // SSP-RK3 stage buffers: two batch-sized arrays, grown on demand
    void *d_rk = nullptr;
    size_t rk_bytes = 0;
};

namespace {

bool size_built(int prec, int d, int N)
{
    if (prec == EF_PREC_F32) return d == 3 ? ef::collide_supported_f32_3d(N) : ef::collide_supported_f32_2d(N);
    return d == 3 ? ef::collide_supported_f64_3d(N) : ef::collide_supported_f64_2d(N);
}

int maxthreads_for(int prec, int d, int N, int occ)
{
    if (prec == EF_PREC_F32) return d == 3 ? ef::collide_maxthreads_f32_3d(N, occ) : ef::collide_maxthreads_f32_2d(N, occ);
    return d == 3 ? ef::collide_maxthreads_f64_3d(N, occ) : ef::collide_maxthreads_f64_2d(N, occ);
}

size_t smem_for(int prec, int d, int N, int planes, int sg, int paired, int occ = 1)
{
    if (prec == EF_PREC_F32)
        return d == 3 ? ef::collide_smem_f32_3d(N, planes, sg, paired, occ) : ef::collide_smem_f32_2d(N, planes, sg, paired, occ);
    return d == 3 ? ef::collide_smem_f64_3d(N, planes, sg, paired, occ) : ef::collide_smem_f64_2d(N, planes, sg, paired, occ);
}

cudaError_t setup_for(int prec, int d, int N, size_t smem, int cl, int tpb, int occ, int *mc)
{
    if (prec == EF_PREC_F32)
        return d == 3 ? ef::collide_setup_f32_3d(N, smem, cl, tpb, occ, mc) : ef::collide_setup_f32_2d(N, smem, cl, tpb, occ, mc);
    return d == 3 ? ef::collide_setup_f64_3d(N, smem, cl, tpb, occ, mc) : ef::collide_setup_f64_2d(N, smem, cl, tpb, occ, mc);
}

cudaError_t launch_for(int prec, int d, int N, const ef::CollideArgs &a, int grid, int tpb, size_t smem, int occ,
                       cudaStream_t s)
{
    if (prec == EF_PREC_F32)
        return d == 3 ? ef::collide_launch_f32_3d(N, a, grid, tpb, smem, occ, s)
                      : ef::collide_launch_f32_2d(N, a, grid, tpb, smem, occ, s);
    return d == 3 ? ef::collide_launch_f64_3d(N, a, grid, tpb, smem, occ, s)
                  : ef::collide_launch_f64_2d(N, a, grid, tpb, smem, occ, s);
}

struct Shape {
    int cluster, tpb, planes, sg_global, paired, occ;
    size_t smem;
    int max_clusters;
};

// Every launch shape that fits one N: cluster sizes C | N with an even number of real rows per
// CTA; threads per CTA enough for one work item each of the widest stage (the stage-A (direction,
// pencil) items, the axis-1 columns or the row pairs), or half of that (two rounds), at most the
// instantiation's thread limit; shared memory within the device's opt-in limit (S/G in global
// memory only when nothing fits otherwise) and at least one co-resident cluster.
std::vector<Shape> candidate_shapes(const Desc &ds, int N, std::string &why)
{
    const int d = ds.d;
    const int H = N / 2 + 1, N1 = d == 3 ? N : 1, NP = N1 * H;
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int cands[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
    std::vector<Shape> out;
    // FP32 3D: the register-accumulator kernel first (one or two rows per thread, threads = rows / RPT)
    if (ds.prec == EF_PREC_F32 && d == 3) {
        for (int C : cands) {
            if (N % C || ef::collide_npc_v(d, N, C, 3) == 0) continue;
            const int planes = N / C, rows = planes * N;
            for (int v = 1; v <= 6; ++v) {
                const int occ = 2 + v;
                const int rpt = ef::rg_rows_per_thread(v);
                const int team = ef::rg_team(v);
                const int tmax = maxthreads_for(ds.prec, d, N, occ);
                if (tmax == 0) continue;
                // G in registers: exactly rows / rpt threads; in shared memory: one or two rows each
                for (int per = (rpt ? rpt : 1); per <= (rpt ? rpt : 2); ++per) {
                    if (rows % per) continue;
                    const int tpb = rows * team / per;
                    if (tpb > tmax || tpb < 32) continue;
                    const size_t smem = smem_for(ds.prec, d, N, planes, 0, 1, occ);
                    if ((long)smem > smem_max) continue;
                    int mc = 0;
                    cudaError_t e = setup_for(ds.prec, d, N, smem, C, tpb, occ, &mc);
                    if (e != cudaSuccess) {
                        cudaGetLastError();
                        why = cudaGetErrorString(e);
                        continue;
                    }
                    if (mc <= 0) continue;
                    out.push_back(Shape{C, tpb, planes, 0, 1, occ, smem, mc});
                }
            }
        }
    }
    const size_t n_rg = out.size();
    for (int sg = 0; sg <= 1 && out.size() == n_rg; ++sg) {
        for (int paired = 1; paired >= 0; --paired) {
            for (int C : cands) {
                if (N % C) continue;
                const int planes = N / C;
                const int rows = planes * N1;
                if (rows % 2) continue;
                const int nb = paired ? 2 : 1;
                const int need = std::max({nb * ef::collide_npc(d, N, C), paired ? rows : rows / 2,
                                           d == 3 ? nb * planes * H : 1});
                const size_t smem = smem_for(ds.prec, d, N, planes, sg, paired, 1);
                if ((long)smem > smem_max) continue;
                for (int occ = 1; occ <= 2; ++occ) {
                    const int tmax = maxthreads_for(ds.prec, d, N, occ);
                    int last = 0;
                    for (int rounds = 1; rounds <= 2; ++rounds) {
                        const int tpb = std::max(64, ((need + rounds - 1) / rounds + 31) / 32 * 32);
                        if (tpb > tmax || tpb == last) continue;
                        last = tpb;
                        int mc = 0;
                        cudaError_t e = setup_for(ds.prec, d, N, smem, C, tpb, occ, &mc);
                        if (e != cudaSuccess) {
                            cudaGetLastError();
                            why = cudaGetErrorString(e);
                            continue;
                        }
                        if (mc <= 0) continue;
                        out.push_back(Shape{C, tpb, planes, sg, paired, occ, smem, mc});
                    }
                }
            }
        }
    }
    return out;
}

void apply_shape(ClassPlan &cp, const Shape &sh)
{
    cp.cluster = sh.cluster;
    cp.tpb = sh.tpb;
    cp.planes = sh.planes;
    cp.sg_global = sh.sg_global;
    cp.paired = sh.paired;
    cp.occ = sh.occ;
    cp.smem = sh.smem;
    cp.max_clusters = sh.max_clusters;
    cp.d_ops = sh.paired ? cp.d_ops_paired : cp.d_ops_single;
    cp.nops = sh.paired ? cp.nops_paired : cp.nops_single;
}

std::string device_key()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string k = prop.name;
    for (char &c : k)
        if (c == ' ') c = '_';
    return k + "_sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "_" + std::to_string(prop.multiProcessorCount);
}

// The cache key: device, discretisation and a bucket of the class's cell count (64, 256, 1024 or
// more: the best shape for a few dozen cells, as in the chunks of a stream plan, is not the best for
// a thousand).
std::string tune_key(const Desc &ds, int N, int64_t ncells)
{
    char buf[256];
    int bucket = 64;
    while (bucket < 4096 && bucket < ncells) bucket *= 4;
    // "v5": kernel layout generation (variants 3 - 8: register-accumulator kernels, 7 / 8 the team ones)
    std::snprintf(buf, sizeof(buf), "v5 %s p%d d%d N%d k%d R%d J%d a%d.%d.%d s%d b%d", device_key().c_str(), (int)ds.prec,
                  ds.d, N, (int)ds.kernel, ds.R, ds.J, ds.nmu, ds.nphi, ds.nc, ds.sigma, bucket);
    return buf;
}

bool cache_lookup(const std::string &key, int &C, int &tpb, int &sg, int &pf, int &pr, int &occ)
{
    const char *path = std::getenv("EF_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        std::string ln(line);
        const size_t bar = ln.find('|');
        if (bar == std::string::npos || ln.substr(0, bar) != key) continue;
        if (std::sscanf(ln.c_str() + bar + 1, "%d %d %d %d %d %d", &C, &tpb, &sg, &pf, &pr, &occ) == 6) found = true;
    }
    std::fclose(f);
    return found;
}

void cache_store(const std::string &key, int C, int tpb, int sg, int pf, int pr, int occ, double ms)
{
    const char *path = std::getenv("EF_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s|%d %d %d %d %d %d %.4f\n", key.c_str(), C, tpb, sg, pf, pr, occ, ms);
    std::fclose(f);
}

// Plan-time autotuner: time every candidate shape (and the L1 prefetch on / off), as an Euler step
// with the diagnostics, on a scratch batch of up to 512 cells, then the three fastest again on a batch of ncells_tune cells (the size
// class's own count, up to 2048: the tail of the last round of clusters and the packing of clusters
// on the SMs depend on it), and keep the fastest of those.  Results are cached per device and
// discretisation in the file named by EF_AUTOTUNE_CACHE when it is set; EF_AUTOTUNE=0 skips the
// timing and takes the smallest cluster.
ef_status choose_shape(const Desc &ds, ClassPlan &cp, int64_t ncells_tune)
{
    std::string why;
    std::vector<Shape> shapes = candidate_shapes(ds, cp.N, why);
    if (shapes.empty())
        return fail(EF_ERR_UNSUPPORTED, "no launch shape fits N=" + std::to_string(cp.N) + " on this device " + why);
    apply_shape(cp, shapes[0]);
    cp.prefetch = 0;
    // EF_SHAPE="N:cluster:threads:variant[,...]" pins the launch shape of size N (tests, experiments);
    // an entry that matches no candidate shape is ignored
    if (const char *pin = std::getenv("EF_SHAPE")) {
        std::string spec(pin);
        size_t pos = 0;
        while (pos < spec.size()) {
            size_t end = spec.find(',', pos);
            if (end == std::string::npos) end = spec.size();
            int n = 0, C = 0, tpb = 0, occ = 0;
            if (std::sscanf(spec.substr(pos, end - pos).c_str(), "%d:%d:%d:%d", &n, &C, &tpb, &occ) == 4 && n == cp.N) {
                for (const Shape &sh : shapes)
                    if (sh.cluster == C && sh.tpb == tpb && sh.occ == occ && sh.sg_global == 0) {
                        apply_shape(cp, sh);
                        return EF_OK;
                    }
            }
            pos = end + 1;
        }
    }
    const char *env = std::getenv("EF_AUTOTUNE");
    const bool tune = ncells_tune > 0 && !(env && env[0] == '0') && shapes.size() > 1;
    if (!tune) return EF_OK;
    const std::string key = tune_key(ds, cp.N, ncells_tune);
    int C = 0, tpb = 0, sg = 0, pf = 1, pr = 0, occ = 1;
    if (cache_lookup(key, C, tpb, sg, pf, pr, occ)) {
        for (const Shape &sh : shapes)
            if (sh.cluster == C && sh.tpb == tpb && sh.sg_global == sg && sh.paired == pr && sh.occ == occ) {
                apply_shape(cp, sh);
                cp.prefetch = pf;
                return EF_OK;
            }
    }
    const int d = ds.d;
    const int64_t cell = d == 3 ? (int64_t)cp.N * cp.N * cp.N : (int64_t)cp.N * cp.N;
    const size_t el = ds.prec == EF_PREC_F32 ? 4 : 8;
    void *F = nullptr, *Q = nullptr, *sgws = nullptr, *fhws = nullptr;
    double *dgws = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&F, ncells_tune * cell * el);
    if (e == cudaSuccess) e = cudaMalloc(&Q, ncells_tune * cell * el);
    if (e == cudaSuccess) e = cudaMemset(F, 0, ncells_tune * cell * el);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dgws, (size_t)ncells_tune * ef::kDiag * sizeof(double));
    int64_t fh_need = 0;
    for (const Shape &sh : shapes) fh_need = std::max<int64_t>(fh_need, std::min<int64_t>(ncells_tune, sh.max_clusters));
    if (e == cudaSuccess) e = cudaMalloc(&fhws, (size_t)fh_need * ef::collide_fh_bytes(ds.prec, d, cp.N));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e30;
    Shape best_sh = shapes[0];
    int best_pf = 0;
    struct Timed {
        double ms;
        size_t shape;
        int pf;
    };
    std::vector<Timed> sweep;
    auto time_one = [&](const Shape &sh, int pfv, int64_t nc, double &tmin) -> cudaError_t {
        const int grid = (int)std::min<int64_t>(nc, sh.max_clusters);
        ef::CollideArgs a{};
        a.F = F;
        a.Q = Q;
        a.ncells = nc;
        a.mult = cp.d_mult;
        a.ops = sh.paired ? cp.d_ops_paired : cp.d_ops_single;
        a.nops = sh.paired ? cp.nops_paired : cp.nops_single;
        a.paired = sh.paired;
        a.cluster = sh.cluster;
        a.planes = sh.planes;
        a.sg_global = sh.sg_global;
        a.sg_ws = sgws;
        a.fh_ws = fhws;
        a.npc = ef::collide_npc_v(d, cp.N, sh.cluster, sh.occ);
        // timed as the step runs it: the Euler output in place (dt = 0 leaves F unchanged) with the
        // per-cell diagnostics, which cost some shapes more than others
        a.Q = F;
        a.out_mode = ef::OUT_EULER;
        a.dt = 0.0;
        a.diag = dgws;
        a.h = 1.0;
        a.prefetch = pfv;
        tmin = 1e30;
        cudaError_t r = cudaSuccess;
        for (int rep = 0; rep < 4 && r == cudaSuccess; ++rep) {
            r = cudaEventRecord(e0, st);
            if (r == cudaSuccess) r = launch_for(ds.prec, d, cp.N, a, grid, sh.tpb, sh.smem, sh.occ, st);
            if (r == cudaSuccess) r = cudaEventRecord(e1, st);
            if (r == cudaSuccess) r = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, (double)ms);
        }
        return r;
    };
    const int64_t n1 = std::min<int64_t>(ncells_tune, 512);
    for (size_t i = 0; e == cudaSuccess && i < shapes.size(); ++i) {
        const Shape &sh = shapes[i];
        const int grid = (int)std::min<int64_t>(ncells_tune, sh.max_clusters);
        if (sh.sg_global) {
            const int64_t rows = (int64_t)sh.planes * (d == 3 ? cp.N : 1);
            cudaFree(sgws);
            sgws = nullptr;
            e = cudaMalloc(&sgws, (size_t)grid * sh.cluster * 2 * rows * cp.N * el);
            if (e != cudaSuccess) break;
        }
        for (int pfv = 0; pfv <= 1 && e == cudaSuccess; ++pfv) {
            double tmin = 1e30;
            e = time_one(sh, pfv, n1, tmin);
            if (e != cudaSuccess) break;
            sweep.push_back(Timed{tmin, i, pfv});
            // EF_AUTOTUNE_LOG names a file that receives every timed candidate (tuning records)
            if (const char *lp = std::getenv("EF_AUTOTUNE_LOG")) {
                if (FILE *lf = std::fopen(lp, "a")) {
                    std::fprintf(lf, "N=%d cells=%lld cluster=%d threads=%d variant=%d sg=%d paired=%d prefetch=%d ms=%.4f\n",
                                 cp.N, (long long)n1, sh.cluster, sh.tpb, sh.occ, sh.sg_global, sh.paired, pfv, tmin);
                    std::fclose(lf);
                }
            }
        }
        if (e != cudaSuccess) break;
    }
    // the three fastest of the sweep, again on the class's own count (global S/G shapes keep their
    // sweep time: their workspace is sized for the last swept shape only)
    std::sort(sweep.begin(), sweep.end(), [](const Timed &x, const Timed &y) { return x.ms < y.ms; });
    for (size_t j = 0; e == cudaSuccess && j < sweep.size() && j < 3; ++j) {
        const Shape &sh = shapes[sweep[j].shape];
        double tmin = sweep[j].ms * (double)ncells_tune / (double)n1;
        if (ncells_tune > n1 && !sh.sg_global) {
            e = time_one(sh, sweep[j].pf, ncells_tune, tmin);
            if (e != cudaSuccess) break;
            if (const char *lp = std::getenv("EF_AUTOTUNE_LOG")) {
                if (FILE *lf = std::fopen(lp, "a")) {
                    std::fprintf(lf, "N=%d cells=%lld cluster=%d threads=%d variant=%d sg=%d paired=%d prefetch=%d ms=%.4f\n",
                                 cp.N, (long long)ncells_tune, sh.cluster, sh.tpb, sh.occ, sh.sg_global, sh.paired,
                                 sweep[j].pf, tmin);
                    std::fclose(lf);
                }
            }
        }
        if (tmin < best) {
            best = tmin;
            best_sh = sh;
            best_pf = sweep[j].pf;
        }
    }
    cudaFree(F);
    cudaFree(Q);
    cudaFree(sgws);
    cudaFree(fhws);
    cudaFree(dgws);
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    apply_shape(cp, best_sh);
    cp.prefetch = best_pf;
    cp.tuned_ms = best;
    cache_store(key, best_sh.cluster, best_sh.tpb, best_sh.sg_global, best_pf, best_sh.paired, best_sh.occ, best);
    return EF_OK;
}

template <typename T>
void *upload_table(const std::vector<double> &h, cudaError_t &err)
{
    std::vector<T> t(h.size());
    for (size_t i = 0; i < h.size(); ++i) t[i] = (T)h[i];
    void *p = nullptr;
    err = cudaMalloc(&p, t.size() * sizeof(T));
    if (err != cudaSuccess) return nullptr;
    err = cudaMemcpy(p, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice);
    return p;
}

ef_status build_class(const Desc &ds, ClassPlan &cp)
{
    const int N = cp.N, d = ds.d;
    const int H = N / 2 + 1, N1 = d == 3 ? N : 1, NP = N1 * H;
    std::vector<Dir> dirs;
    std::vector<Pair> pairs;
    build_directions(ds, dirs, pairs);
    const int ndir = (int)dirs.size();
    const int64_t per = (int64_t)N * NP;
    std::vector<double> tab((size_t)(ndir + 1) * per, 0.0);
    std::vector<double> sig1(N);
    for (int i = 0; i < N; ++i) {
        const int k = mode_of(N, i);
        if (ds.gal_N > 0) sig1[i] = std::abs(k) <= ds.gal_N / 2 - 1 ? jackson(ds.gal_N, k, ds.sigma != 0) : 0.0;
        else sig1[i] = jackson(N, k, ds.sigma != 0);
    }
    RadialEval rad(ds.T, ds.Rtr);
    parallel_for((int64_t)ndir * per, [&](int64_t idx) {
        const int u = (int)(idx / per);
        const int64_t i = idx % per;
        const int lz = (int)(i / NP), p = (int)(i % NP);
        int k[3] = {mode_of(N, lz), 0, 0};
        double s = sig1[lz];
        if (d == 3) {
            const int ly = p / H, lx = p % H;
            k[1] = mode_of(N, ly);
            k[2] = lx < N / 2 ? lx : lx - N;
            s *= sig1[ly] * sig1[lx < N / 2 ? lx : N / 2];
        } else {
            const int lx = p;
            k[1] = lx < N / 2 ? lx : lx - N;
            s *= sig1[lx < N / 2 ? lx : N / 2];
        }
        double val = 0.0;
        if (s != 0.0) {
            const Dir &D0 = dirs[u];
            const double x = k[0] * D0.e[0] + k[1] * D0.e[1] + k[2] * D0.e[2];
            val = s * rad(D0.prof, x);
        }
        tab[(size_t)u * per + i] = val;
    });
    // Group the gain pairs by their first direction e: sum_c w_c a_e a_{e*_c} = a_e S_e with
    // S_e = IFFT(Gamma_e Fhat), Gamma_e = sum_c w_c M_{e*_c} (linearity of the inverse transform),
    // so each e costs two inverse transforms however many partners it has.
    std::map<int, std::vector<const Pair *>> groups;
    std::vector<int> order;
    for (const Pair &pr : pairs) {
        if (!groups.count(pr.de)) order.push_back(pr.de);
        groups[pr.de].push_back(&pr);
    }
    const int ne = (int)order.size();
    // output table rows: [0, ne) = M_e, [ne, 2 ne) = Gamma_e, 2 ne = loss
    std::vector<double> out((size_t)(2 * ne + 1) * per, 0.0);
    for (int g = 0; g < ne; ++g) {
        const int de = order[g];
        double *Me = &out[(size_t)g * per], *Ge = &out[(size_t)(ne + g) * per];
        std::memcpy(Me, &tab[(size_t)de * per], per * sizeof(double));
        for (const Pair *pr : groups[de])
            for (int64_t i = 0; i < per; ++i) Ge[i] += pr->w * tab[(size_t)pr->ds * per + i];
    }
    double *loss = &out[(size_t)(2 * ne) * per];      // L(m) = sigma(m)^2 B_fast(m, m)
    for (int g = 0; g < ne; ++g)
        for (int64_t i = 0; i < per; ++i) loss[i] += out[(size_t)g * per + i] * out[(size_t)(ne + g) * per + i];
    // single-slab op list: S = a(Gamma_e); G (+)= a(M_e) S; ...; Q = G - F nu
    std::vector<ef::Op> ops1, ops2;
    for (int g = 0; g < ne; ++g) {
        ops1.push_back(ef::Op{ne + g, ef::OP_S_SET, 1.0, 0, 0});
        ops1.push_back(ef::Op{g, g == 0 ? ef::OP_G_SET : ef::OP_G_ADD, 1.0, 0, 0});
    }
    ops1.push_back(ef::Op{2 * ne, ef::OP_LOSS, 1.0, 0, 0});
    // paired op list: G = -F nu; G += a(M_e) a(Gamma_e) for each e; the last pair writes Q
    ops2.push_back(ef::Op{2 * ne, ef::OP_NU_INIT, 1.0, 0, 0});
    for (int g = 0; g < ne; ++g)
        ops2.push_back(ef::Op{g, g + 1 == ne ? ef::OP_PAIR_LAST : ef::OP_PAIR, 1.0, ne + g, 0});
    if ((int)ops1.size() > ef::kMaxOps) return fail(EF_ERR_UNSUPPORTED, "too many spectral directions");
    tab.swap(out);
    cp.ndir = 2 * ne + 1;
    cp.nops_single = (int)ops1.size();
    cp.nops_paired = (int)ops2.size();

    cudaError_t e = cudaSuccess;
    cp.d_mult = ds.prec == EF_PREC_F32 ? upload_table<float>(tab, e) : upload_table<double>(tab, e);
    if (e != cudaSuccess) return cuda_fail(e, "multiplier table");
    e = cudaMalloc((void **)&cp.d_ops_single, ops1.size() * sizeof(ef::Op));
    if (e == cudaSuccess) e = cudaMalloc((void **)&cp.d_ops_paired, ops2.size() * sizeof(ef::Op));
    if (e != cudaSuccess) return cuda_fail(e, "op list");
    e = cudaMemcpy(cp.d_ops_single, ops1.data(), ops1.size() * sizeof(ef::Op), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cp.d_ops_paired, ops2.data(), ops2.size() * sizeof(ef::Op), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "op list copy");
    // feature slots: modes with |k| <= EF_FEATURE_K in the canonical half space (k2 > 0, or
    // k2 = 0 and k1 > 0, or k2 = k1 = 0 and k0 >= 0), in lexicographic order of (k0, k1, k2);
    // stored as (k_axis0, k_axis1, k_axis2) for 3D and (0, k0, k1) for 2D (k2 = 0)
    if (N / 2 > EF_FEATURE_K) {
        std::vector<int> modes;
        const int K = EF_FEATURE_K;
        for (int k0 = -K; k0 <= K; ++k0)
            for (int k1 = -K; k1 <= K; ++k1)
                for (int k2 = 0; k2 <= K; ++k2) {
                    if (k0 * k0 + k1 * k1 + k2 * k2 > K * K) continue;
                    if (!(k2 > 0 || (k2 == 0 && (k1 > 0 || (k1 == 0 && k0 >= 0))))) continue;
                    if (d == 2 && k2 != 0) continue;
                    if (d == 3) {
                        modes.push_back(k0);
                        modes.push_back(k1);
                        modes.push_back(k2);
                    } else {
                        modes.push_back(0);
                        modes.push_back(k0);
                        modes.push_back(k1);
                    }
                }
        e = cudaMalloc((void **)&cp.d_modes, modes.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(cp.d_modes, modes.data(), modes.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "feature table");
        cp.nfeat = (int)modes.size() / 3;
    }
    return choose_shape(ds, cp, cp.ncells > 0 ? std::min<int64_t>(cp.ncells, 2048) : 0);
}

// Workspaces of one class for every cluster that can be resident at once (max_clusters, fixed by
// the chosen launch shape): the forward-spectrum slots and, for the global-accumulator shapes, the
// S/G slots.  Called once at plan creation, so that no operation allocates.
ef_status alloc_workspaces(ef_plan_s *p, ClassPlan &cp)
{
    const int slots_c = std::max(1, cp.max_clusters);
    cudaError_t e = cudaMalloc(&cp.d_fh, (size_t)slots_c * ef::collide_fh_bytes(p->desc.prec, p->desc.d, cp.N));
    if (e != cudaSuccess) { cp.d_fh = nullptr; return cuda_fail(e, "spectrum workspace"); }
    cp.fh_slots = slots_c;
    if (!cp.sg_global) return EF_OK;
    const int N = cp.N, N1 = p->desc.d == 3 ? N : 1;
    const int64_t rows = (int64_t)cp.planes * N1;
    const int64_t slots = (int64_t)slots_c * cp.cluster;
    const size_t el = p->desc.prec == EF_PREC_F32 ? 4 : 8;
    e = cudaMalloc(&cp.d_sg, (size_t)slots * 2 * rows * N * el);
    if (e != cudaSuccess) { cp.d_sg = nullptr; return cuda_fail(e, "S/G workspace"); }
    cp.sg_slots = slots;
    return EF_OK;
}

// The launch of grid_clusters clusters fits the workspaces made at plan creation (always true,
// since the grid never exceeds max_clusters; checked so that a violation fails loudly).
ef_status check_workspaces(const ClassPlan &cp, int grid_clusters)
{
    if (grid_clusters > cp.fh_slots || (cp.sg_global && (int64_t)grid_clusters * cp.cluster > cp.sg_slots))
        return fail(EF_ERR_INVALID_ARG, "launch exceeds the plan's workspaces");
    return EF_OK;
}

void destroy_plan(ef_plan_s *p)
{
    if (!p) return;
    for (ClassPlan &cp : p->classes) {
        cudaFree(cp.d_mult);
        cudaFree(cp.d_ops_single);
        cudaFree(cp.d_modes);
        cudaFree(cp.d_ops_paired);
        cudaFree(cp.d_cell_off);
        cudaFree(cp.d_cell_id);
        cudaFree(cp.d_sg);
        cudaFree(cp.d_fh);
    }
    cudaFree(p->d_all_off);
    cudaFree(p->d_all_N);
    cudaFree(p->d_rk);
    cudaFree(p->d_status);
    cudaFree(p->d_counters);
    for (cudaStream_t st : p->cstreams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : p->cevents) cudaEventDestroy(ev);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    delete p;
}

ef_status fill_desc(const ef_plan_desc *in, Desc &ds)
{
    if (!in) return fail(EF_ERR_INVALID_ARG, "null plan description");
    ds.d = in->d;
    ds.N = in->N;
    ds.L = in->L;
    ds.kernel = in->kernel;
    ds.R = in->R;
    ds.prec = in->prec;
    if (ds.d != 2 && ds.d != 3) return fail(EF_ERR_INVALID_ARG, "d must be 2 or 3");
    if (!(ds.L > 0.0) || !std::isfinite(ds.L)) return fail(EF_ERR_INVALID_ARG, "L must be positive");
    if (ds.prec != EF_PREC_F32 && ds.prec != EF_PREC_F64) return fail(EF_ERR_INVALID_ARG, "bad precision");
    if (ds.kernel != EF_KERNEL_MAXWELL && ds.kernel != EF_KERNEL_HARD_SPHERE) return fail(EF_ERR_INVALID_ARG, "bad kernel");
    if (ds.d == 2 && ds.kernel != EF_KERNEL_MAXWELL) return fail(EF_ERR_UNSUPPORTED, "2D supports Maxwell molecules only");
    ds.T = ds.L;
    ds.Rtr = in->R_tr > 0 ? in->R_tr : 4.0 * ds.L / (3.0 * std::sqrt(2.0) + 1.0);
    ds.sigma = in->sigma_enabled < 0 ? 1 : (in->sigma_enabled ? 1 : 0);
    ds.J = in->J > 0 ? in->J : 6;
    if (ds.d == 2) {
        if (ds.R < 2 || ds.R % 2) return fail(EF_ERR_INVALID_ARG, "2D needs an even R >= 2");
        ds.nmu = ds.nphi = ds.nc = 0;
    } else {
        if (in->n_mu > 0 && in->n_phi > 0 && in->n_c > 0) {
            ds.nmu = in->n_mu;
            ds.nphi = in->n_phi;
            ds.nc = in->n_c;
        } else {
            switch (ds.R) {
            case 8: ds.nmu = 1; ds.nphi = 2; ds.nc = 2; break;
            case 16: ds.nmu = 1; ds.nphi = 4; ds.nc = 2; break;
            case 32: ds.nmu = 2; ds.nphi = 4; ds.nc = 2; break;
            case 64: ds.nmu = 2; ds.nphi = 4; ds.nc = 4; break;
            case 128: ds.nmu = 4; ds.nphi = 4; ds.nc = 4; break;
            default: return fail(EF_ERR_UNSUPPORTED, "no default angular quadrature for this R; set n_mu, n_phi, n_c");
            }
        }
        if (2 * ds.nmu * ds.nphi * ds.nc != ds.R) return fail(EF_ERR_INVALID_ARG, "R must equal 2 n_mu n_phi n_c");
    }
    return EF_OK;
}

ef_status check_N(const Desc &ds, int N)
{
    if (N < 8 || N % 2) return fail(EF_ERR_INVALID_ARG, "N must be even and >= 8");
    if (!size_built(ds.prec, ds.d, N)) return fail(EF_ERR_UNSUPPORTED, "N=" + std::to_string(N) + " is not a built size");
    return EF_OK;
}

ef_status check_device(const ef_plan_s *p)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(EF_ERR_INVALID_ARG, "the plan's device is not current");
    return EF_OK;
}

// Enqueue one step: every size class on its own internal stream (forked from and joined back
// to the caller's stream), each with a dynamic cell queue, so that clusters of one class fill
// the SMs another class leaves idle.  A single class launches directly on the caller's stream.
ef_status run(ef_plan_s *p, const void *F, void *Out, int64_t ncells, int mode, double dt, double *diag,
              cudaStream_t s)
{
    const Desc &ds = p->desc;
    // size classes run back to back on the caller's stream unless EF_CONCURRENT_CLASSES=1 forks
    // them onto their own streams (concurrent clusters of different sizes fragment the SMs'
    // shared memory, which measured slower)
    static const bool concurrent = [] {
        const char *v = std::getenv("EF_CONCURRENT_CLASSES");
        return v && v[0] == '1';
    }();
    const bool multi = concurrent && p->classes.size() > 1;
    cudaError_t e;
    if (multi) {
        e = cudaEventRecord(p->fork, s);
        if (e != cudaSuccess) return cuda_fail(e, "fork event");
    }
    for (size_t ci = 0; ci < p->classes.size(); ++ci) {
        ClassPlan &cp = p->classes[ci];
        const int64_t n = p->batched ? cp.ncells : ncells;
        if (n <= 0) continue;
        const int grid = (int)std::min<int64_t>(n, cp.max_clusters);
        ef_status st = check_workspaces(cp, grid);
        if (st != EF_OK) return st;
        cudaStream_t cs = s;
        if (multi) {
            cs = p->cstreams[ci];
            e = cudaStreamWaitEvent(cs, p->fork, 0);
            if (e != cudaSuccess) return cuda_fail(e, "fork wait");
            e = cudaMemsetAsync(p->d_counters + ci, 0, sizeof(unsigned long long), cs);
            if (e != cudaSuccess) return cuda_fail(e, "queue reset");
        }
        ef::CollideArgs a{};
        a.F = F;
        a.Q = Out;
        a.cell_off = cp.d_cell_off;
        a.cell_id = cp.d_cell_id;
        a.ncells = n;
        a.mult = cp.d_mult;
        a.ops = cp.d_ops;
        a.nops = cp.nops;
        a.cluster = cp.cluster;
        a.planes = cp.planes;
        a.sg_global = cp.sg_global;
        a.sg_ws = cp.d_sg;
        a.fh_ws = cp.d_fh;
        a.npc = ef::collide_npc_v(ds.d, cp.N, cp.cluster, cp.occ);
        a.out_mode = mode;
        a.dt = dt;
        a.h = 2.0 * ds.L / cp.N;
        a.diag = diag;
        a.status = p->d_status;
        a.counter = multi ? p->d_counters + ci : nullptr;
        a.prefetch = cp.prefetch;
        a.paired = cp.paired;
        e = launch_for(ds.prec, ds.d, cp.N, a, grid, cp.tpb, cp.smem, cp.occ, cs);
        if (e != cudaSuccess) return cuda_fail(e, "collide launch");
        if (multi) {
            e = cudaEventRecord(p->cevents[ci], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->cevents[ci], 0);
            if (e != cudaSuccess) return cuda_fail(e, "join");
        }
    }
    return EF_OK;
}

ef_status finish_plan(ef_plan_s *p)
{
    cudaError_t e = cudaMalloc((void **)&p->d_status, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    for (ClassPlan &cp : p->classes) {
        ef_status st = build_class(p->desc, cp);
        if (st != EF_OK) return st;
        st = alloc_workspaces(p, cp);
        if (st != EF_OK) return st;
    }
    if (p->classes.size() > 1) {
        e = cudaMalloc((void **)&p->d_counters, p->classes.size() * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "cell queues");
        e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "events");
        for (size_t i = 0; i < p->classes.size(); ++i) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (st) p->cstreams.push_back(st);
            if (ev) p->cevents.push_back(ev);
            if (e != cudaSuccess) return cuda_fail(e, "class streams");
        }
    }
    return EF_OK;
}

}  // namespace

extern "C" {

const char *ef_status_string(ef_status s)
{
    switch (s) {
    case EF_OK: return "EF_OK";
    case EF_ERR_INVALID_ARG: return "EF_ERR_INVALID_ARG";
    case EF_ERR_UNSUPPORTED: return "EF_ERR_UNSUPPORTED";
    case EF_ERR_CUDA: return "EF_ERR_CUDA";
    case EF_ERR_OOM: return "EF_ERR_OOM";
    case EF_ERR_TIMEOUT: return "EF_ERR_TIMEOUT";
    case EF_ERR_POSITIVITY: return "EF_ERR_POSITIVITY";
    case EF_ERR_NOT_FINITE: return "EF_ERR_NOT_FINITE";
    }
    return "EF_UNKNOWN_STATUS";
}

const char *ef_last_error(void) { return g_last_error.c_str(); }

ef_status ef_plan_create_ex(const ef_plan_desc *desc, ef_plan_t *out)
{
    if (!out) return fail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    Desc ds;
    ef_status st = fill_desc(desc, ds);
    if (st != EF_OK) return st;
    st = check_N(ds, desc->N);
    if (st != EF_OK) return st;
    ef_plan_s *p = new ef_plan_s();
    p->desc = ds;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    ClassPlan cp;
    cp.N = ds.N;
    p->classes.push_back(cp);
    st = finish_plan(p);
    if (st != EF_OK) { destroy_plan(p); return st; }
    *out = p;
    return EF_OK;
}

}  // extern "C"

namespace ef {

// A uniform plan on the grid of 2 N points per axis whose multiplier tables keep only the modes of
// the N grid's Galerkin set (used by ef_galerkin_*: products of band-limited factors do not wrap on
// the doubled grid).  desc describes the N-grid discretisation.
ef_status plan_create_padded(const ef_plan_desc *desc, ef_plan_t *out)
{
    if (!out) return fail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    Desc ds;
    ef_status st = fill_desc(desc, ds);
    if (st != EF_OK) return st;
    if (desc->N < 8 || desc->N % 2) return fail(EF_ERR_INVALID_ARG, "N must be even and >= 8");
    ds.gal_N = desc->N;
    ds.N = 2 * desc->N;
    st = check_N(ds, ds.N);
    if (st != EF_OK) return fail(EF_ERR_UNSUPPORTED, "the doubled grid 2N = " + std::to_string(ds.N) + " is not a built size");
    ef_plan_s *p = new ef_plan_s();
    p->desc = ds;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    ClassPlan cp;
    cp.N = ds.N;
    p->classes.push_back(cp);
    st = finish_plan(p);
    if (st != EF_OK) { destroy_plan(p); return st; }
    *out = p;
    return EF_OK;
}

}  // namespace ef

extern "C" {

ef_status ef_plan_create(int d, int N, double L, ef_kernel kernel, int R, ef_precision prec, ef_plan_t *out)
{
    ef_plan_desc desc;
    std::memset(&desc, 0, sizeof(desc));
    desc.d = d;
    desc.N = N;
    desc.L = L;
    desc.kernel = kernel;
    desc.R = R;
    desc.prec = prec;
    desc.sigma_enabled = -1;
    return ef_plan_create_ex(&desc, out);
}

ef_status ef_plan_create_batched(int d, int64_t ncells, const int *N_host, double L, ef_kernel kernel, int R,
                                 ef_precision prec, ef_plan_t *out)
{
    if (!out) return fail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (ncells <= 0 || !N_host) return fail(EF_ERR_INVALID_ARG, "batched plan needs ncells > 0 and N_host");
    ef_plan_desc desc;
    std::memset(&desc, 0, sizeof(desc));
    desc.d = d;
    desc.N = N_host[0];
    desc.L = L;
    desc.kernel = kernel;
    desc.R = R;
    desc.prec = prec;
    desc.sigma_enabled = -1;
    Desc ds;
    ef_status st = fill_desc(&desc, ds);
    if (st != EF_OK) return st;
    std::map<int, std::vector<int64_t>> byN;
    std::vector<int64_t> off(ncells), Ns(ncells);
    int64_t acc = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        st = check_N(ds, N_host[c]);
        if (st != EF_OK) return st;
        off[c] = acc;
        Ns[c] = N_host[c];
        acc += d == 3 ? (int64_t)N_host[c] * N_host[c] * N_host[c] : (int64_t)N_host[c] * N_host[c];
        byN[N_host[c]].push_back(c);
    }
    ef_plan_s *p = new ef_plan_s();
    p->desc = ds;
    p->batched = true;
    p->ncells = ncells;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    // largest cells first: their launches go first, smaller ones fill in behind
    for (auto it = byN.rbegin(); it != byN.rend(); ++it) {
        ClassPlan cp;
        cp.N = it->first;
        cp.ncells = (int64_t)it->second.size();
        std::vector<int64_t> co(cp.ncells), ci(cp.ncells);
        for (int64_t i = 0; i < cp.ncells; ++i) {
            ci[i] = it->second[i];
            co[i] = off[ci[i]];
        }
        e = cudaMalloc((void **)&cp.d_cell_off, cp.ncells * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&cp.d_cell_id, cp.ncells * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMemcpy(cp.d_cell_off, co.data(), cp.ncells * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(cp.d_cell_id, ci.data(), cp.ncells * sizeof(int64_t), cudaMemcpyHostToDevice);
        p->classes.push_back(cp);
        if (e != cudaSuccess) { destroy_plan(p); return cuda_fail(e, "cell tables"); }
    }
    e = cudaMalloc((void **)&p->d_all_off, ncells * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_all_N, ncells * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_all_off, off.data(), ncells * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_all_N, Ns.data(), ncells * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { destroy_plan(p); return cuda_fail(e, "cell tables"); }
    st = finish_plan(p);
    if (st != EF_OK) { destroy_plan(p); return st; }
    *out = p;
    return EF_OK;
}

ef_status ef_plan_destroy(ef_plan_t plan)
{
    if (!plan) return fail(EF_ERR_INVALID_ARG, "null plan");
    destroy_plan(plan);
    return EF_OK;
}

}  // extern "C"

namespace {

// One step (all size classes) either launched directly or through the plan's cached CUDA graph.
ef_status step(ef_plan_s *p, const void *F, void *Q, int64_t ncells, int mode, double dt, double *diag, cudaStream_t s)
{
    if (!(p->use_graph && s != nullptr)) return run(p, F, Q, ncells, mode, dt, diag, s);
    const bool hit = p->gexec && p->g_F == F && p->g_Q == Q && p->g_n == ncells && p->g_stream == s &&
                     p->g_mode == mode && p->g_dt == dt && p->g_diag == diag;
    if (!hit) {
        if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
        ef_status st;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        st = run(p, F, Q, ncells, mode, dt, diag, s);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (st != EF_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p->gexec = nullptr; return cuda_fail(e, "graph instantiate"); }
        p->g_F = F;
        p->g_Q = Q;
        p->g_n = ncells;
        p->g_stream = s;
        p->g_mode = mode;
        p->g_dt = dt;
        p->g_diag = diag;
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return EF_OK;
}

}  // namespace

namespace ef {

bool plan_view(const ef_plan_s *p, PlanView *out)
{
    if (!p || !out || p->batched || p->classes.size() != 1) return false;
    const ClassPlan &cp = p->classes[0];
    out->prec = p->desc.prec;
    out->d = p->desc.d;
    out->N = cp.N;
    out->cluster = cp.cluster;
    out->tpb = cp.tpb;
    out->planes = cp.planes;
    out->paired = cp.paired;
    out->nops = cp.nops;
    out->max_clusters = cp.max_clusters;
    out->sg_global = cp.sg_global;
    out->nfeat = cp.nfeat;
    out->occ = cp.occ;
    out->prefetch = cp.prefetch;
    out->ndir = cp.ndir;
    out->smem = cp.smem;
    out->modes = cp.d_modes;
    out->L = p->desc.L;
    out->mult = cp.d_mult;
    out->ops = cp.d_ops;
    out->status = p->d_status;
    out->device = p->device;
    return true;
}

bool features_fits(int prec, int d, int N, int nf)
{
    return prec == EF_PREC_F32 ? features_fits_f32(d, N, nf) : features_fits_f64(d, N, nf);
}

cudaError_t features_launch(int prec, int d, int N, const FeatArgs &a, cudaStream_t s)
{
    if (a.featL && !features_fits(prec, d, N, 2)) {
        // both fields do not fit in one CTA's shared memory: one launch per field
        FeatArgs a0 = a, a1 = a;
        a0.featL = nullptr;
        a1.featL = nullptr;
        a1.feat = a.featL;
        a1.log_input = 1;
        a1.mom = nullptr;
        cudaError_t e = features_launch(prec, d, N, a0, s);
        return e != cudaSuccess ? e : features_launch(prec, d, N, a1, s);
    }
    return prec == EF_PREC_F32 ? features_launch_f32(d, N, a, s) : features_launch_f64(d, N, a, s);
}

size_t collide_smem(int prec, int d, int N, int planes, int sg_global, int paired, int occ)
{
    return smem_for(prec, d, N, planes, sg_global, paired, occ);
}

cudaError_t collide_launch(int prec, int d, int N, const CollideArgs &a, int grid_clusters, int tpb, size_t smem,
                           int occ, cudaStream_t s)
{
    return launch_for(prec, d, N, a, grid_clusters, tpb, smem, occ, s);
}

void set_last_error(const char *msg) { g_last_error = msg; }

double jackson_filter(int N, int k, bool enabled) { return jackson(N, k, enabled); }

}  // namespace ef

extern "C" {

ef_status ef_collide(ef_plan_t p, const void *F, void *Q, int64_t ncells, ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (ncells < 0) return fail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (p->batched && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    if (ncells == 0) return EF_OK;
    if (!F || !Q) return fail(EF_ERR_INVALID_ARG, "null F or Q");
    if (F == Q) return fail(EF_ERR_INVALID_ARG, "F and Q must not overlap");
    if (((uintptr_t)F | (uintptr_t)Q) % 16) return fail(EF_ERR_INVALID_ARG, "F and Q must be 16-byte aligned");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    return step(p, F, Q, ncells, ef::OUT_COLLIDE, 0.0, nullptr, (cudaStream_t)stream);
}

ef_status ef_euler_step(ef_plan_t p, void *F, double dt, int nsteps, double *diag, int64_t ncells, ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (nsteps < 0 || ncells < 0) return fail(EF_ERR_INVALID_ARG, "negative nsteps or ncells");
    if (!std::isfinite(dt)) return fail(EF_ERR_INVALID_ARG, "dt must be finite");
    if (p->batched && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    if (nsteps == 0 || ncells == 0) return EF_OK;
    if (!F) return fail(EF_ERR_INVALID_ARG, "null F");
    if ((uintptr_t)F % 16) return fail(EF_ERR_INVALID_ARG, "F must be 16-byte aligned");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    for (int k = 0; k < nsteps; ++k) {
        st = step(p, F, F, ncells, ef::OUT_EULER, dt, diag ? diag + (int64_t)k * ncells * ef::kDiag : nullptr,
                  (cudaStream_t)stream);
        if (st != EF_OK) return st;
    }
    return EF_OK;
}

}  // extern "C"

namespace {

// values (grid points) in a batch of ncells cells of the plan (the whole batch for a batched plan)
int64_t batch_values(const ef_plan_s *p, int64_t ncells)
{
    const Desc &ds = p->desc;
    int64_t total = 0;
    if (p->batched) {
        for (const ClassPlan &cp : p->classes) total += cp.ncells * (int64_t)cp.N * cp.N * (ds.d == 3 ? cp.N : 1);
    } else {
        total = ncells * (int64_t)ds.N * ds.N * (ds.d == 3 ? ds.N : 1);
    }
    return total;
}

}  // namespace

extern "C" {

ef_status ef_plan_reserve(ef_plan_t p, int64_t ncells)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (ncells < 0) return fail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (p->batched && ncells != 0 && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    const size_t el = p->desc.prec == EF_PREC_F32 ? 4 : 8;
    const int64_t total = batch_values(p, p->batched ? p->ncells : ncells);
    const size_t half = ((size_t)total * el + 255) / 256 * 256;
    if (2 * half <= p->rk_bytes) return EF_OK;
    cudaError_t e = cudaDeviceSynchronize();             // the old buffers may still be in use
    if (e == cudaSuccess && p->d_rk) e = cudaFree(p->d_rk);
    p->d_rk = nullptr;
    p->rk_bytes = 0;
    if (e == cudaSuccess) e = cudaMalloc(&p->d_rk, 2 * half);
    if (e != cudaSuccess) { p->d_rk = nullptr; return cuda_fail(e, "SSP-RK3 stage buffers"); }
    p->rk_bytes = 2 * half;
    return EF_OK;
}

ef_status ef_rk3_step(ef_plan_t p, void *F, double dt, int nsteps, double *diag, int64_t ncells, ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (nsteps < 0 || ncells < 0) return fail(EF_ERR_INVALID_ARG, "negative nsteps or ncells");
    if (!std::isfinite(dt)) return fail(EF_ERR_INVALID_ARG, "dt must be finite");
    if (p->batched && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    if (nsteps == 0 || ncells == 0) return EF_OK;
    if (!F) return fail(EF_ERR_INVALID_ARG, "null F");
    if ((uintptr_t)F % 16) return fail(EF_ERR_INVALID_ARG, "F must be 16-byte aligned");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    const Desc &ds = p->desc;
    const int64_t total = batch_values(p, ncells);
    const size_t el = ds.prec == EF_PREC_F32 ? 4 : 8;
    const size_t half = ((size_t)total * el + 255) / 256 * 256;
    if (2 * half > p->rk_bytes)
        return fail(EF_ERR_INVALID_ARG, "SSP-RK3 stage buffers too small for " + std::to_string(ncells) +
                                            " cells: call ef_plan_reserve(plan, ncells) first");
    void *A = p->d_rk, *B = static_cast<unsigned char *>(p->d_rk) + half;
    cudaStream_t s = (cudaStream_t)stream;
    const int prec = ds.prec == EF_PREC_F32 ? 0 : 1;
    for (int k = 0; k < nsteps; ++k) {
        double *dk = diag ? diag + (int64_t)k * ncells * ef::kDiag : nullptr;
        // F1 = F + dt Q[F]
        st = run(p, F, A, ncells, ef::OUT_EULER, dt, dk, s);
        if (st != EF_OK) return st;
        // F2 = 3/4 F + 1/4 (F1 + dt Q[F1])
        st = run(p, A, B, ncells, ef::OUT_EULER, dt, nullptr, s);
        if (st != EF_OK) return st;
        cudaError_t e = ef::axpby_launch(prec, B, F, B, 0.75, 0.25, total, s);
        if (e != cudaSuccess) return cuda_fail(e, "RK3 combine");
        // F <- 1/3 F + 2/3 (F2 + dt Q[F2])
        st = run(p, B, A, ncells, ef::OUT_EULER, dt, nullptr, s);
        if (st != EF_OK) return st;
        e = ef::axpby_launch(prec, F, F, A, 1.0 / 3.0, 2.0 / 3.0, total, s);
        if (e != cudaSuccess) return cuda_fail(e, "RK3 combine");
    }
    return EF_OK;
}

ef_status ef_moments_entropy(ef_plan_t p, const void *F, const void *Q, double *out, int64_t ncells, ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (ncells < 0) return fail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (p->batched && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    if (ncells == 0) return EF_OK;
    if (!F || !out) return fail(EF_ERR_INVALID_ARG, "null F or out");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    cudaError_t e = ef::moments_launch(p->desc.prec == EF_PREC_F32 ? 0 : 1, p->desc.d, F, Q, p->d_all_off, p->d_all_N,
                                       ncells, p->desc.N, 2.0 * p->desc.L, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
    return EF_OK;
}

ef_status ef_transport_step(ef_plan_t p, const void *F_in, void *F_out, int64_t ncells, double dx, double dt,
                            ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (p->batched) return fail(EF_ERR_INVALID_ARG, "transport needs a uniform plan (one N for every spatial cell)");
    if (ncells < 0) return fail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (!(dx > 0.0) || !std::isfinite(dx) || !std::isfinite(dt)) return fail(EF_ERR_INVALID_ARG, "dx must be > 0, dt finite");
    if (ncells == 0) return EF_OK;
    if (!F_in || !F_out) return fail(EF_ERR_INVALID_ARG, "null F_in or F_out");
    if (((uintptr_t)F_in | (uintptr_t)F_out) % 16) return fail(EF_ERR_INVALID_ARG, "F_in and F_out must be 16-byte aligned");
    const Desc &ds = p->desc;
    const int64_t cell = ds.d == 3 ? (int64_t)ds.N * ds.N * ds.N : (int64_t)ds.N * ds.N;
    const uintptr_t bytes = (uintptr_t)(ncells * cell * (ds.prec == EF_PREC_F32 ? 4 : 8));
    const uintptr_t a = (uintptr_t)F_in, b = (uintptr_t)F_out;
    if (a < b + bytes && b < a + bytes) return fail(EF_ERR_INVALID_ARG, "F_out must not overlap F_in");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    const double h = 2.0 * ds.L / ds.N;
    cudaError_t e = ef::transport_launch(ds.prec == EF_PREC_F32 ? 0 : 1, ds.d, ds.N, F_in, F_out, ncells, dt * h / dx,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "transport launch");
    return EF_OK;
}

ef_status ef_features(ef_plan_t p, const void *F, float *feat, int64_t ncells, int log_input, ef_stream_t stream)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (ncells < 0) return fail(EF_ERR_INVALID_ARG, "ncells < 0");
    if (p->batched && ncells != p->ncells) return fail(EF_ERR_INVALID_ARG, "ncells differs from the batched plan");
    if (ncells == 0) return EF_OK;
    if (!F || !feat) return fail(EF_ERR_INVALID_ARG, "null F or feat");
    if ((uintptr_t)F % 16) return fail(EF_ERR_INVALID_ARG, "F must be 16-byte aligned");
    for (const ClassPlan &cp : p->classes)
        if (cp.nfeat == 0) return fail(EF_ERR_UNSUPPORTED, "N too small for the feature band");
    ef_status st = check_device(p);
    if (st != EF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const Desc &ds = p->desc;
    for (ClassPlan &cp : p->classes) {
        const int64_t n = p->batched ? cp.ncells : ncells;
        if (n <= 0) continue;
        ef::FeatArgs a{};
        a.F = F;
        a.cell_off = cp.d_cell_off;
        a.cell_id = cp.d_cell_id;
        a.ncells = n;
        a.log_input = log_input ? 1 : 0;
        a.feat = feat;
        a.fstride = EF_FEATURE_STRIDE;
        a.h = 2.0 * ds.L / cp.N;
        a.modes = cp.d_modes;
        a.nmodes = cp.nfeat;
        cudaError_t e = ef::features_launch(ds.prec, ds.d, cp.N, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "features launch");
    }
    return EF_OK;
}

ef_status ef_plan_status(ef_plan_t p, int sync, int reset)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    if (sync) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
        e = cudaMemcpy(&p->h_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "status read");
        if (reset) {
            e = cudaMemset(p->d_status, 0, sizeof(int));
            if (e != cudaSuccess) return cuda_fail(e, "status reset");
        }
    }
    const int s = p->h_status;
    if (reset) p->h_status = 0;
    return (ef_status)s;
}

ef_status ef_plan_set_graph(ef_plan_t p, int enable)
{
    if (!p) return fail(EF_ERR_INVALID_ARG, "null plan");
    p->use_graph = enable != 0;
    if (!p->use_graph && p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return EF_OK;
}

ef_status ef_plan_class_info(ef_plan_t p, int i, int64_t out[8])
{
    if (!p || !out) return fail(EF_ERR_INVALID_ARG, "null plan or output");
    if (i < 0 || i >= (int)p->classes.size()) return fail(EF_ERR_INVALID_ARG, "class index out of range");
    const ClassPlan &cp = p->classes[i];
    out[0] = cp.N;
    out[1] = cp.ncells;
    out[2] = cp.cluster;
    out[3] = cp.tpb;
    out[4] = cp.planes;
    out[5] = cp.sg_global;
    out[6] = cp.prefetch;
    out[7] = (int64_t)(cp.tuned_ms * 1000.0);
    return EF_OK;
}

ef_status ef_plan_info(ef_plan_t p, int64_t info[8])
{
    if (!p || !info) return fail(EF_ERR_INVALID_ARG, "null plan or info");
    info[0] = p->desc.d;
    info[1] = (int64_t)p->classes.size();
    info[2] = p->classes.empty() ? 0 : p->classes[0].ndir;
    info[3] = p->classes.empty() ? 0 : p->classes[0].cluster;
    info[4] = p->classes.empty() ? 0 : p->classes[0].tpb;
    info[5] = p->batched ? p->ncells : 0;
    info[6] = p->desc.prec;
    info[7] = (int64_t)p->classes.size();
    return EF_OK;
}

}  // extern "C"
