/*
 * ef_oracle.c -- plain, slow, FP64 CPU oracle for the entropic Fourier method (EFM)
 * collision operator of Cai, Fan & Ying, "An entropic Fourier method for the Boltzmann
 * equation" (arXiv:1704.07369).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may include, link or call
 * this file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg use
 * it.  It shares no source, header, table or constant generator with the CUDA library.
 *
 * What it computes (all in double precision, with no FFT):
 *   - the modified Jackson filter sigma_N (Sec. 3.2.2, eq. JacksonFilter2), with the even-N rule
 *     of Sec. 4.1 (modes with any component -N/2 carry no kernel weight);
 *   - the low-rank kernel modes B_fast(l,m) = sum_t w_t beta_t(l) gamma_t(m) (Sec. 4.1,
 *     eq. fastAlg) for three collision kernels:
 *       * 2D Maxwell molecules, B = 1/(2 pi): the polar decomposition of eqs. spherical_hatB /
 *         fast_hatB with the rectangle rule of eq. discrete_hatB over [0, pi);
 *       * 3D hard spheres, B = |g|/(4 pi): Carleman form (Sec. 1, eq. Carleman) in polar
 *         coordinates, Gauss-Legendre in cos(polar) x uniform azimuth on the half sphere, uniform
 *         angles on the half great circle orthogonal to each direction, swap-symmetrised;
 *       * 3D Maxwell molecules, B = 1/(4 pi): as hard spheres, with 1/|y+z| expanded in J
 *         positive Gaussian terms so each radial factor stays separable and non-negative;
 *   - the discrete Fourier transform of eq. DFT by its direct definition;
 *   - Q^sigma by the plain double sum of eq. Qsk over (l, m) (aliased indicator 1_N), followed
 *     by the direct inverse DFT (oracle_collide), O(R N^{2d});
 *   - the same operator at selected grid points in the rank-separated form of eq. fastFGM
 *     (sum over t outside), for sampled checks at large N (oracle_collide_points);
 *   - the DVM form eq. Qsr with A^sigma from eq. A_simplified / tildetildeA, by brute force over
 *     (p, q, s), O(N^{3d}), for tiny grids (oracle_dvm);
 *   - G(y, z) of eq. G / tildeG on the grid (oracle_G), for the positivity checks of Sec. 3.2;
 *   - the Fourier Galerkin method's unaliased sum (oracle_collide_galerkin, eq. FGM_Q), the
 *     comparison method of Fig. 2;
 *   - the entropic Fourier method on the classical form of the collision operator (remark after
 *     eq. EFMk) for 3D Maxwell molecules, B_hat from eq. classical_hatB with its angular and
 *     radial integrals done in closed form, by the plain double sum (oracle_collide_classical).
 *
 * Grid and mode conventions: velocity index j in {-N/2, ..., N/2-1} per axis (array index
 * i = j + N/2, C order, axis 0 slowest), v = h j with h = 2T/N.  Modes are stored in FFT order:
 * index i in [0, N) stands for k = i (i < ceil(N/2)) or k = i - N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

enum { OR_K_MAXWELL_2D = 0, OR_K_HARD_SPHERE_3D = 1, OR_K_MAXWELL_3D = 2 };

typedef struct {
    int d;        /* dimension, 2 or 3 */
    int N;        /* points per axis */
    int kernel;   /* OR_K_* */
    int R;        /* angular rank: number of (symmetrised) angular terms */
    int nmu;      /* 3D: Gauss-Legendre nodes in cos(polar) on [0,1] */
    int nphi;     /* 3D: azimuth samples on [0, 2 pi) */
    int nc;       /* 3D: samples on the half circle orthogonal to e */
    int J;        /* 3D Maxwell: Gaussian terms for 1/|y+z| */
    int filter;   /* 1: modified Jackson filter (EFM); 0: none (collocation method) */
    int pad;
    double T;     /* half width of the periodic box [-T, T]^d */
    double Rtr;   /* truncation radius R of eq. approximated_collision */
} oracle_params;

/* ---------------------------------------------------------------- small helpers ---------- */

static int64_t ipow(int b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

/* mode number of FFT-order index i */
static int mode_of(int N, int i) { return (i < (N + 1) / 2) ? i : i - N; }

/* modified Jackson filter, eq. JacksonFilter2.  For odd N = 2n+1 the paper's n; for even N the
 * reading n = N/2, which gives sigma(+-N/2) = 0, i.e. the even-N rule of Sec. 4.1. */
double oracle_sigma1(int N, int k)
{
    int n = (N % 2) ? (N - 1) / 2 : N / 2;
    int b = k < 0 ? -k : k;
    if (N % 2 == 0 && k == -N / 2) return 0.0;
    if (b > n) return 0.0;
    double np1 = (double)(n + 1);
    double a = ORACLE_PI * (double)b / np1;
    double c = ORACLE_PI / np1;
    return ((np1 - (double)b) * cos(a) + sin(a) * cos(c) / sin(c)) / np1;
}

static double sinc(double y) { return (fabs(y) < 1e-8) ? 1.0 - y * y / 6.0 : sin(y) / y; }

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------- kernel decompositions ---------- */

/* 2D: psi_R(l, e) = int_{-R}^{R} E_l(rho e) d rho = 2 R sinc(pi R (l.e) / T)  (Sec. 4.1). */
static double psi2d(double x, double T, double Rtr) { return 2.0 * Rtr * sinc(ORACLE_PI * Rtr * x / T); }

/* 3D hard spheres: phi(x) = int_{-R}^{R} |rho| E(rho x) d rho = 2 int_0^R rho cos(pi rho x/T) d rho
 *                = R^2 [2 sinc(a R) - sinc(a R / 2)^2],  a = pi x / T. */
static double phi3d(double x, double T, double Rtr)
{
    double a = ORACLE_PI * x / T;
    double s1 = sinc(a * Rtr), s2 = sinc(0.5 * a * Rtr);
    return Rtr * Rtr * (2.0 * s1 - s2 * s2);
}

/* 3D Maxwell: 1/sqrt(s) = (2/sqrt(pi)) int_0^inf exp(-u^2 s) du.  With u = exp(tau) the
 * integral over tau in [tau_a, tau_b], tau_a = ln(0.4/R), tau_b = ln(35/R), is taken by
 * Gauss-Legendre with J-1 nodes, and the piece u in [0, exp(tau_a)] by the single term u = 0
 * (exp(-u^2 s) ~ 1 there).  So 1/sqrt(s) ~ sum_{j<J} c_j exp(-u_j^2 s) with every c_j > 0. */
static void maxwell3d_terms(int J, double Rtr, double *u, double *c)
{
    int n = J - 1;
    double *x = malloc(sizeof(double) * (n > 0 ? n : 1)), *w = malloc(sizeof(double) * (n > 0 ? n : 1));
    if (n > 0) gauss_legendre(n, x, w);
    double ta = log(0.4 / Rtr), tb = log(35.0 / Rtr);
    u[0] = 0.0;
    c[0] = 2.0 / sqrt(ORACLE_PI) * exp(ta);
    for (int j = 0; j < n; ++j) {
        double tau = ta + 0.5 * (x[j] + 1.0) * (tb - ta);
        u[j + 1] = exp(tau);
        c[j + 1] = 2.0 / sqrt(ORACLE_PI) * 0.5 * (tb - ta) * w[j] * exp(tau);
    }
    free(x); free(w);
}

/* radial factor of the Maxwell 3D term j: 2 int_0^R rho exp(-u^2 rho^2) cos(pi rho x / T) d rho,
 * composite Gauss-Legendre, 16 panels x 8 nodes. */
static double phi3d_gauss(double x, double u, double T, double Rtr)
{
    static const int P = 16, n = 8;
    double gx[8], gw[8];
    gauss_legendre(n, gx, gw);
    double a = ORACLE_PI * x / T, hpan = Rtr / P, acc = 0.0;
    for (int p = 0; p < P; ++p)
        for (int i = 0; i < n; ++i) {
            double rho = hpan * (p + 0.5 * (gx[i] + 1.0));
            acc += 0.5 * hpan * gw[i] * rho * exp(-u * u * rho * rho) * cos(a * rho);
        }
    return 2.0 * acc;
}

/* Number of (l, m) product terms t in B_fast(l, m) = sum_t w_t beta_t(l) gamma_t(m). */
int oracle_nterms(const oracle_params *p)
{
    if (p->kernel == OR_K_MAXWELL_2D) return p->R;
    int base = 2 * p->nmu * p->nphi * p->nc;
    return p->kernel == OR_K_MAXWELL_3D ? base * p->J : base;
}

/* 3D angular quadrature: e_ab on the half sphere (mu_a = cos polar in (0,1), azimuth alpha_b),
 * e*_abc = cos(c pi/nc) u_ab + sin(c pi/nc) v_ab on the half circle orthogonal to e_ab,
 * with u = d e / d polar, v = d e / d alpha normalised.  Weight of (a,b,c):
 *   (1/pi) * wmu_a * (2 pi / nphi) * (pi / nc). */
static void angular3d(const oracle_params *p, double *e, double *es, double *wt)
{
    double *x = malloc(sizeof(double) * p->nmu), *w = malloc(sizeof(double) * p->nmu);
    gauss_legendre(p->nmu, x, w);
    int t = 0;
    for (int a = 0; a < p->nmu; ++a) {
        double mu = 0.5 * (x[a] + 1.0), wmu = 0.5 * w[a];
        double st = sqrt(1.0 - mu * mu);
        for (int b = 0; b < p->nphi; ++b) {
            double al = 2.0 * ORACLE_PI * b / p->nphi;
            double ev[3] = { st * cos(al), st * sin(al), mu };
            double uv[3] = { mu * cos(al), mu * sin(al), -st };
            double vv[3] = { -sin(al), cos(al), 0.0 };
            for (int c = 0; c < p->nc; ++c) {
                double ph = ORACLE_PI * c / p->nc;
                for (int q = 0; q < 3; ++q) {
                    e[3 * t + q] = ev[q];
                    es[3 * t + q] = cos(ph) * uv[q] + sin(ph) * vv[q];
                }
                wt[t] = (1.0 / ORACLE_PI) * wmu * (2.0 * ORACLE_PI / p->nphi) * (ORACLE_PI / p->nc);
                ++t;
            }
        }
    }
    free(x); free(w);
}

/* Fill w[t], beta[t*M + l], gamma[t*M + l] (M = N^d modes, FFT order), unfiltered. */
int oracle_factors(const oracle_params *p, double *w, double *beta, double *gamma)
{
    const int N = p->N, d = p->d;
    const int64_t M = ipow(N, d);
    if (p->kernel == OR_K_MAXWELL_2D) {
        if (d != 2 || p->R < 2 || p->R % 2) return -1;
        for (int t = 0; t < p->R; ++t) {
            double th = ORACLE_PI * t / p->R;
            double e0 = cos(th), e1 = sin(th);          /* e_theta */
            double f0 = -sin(th), f1 = cos(th);         /* e_{theta + pi/2} */
            w[t] = (1.0 / ORACLE_PI) * (ORACLE_PI / p->R);
            for (int64_t l = 0; l < M; ++l) {
                double k0 = mode_of(N, (int)(l / N)), k1 = mode_of(N, (int)(l % N));
                beta[t * M + l] = psi2d(k0 * e0 + k1 * e1, p->T, p->Rtr);
                gamma[t * M + l] = psi2d(k0 * f0 + k1 * f1, p->T, p->Rtr);
            }
        }
        return 0;
    }
    if (d != 3) return -1;
    int na = p->nmu * p->nphi * p->nc;
    double *e = malloc(sizeof(double) * 3 * na), *es = malloc(sizeof(double) * 3 * na);
    double *wa = malloc(sizeof(double) * na);
    angular3d(p, e, es, wa);
    int J = p->kernel == OR_K_MAXWELL_3D ? p->J : 1;
    double *u = malloc(sizeof(double) * J), *c = malloc(sizeof(double) * J);
    if (p->kernel == OR_K_MAXWELL_3D) maxwell3d_terms(J, p->Rtr, u, c);
    else { u[0] = 0.0; c[0] = 1.0; }
    int t = 0;
    for (int j = 0; j < J; ++j)
        for (int a = 0; a < na; ++a)
            for (int sw = 0; sw < 2; ++sw) {     /* swap symmetrisation */
                const double *eb = sw ? es + 3 * a : e + 3 * a;
                const double *eg = sw ? e + 3 * a : es + 3 * a;
                w[t] = 0.5 * wa[a] * c[j];
                for (int64_t l = 0; l < M; ++l) {
                    double k0 = mode_of(N, (int)(l / (N * N)));
                    double k1 = mode_of(N, (int)((l / N) % N));
                    double k2 = mode_of(N, (int)(l % N));
                    double xb = k0 * eb[0] + k1 * eb[1] + k2 * eb[2];
                    double xg = k0 * eg[0] + k1 * eg[1] + k2 * eg[2];
                    if (p->kernel == OR_K_MAXWELL_3D) {
                        beta[t * M + l] = phi3d_gauss(xb, u[j], p->T, p->Rtr);
                        gamma[t * M + l] = phi3d_gauss(xg, u[j], p->T, p->Rtr);
                    } else {
                        beta[t * M + l] = phi3d(xb, p->T, p->Rtr);
                        gamma[t * M + l] = phi3d(xg, p->T, p->Rtr);
                    }
                }
                ++t;
            }
    free(e); free(es); free(wa); free(u); free(c);
    return 0;
}

/* sigma_N(l) for every mode l (tensor product), or 1 when the filter is off; modes with any
 * component -N/2 (even N) are zero either way (Sec. 4.1). */
static void filter_table(const oracle_params *p, double *sig)
{
    const int N = p->N, d = p->d;
    const int64_t M = ipow(N, d);
    for (int64_t l = 0; l < M; ++l) {
        int64_t r = l;
        double s = 1.0;
        for (int a = d - 1; a >= 0; --a) {
            int k = mode_of(N, (int)(r % N));
            r /= N;
            if (N % 2 == 0 && k == -N / 2) s = 0.0;
            else if (p->filter) s *= oracle_sigma1(N, k);
        }
        sig[l] = s;
    }
}

/* ------------------------------------------------------------- direct DFT ---------------- */

/* Fh_k = N^{-d} sum_p F_p E_{-k}(p), E_k(v) = exp(i pi k.v / T), v = h j (eq. DFT). */
void oracle_dft(int d, int N, const double *F, double *Fre, double *Fim)
{
    const int64_t M = ipow(N, d);
    double *ct = malloc(sizeof(double) * N * N), *st = malloc(sizeof(double) * N * N);
    for (int i = 0; i < N; ++i)          /* mode index */
        for (int q = 0; q < N; ++q) {    /* grid index, j = q - N/2 */
            double ang = 2.0 * ORACLE_PI * (double)mode_of(N, i) * (double)(q - N / 2) / N;
            ct[i * N + q] = cos(ang); st[i * N + q] = sin(ang);
        }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < M; ++k) {
        int ki[3] = { 0, 0, 0 };
        int64_t r = k;
        for (int a = d - 1; a >= 0; --a) { ki[a] = (int)(r % N); r /= N; }
        double re = 0.0, im = 0.0;
        for (int64_t pidx = 0; pidx < M; ++pidx) {
            int pi_[3] = { 0, 0, 0 };
            int64_t s = pidx;
            for (int a = d - 1; a >= 0; --a) { pi_[a] = (int)(s % N); s /= N; }
            /* E_{-k}(p) = prod_a exp(-i 2 pi k_a j_a / N) */
            double cr = 1.0, ci = 0.0;
            for (int a = 0; a < d; ++a) {
                double c = ct[ki[a] * N + pi_[a]], sn = -st[ki[a] * N + pi_[a]];
                double nr = cr * c - ci * sn, ni = cr * sn + ci * c;
                cr = nr; ci = ni;
            }
            re += F[pidx] * cr; im += F[pidx] * ci;
        }
        double sc = 1.0 / (double)M;
        Fre[k] = re * sc; Fim[k] = im * sc;
    }
    free(ct); free(st);
}

/* F_p = sum_k Fh_k E_k(p), real part (the result is real for Hermitian input). */
void oracle_idft_real(int d, int N, const double *Fre, const double *Fim, double *F)
{
    const int64_t M = ipow(N, d);
    double *ct = malloc(sizeof(double) * N * N), *st = malloc(sizeof(double) * N * N);
    for (int i = 0; i < N; ++i)
        for (int q = 0; q < N; ++q) {
            double ang = 2.0 * ORACLE_PI * (double)mode_of(N, i) * (double)(q - N / 2) / N;
            ct[i * N + q] = cos(ang); st[i * N + q] = sin(ang);
        }
#pragma omp parallel for schedule(static)
    for (int64_t pidx = 0; pidx < M; ++pidx) {
        int pi_[3] = { 0, 0, 0 };
        int64_t s = pidx;
        for (int a = d - 1; a >= 0; --a) { pi_[a] = (int)(s % N); s /= N; }
        double re = 0.0;
        for (int64_t k = 0; k < M; ++k) {
            int ki[3] = { 0, 0, 0 };
            int64_t r = k;
            for (int a = d - 1; a >= 0; --a) { ki[a] = (int)(r % N); r /= N; }
            double cr = 1.0, ci = 0.0;
            for (int a = 0; a < d; ++a) {
                double c = ct[ki[a] * N + pi_[a]], sn = st[ki[a] * N + pi_[a]];
                double nr = cr * c - ci * sn, ni = cr * sn + ci * c;
                cr = nr; ci = ni;
            }
            re += Fre[k] * cr - Fim[k] * ci;
        }
        F[pidx] = re;
    }
    free(ct); free(st);
}

/* ------------------------------------------------------------ the operator ---------------- */

typedef struct {
    int64_t M;
    int T;
    double *w, *beta, *gamma, *sig;
} kern_tables;

static int make_tables(const oracle_params *p, kern_tables *kt)
{
    kt->M = ipow(p->N, p->d);
    kt->T = oracle_nterms(p);
    kt->w = malloc(sizeof(double) * kt->T);
    kt->beta = malloc(sizeof(double) * kt->T * kt->M);
    kt->gamma = malloc(sizeof(double) * kt->T * kt->M);
    kt->sig = malloc(sizeof(double) * kt->M);
    if (!kt->w || !kt->beta || !kt->gamma || !kt->sig) return -1;
    if (oracle_factors(p, kt->w, kt->beta, kt->gamma)) return -1;
    filter_table(p, kt->sig);
    return 0;
}

static void free_tables(kern_tables *kt) { free(kt->w); free(kt->beta); free(kt->gamma); free(kt->sig); }

/* filtered fast kernel B^sigma_fast(l, m) = sigma(l) sigma(m) sum_t w_t beta_t(l) gamma_t(m) */
static double bsig(const kern_tables *kt, int64_t l, int64_t m)
{
    double acc = 0.0;
    for (int t = 0; t < kt->T; ++t) acc += kt->w[t] * kt->beta[t * kt->M + l] * kt->gamma[t * kt->M + m];
    return kt->sig[l] * kt->sig[m] * acc;
}

/* flat FFT-order index of (k - l) mod N, componentwise */
static int64_t diff_mod(int d, int N, int64_t k, int64_t l)
{
    int64_t out = 0, mul = 1;
    for (int a = 0; a < d; ++a) {
        int ka = (int)(k % N), la = (int)(l % N);
        k /= N; l /= N;
        int m = ((ka - la) % N + N) % N;
        out += m * mul; mul *= N;
    }
    return out;
}

/* Q^sigma on the grid: Qh_k = sum_{l,m} 1_N(l+m-k) (B(l,m) - B(m,m)) Fh_l Fh_m (eq. Qsk), then
 * Q_r = sum_k Qh_k E_k(r).  F and Q are real arrays of N^d points. Returns 0 on success. */
int oracle_collide(const oracle_params *p, const double *F, double *Q)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    double *Fr = malloc(sizeof(double) * M), *Fi = malloc(sizeof(double) * M);
    double *Qr = malloc(sizeof(double) * M), *Qi = malloc(sizeof(double) * M);
    double *bmm = malloc(sizeof(double) * M);
    oracle_dft(p->d, p->N, F, Fr, Fi);
    for (int64_t m = 0; m < M; ++m) bmm[m] = bsig(&kt, m, m);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < M; ++k) {
        double re = 0.0, im = 0.0;
        for (int64_t l = 0; l < M; ++l) {
            int64_t m = diff_mod(p->d, p->N, k, l);      /* the unique m with 1_N(l+m-k) = 1 */
            double b = bsig(&kt, l, m) - bmm[m];
            double pr = Fr[l] * Fr[m] - Fi[l] * Fi[m];
            double pim = Fr[l] * Fi[m] + Fi[l] * Fr[m];
            re += b * pr; im += b * pim;
        }
        Qr[k] = re; Qi[k] = im;
    }
    oracle_idft_real(p->d, p->N, Qr, Qi, Q);
    free(Fr); free(Fi); free(Qr); free(Qi); free(bmm); free_tables(&kt);
    return 0;
}

/* ------------------------------------------ Fourier Galerkin method (Sec. 1.2) ------------ */

/* The Fourier Galerkin method (FGM, eq. FGM_Q / eq. FG): the unaliased sum
 *   Qh^G_k = sum_{l, m in K, l + m = k} (B(l,m) - B(m,m)) Fh_l Fh_m,   k in K,
 * with K = {-n, ..., n}^d, n = (N-1)/2 (odd N) or N/2 - 1 (even N: the modes with a component
 * -N/2 are dropped, Sec. 4.1), B the plan's low-rank kernel (eq. fastFGM) with the filter if
 * p->filter is set (the FGM of the literature has none), and Fh the DFT of the grid values (the
 * interpolation initial data of Fig. 2).  Q = the grid values of sum_k Qh^G_k E_k.  Unlike the
 * collocation sum (oracle_collide) the index l + m is not reduced mod N: modes that leave K are
 * discarded.  O(R N^{2d}). */
int oracle_collide_galerkin(const oracle_params *p, const double *F, double *Q)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    const int N = p->N, d = p->d;
    const int n = (N % 2) ? (N - 1) / 2 : N / 2 - 1;
    double *Fr = malloc(sizeof(double) * M), *Fi = malloc(sizeof(double) * M);
    double *Qr = malloc(sizeof(double) * M), *Qi = malloc(sizeof(double) * M);
    double *bmm = malloc(sizeof(double) * M);
    int *in = malloc(sizeof(int) * M);
    oracle_dft(d, N, F, Fr, Fi);
    for (int64_t l = 0; l < M; ++l) {
        int64_t r = l;
        int ok = 1;
        for (int a = 0; a < d; ++a) { int k = mode_of(N, (int)(r % N)); r /= N; if (k < -n || k > n) ok = 0; }
        in[l] = ok;
        if (!ok) { Fr[l] = 0.0; Fi[l] = 0.0; }
        bmm[l] = bsig(&kt, l, l);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < M; ++k) {
        double re = 0.0, im = 0.0;
        if (in[k]) {
            for (int64_t l = 0; l < M; ++l) {
                if (!in[l]) continue;
                /* m = k - l componentwise, without reduction; skip if it leaves K */
                int64_t kk = k, ll = l, m = 0, mul = 1;
                int ok = 1;
                for (int a = 0; a < d; ++a) {
                    const int ka = mode_of(N, (int)(kk % N)), la = mode_of(N, (int)(ll % N));
                    kk /= N; ll /= N;
                    const int ma = ka - la;
                    if (ma < -n || ma > n) { ok = 0; break; }
                    m += (int64_t)((ma + N) % N) * mul;
                    mul *= N;
                }
                if (!ok) continue;
                const double b = bsig(&kt, l, m) - bmm[m];
                re += b * (Fr[l] * Fr[m] - Fi[l] * Fi[m]);
                im += b * (Fr[l] * Fi[m] + Fi[l] * Fr[m]);
            }
        }
        Qr[k] = re; Qi[k] = im;
    }
    oracle_idft_real(d, N, Qr, Qi, Q);
    free(Fr); free(Fi); free(Qr); free(Qi); free(bmm); free(in); free_tables(&kt);
    return 0;
}

/* ------------------------------------------ classical form, 3D Maxwell molecules ---------- */

/* Radial integral of the classical-form kernel, I(a, b) = int_0^R r^2 sinc(a r) sinc(b r) dr
 * (sinc x = sin x / x), in closed form.  For a, b > 0 it is (1/ab) int_0^R sin(ar) sin(br) dr
 * = [sin((a-b)R) / (2(a-b)) - sin((a+b)R) / (2(a+b))] / (ab); the cases a = b, a = 0 or b = 0
 * are the limits of the same integral. */
double oracle_classical_radial(double a, double b, double R)
{
    const double tiny = 1e-12;
    if (a < tiny && b < tiny) return R * R * R / 3.0;
    if (a < tiny || b < tiny) {
        const double c = a < tiny ? b : a;     /* (1/c) int_0^R r sin(c r) dr */
        return (sin(c * R) / (c * c) - R * cos(c * R) / c) / c;
    }
    const double d = a - b, t = a + b;
    const double t1 = fabs(d) < tiny ? R / 2.0 : sin(d * R) / (2.0 * d);
    return (t1 - sin(t * R) / (2.0 * t)) / (a * b);
}

/* B_hat(l, m) of eq. classical_hatB for Maxwell molecules (B = 1/(4 pi)), for integer mode
 * vectors l, m (not reduced mod N).  With g = r e: the integral over omega of
 * exp(i pi r (l-m).omega / (2T)) is 4 pi sinc(pi r |l-m| / (2T)), the integral over the
 * directions e of exp(i pi r (l+m).e / (2T)) is 4 pi sinc(pi r |l+m| / (2T)), so
 * B_hat(l, m) = (1/(4 pi)) (4 pi)^2 I(pi |l+m| / (2T), pi |l-m| / (2T)). */
double oracle_classical_bhat(const int *l, const int *m, double T, double R)
{
    double s2 = 0.0, d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        s2 += (double)(l[a] + m[a]) * (l[a] + m[a]);
        d2 += (double)(l[a] - m[a]) * (l[a] - m[a]);
    }
    const double c = ORACLE_PI / (2.0 * T);
    return 4.0 * ORACLE_PI * oracle_classical_radial(c * sqrt(s2), c * sqrt(d2), R);
}

/* Q^sigma of the entropic Fourier method built on the classical form (the remark after
 * eq. EFMk): Qh_k = sum_{l,m} 1_N(l+m-k) (B^sigma(l,m) - B^sigma(m,m)) Fh_l Fh_m with
 * B^sigma(l,m) = sigma(l) sigma(m) B_hat(l,m) and B_hat from eq. classical_hatB (3D Maxwell
 * molecules, truncation radius p->Rtr, box p->T), by the plain double sum, then the inverse DFT.
 * B_hat depends on l, m only through |l+m|^2 and |l-m|^2 (integers up to 3 N^2), so it is
 * tabulated over those. */
int oracle_collide_classical(const oracle_params *p, const double *F, double *Q)
{
    if (p->d != 3 || p->N < 2) return -1;
    const int N = p->N;
    const int64_t M = ipow(N, 3);
    const int64_t nn = 3 * (int64_t)N * N + 1;
    double *tab = malloc(sizeof(double) * nn * nn);
    double *sig = malloc(sizeof(double) * M), *bmm = malloc(sizeof(double) * M);
    double *Fr = malloc(sizeof(double) * M), *Fi = malloc(sizeof(double) * M);
    double *Qr = malloc(sizeof(double) * M), *Qi = malloc(sizeof(double) * M);
    if (!tab || !sig || !bmm || !Fr || !Fi || !Qr || !Qi) {
        free(tab); free(sig); free(bmm); free(Fr); free(Fi); free(Qr); free(Qi);
        return -1;
    }
    const double c = ORACLE_PI / (2.0 * p->T);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; ++i)
        for (int64_t j = 0; j < nn; ++j)
            tab[i * nn + j] = 4.0 * ORACLE_PI * oracle_classical_radial(c * sqrt((double)i), c * sqrt((double)j), p->Rtr);
    filter_table(p, sig);
    oracle_dft(3, N, F, Fr, Fi);
    for (int64_t m = 0; m < M; ++m) {
        int64_t r = m, m2 = 0;
        for (int a = 0; a < 3; ++a) { const int k = mode_of(N, (int)(r % N)); r /= N; m2 += 4 * (int64_t)k * k; }
        bmm[m] = sig[m] * sig[m] * tab[m2 * nn + 0];
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < M; ++k) {
        double re = 0.0, im = 0.0;
        for (int64_t l = 0; l < M; ++l) {
            const int64_t m = diff_mod(3, N, k, l);
            if (sig[l] == 0.0 && bmm[m] == 0.0) continue;
            int64_t rl = l, rm = m, s2 = 0, d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const int la = mode_of(N, (int)(rl % N)), ma = mode_of(N, (int)(rm % N));
                rl /= N; rm /= N;
                s2 += (int64_t)(la + ma) * (la + ma);
                d2 += (int64_t)(la - ma) * (la - ma);
            }
            const double b = sig[l] * sig[m] * tab[s2 * nn + d2] - bmm[m];
            re += b * (Fr[l] * Fr[m] - Fi[l] * Fi[m]);
            im += b * (Fr[l] * Fi[m] + Fi[l] * Fr[m]);
        }
        Qr[k] = re; Qi[k] = im;
    }
    oracle_idft_real(3, N, Qr, Qi, Q);
    free(tab); free(sig); free(bmm); free(Fr); free(Fi); free(Qr); free(Qi);
    return 0;
}

/* Q^sigma at selected grid points (flat indices idx[0..npts)), from the rank-separated form
 * (eq. fastFGM evaluated by collocation):
 *   Q_r = sum_t w_t [sum_l sigma beta_t Fh_l E_l(r)] [sum_m sigma gamma_t Fh_m E_m(r)]
 *         - F_r [sum_m B^sigma(m,m) Fh_m E_m(r)].
 * Fh (the DFT of F, eq. DFT) is given; F_r is the grid value.  Cost O(npts R N^d). */
int oracle_collide_points_hat(const oracle_params *p, const double *Fr, const double *Fi, const double *F,
                              int npts, const int64_t *idx, double *Q)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    const int N = p->N, d = p->d;
    double *bmm = malloc(sizeof(double) * M);
    for (int64_t m = 0; m < M; ++m) bmm[m] = bsig(&kt, m, m);
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < npts; ++n) {
        int pj[3] = { 0, 0, 0 };
        int64_t s = idx[n];
        for (int a = d - 1; a >= 0; --a) { pj[a] = (int)(s % N) - N / 2; s /= N; }
        double *er = malloc(sizeof(double) * M), *ei = malloc(sizeof(double) * M);
        for (int64_t l = 0; l < M; ++l) {          /* E_l(r) */
            int64_t r = l;
            double ph = 0.0;
            for (int a = d - 1; a >= 0; --a) { ph += (double)mode_of(N, (int)(r % N)) * pj[a]; r /= N; }
            ph = 2.0 * ORACLE_PI * fmod(ph, (double)N) / N;
            er[l] = cos(ph); ei[l] = sin(ph);
        }
        double gain = 0.0;
        for (int t = 0; t < kt.T; ++t) {
            double ar = 0, ai = 0, br = 0, bi = 0;
            for (int64_t l = 0; l < M; ++l) {
                double sb = kt.sig[l] * kt.beta[t * M + l], sg = kt.sig[l] * kt.gamma[t * M + l];
                double xr = Fr[l] * er[l] - Fi[l] * ei[l], xi = Fr[l] * ei[l] + Fi[l] * er[l];
                ar += sb * xr; ai += sb * xi; br += sg * xr; bi += sg * xi;
            }
            gain += kt.w[t] * (ar * br - ai * bi);
        }
        double nr = 0;
        for (int64_t l = 0; l < M; ++l) nr += bmm[l] * (Fr[l] * er[l] - Fi[l] * ei[l]);
        Q[n] = gain - F[idx[n]] * nr;
        free(er); free(ei);
    }
    free(bmm); free_tables(&kt);
    return 0;
}

/* As oracle_collide_points_hat with Fh from the direct DFT, O(N^{2d} + npts R N^d). */
int oracle_collide_points(const oracle_params *p, const double *F, int npts, const int64_t *idx, double *Q)
{
    const int64_t M = ipow(p->N, p->d);
    double *Fr = malloc(sizeof(double) * M), *Fi = malloc(sizeof(double) * M);
    oracle_dft(p->d, p->N, F, Fr, Fi);
    int rc = oracle_collide_points_hat(p, Fr, Fi, F, npts, idx, Q);
    free(Fr); free(Fi);
    return rc;
}

/* G(y, z) = sum_{i,j} B^sigma(i,j) E_{-i}(y) E_{-j}(z) (eq. G / tildeG without the N^{-2d}
 * factor, i.e. the reading of eq. A_G), for one grid point z (flat index zi) and every grid
 * point y.  Output G[y] (real). */
int oracle_G(const oracle_params *p, int64_t zi, double *G)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    const int N = p->N, d = p->d;
    int zj[3] = { 0, 0, 0 };
    int64_t s = zi;
    for (int a = d - 1; a >= 0; --a) { zj[a] = (int)(s % N) - N / 2; s /= N; }
    double *cr = malloc(sizeof(double) * M), *ci = malloc(sizeof(double) * M);
    /* c_i = sum_j B(i, j) E_{-j}(z) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double re = 0, im = 0;
        for (int64_t j = 0; j < M; ++j) {
            int64_t r = j;
            double ph = 0.0;
            for (int a = d - 1; a >= 0; --a) { ph += (double)mode_of(N, (int)(r % N)) * zj[a]; r /= N; }
            ph = -2.0 * ORACLE_PI * fmod(ph, (double)N) / N;
            double b = bsig(&kt, i, j);
            re += b * cos(ph); im += b * sin(ph);
        }
        cr[i] = re; ci[i] = im;
    }
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < M; ++y) {
        int yj[3] = { 0, 0, 0 };
        int64_t t = y;
        for (int a = d - 1; a >= 0; --a) { yj[a] = (int)(t % N) - N / 2; t /= N; }
        double re = 0;
        for (int64_t i = 0; i < M; ++i) {
            int64_t r = i;
            double ph = 0.0;
            for (int a = d - 1; a >= 0; --a) { ph += (double)mode_of(N, (int)(r % N)) * yj[a]; r /= N; }
            ph = -2.0 * ORACLE_PI * fmod(ph, (double)N) / N;
            re += cr[i] * cos(ph) - ci[i] * sin(ph);
        }
        G[y] = re;
    }
    free(cr); free(ci); free_tables(&kt);
    return 0;
}

/* DVM form eq. Qsr: Q_r = sum_{p,q,s} A^{rs}_{pq} (F_p F_q - F_r F_s) with
 * A^{rs}_{pq} = N^{-2d} 1_N(r+s-p-q) G(p-s, q-s)  (eq. A_simplified / tildetildeA).
 * Brute force for tiny grids.  Also returns min over (y,z) of G and the largest asymmetry
 * |A^{rs}_{pq} - A^{pq}_{rs}| + |A^{rs}_{pq} - A^{rs}_{qp}| seen (checks of eq. symA). */
int oracle_dvm(const oracle_params *p, const double *F, double *Q, double *Gmin, double *asym)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    const int N = p->N, d = p->d;
    /* G on all grid differences: Gt[y * M + z], y, z flat grid indices of the difference vector
     * (j components taken mod N, stored at index (j mod N)). */
    double *Gt = malloc(sizeof(double) * M * M);
    double *er = malloc(sizeof(double) * M * M), *ei = malloc(sizeof(double) * M * M);
    if (!Gt || !er || !ei) { free(Gt); free(er); free(ei); free_tables(&kt); return -1; }
    for (int64_t i = 0; i < M; ++i)          /* E_{-i}(y), y with components j_a = y_a (mod N) */
        for (int64_t y = 0; y < M; ++y) {
            int64_t r = i, t = y;
            double ph = 0.0;
            for (int a = d - 1; a >= 0; --a) {
                ph += (double)mode_of(N, (int)(r % N)) * (double)(t % N);
                r /= N; t /= N;
            }
            ph = -2.0 * ORACLE_PI * fmod(ph, (double)N) / N;
            er[i * M + y] = cos(ph); ei[i * M + y] = sin(ph);
        }
    double *B = malloc(sizeof(double) * M * M);
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < M; ++j) B[i * M + j] = bsig(&kt, i, j);
    double gmin = 1e300;
#pragma omp parallel for schedule(static) reduction(min : gmin)
    for (int64_t y = 0; y < M; ++y)
        for (int64_t z = 0; z < M; ++z) {
            double g = 0.0;
            for (int64_t i = 0; i < M; ++i)
                for (int64_t j = 0; j < M; ++j) {
                    double ar = er[i * M + y], ai = ei[i * M + y];
                    double br = er[j * M + z], bi = ei[j * M + z];
                    g += B[i * M + j] * (ar * br - ai * bi);
                }
            Gt[y * M + z] = g;
            if (g < gmin) gmin = g;
        }
    const double scale = 1.0 / ((double)M * (double)M);
    /* grid flat index -> components (array index, j = i - N/2; differences taken mod N so the
     * offset cancels) */
    double amax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : amax)
    for (int64_t r = 0; r < M; ++r) {
        double acc = 0.0;
        for (int64_t pp = 0; pp < M; ++pp)
            for (int64_t q = 0; q < M; ++q) {
                /* s = p + q - r (mod N): the only s with 1_N(r+s-p-q) = 1 */
                int64_t s = 0, ps = 0, qs = 0, rq = 0, sq = 0, qr = 0, mul = 1;
                int64_t a_ = pp, b_ = q, c_ = r;
                for (int a = 0; a < d; ++a) {
                    int pa = (int)(a_ % N), qa = (int)(b_ % N), ra = (int)(c_ % N);
                    a_ /= N; b_ /= N; c_ /= N;
                    int sa = ((pa + qa - ra) % N + N) % N;
                    s += sa * mul;
                    ps += (((pa - sa) % N + N) % N) * mul;
                    qs += (((qa - sa) % N + N) % N) * mul;
                    rq += (((ra - qa) % N + N) % N) * mul;
                    sq += (((sa - qa) % N + N) % N) * mul;
                    qr += (((qa - ra) % N + N) % N) * mul;
                    mul *= N;
                }
                (void)qr;
                double A = scale * Gt[ps * M + qs];
                double Aswap = scale * Gt[rq * M + sq];          /* A^{pq}_{rs} = G(r-q, s-q) */
                double Apq = scale * Gt[qs * M + ps];            /* A^{rs}_{qp} = G(q-s, p-s) */
                double dv = fabs(A - Aswap) + fabs(A - Apq);
                if (dv > amax) amax = dv;
                acc += A * (F[pp] * F[q] - F[r] * F[s]);
            }
        Q[r] = acc;
    }
    if (Gmin) *Gmin = gmin;
    if (asym) *asym = amax;
    free(Gt); free(er); free(ei); free(B); free_tables(&kt);
    return 0;
}

/* Loss frequency nu_r = sum_m B^sigma(m,m) Fh_m E_m(r) on the grid, so that the loss part of
 * Q^sigma at r is F_r nu_r (the identity of eq. def_A and the DVM form eq. QCvr). */
int oracle_nu(const oracle_params *p, const double *F, double *nu)
{
    kern_tables kt;
    if (make_tables(p, &kt)) { free_tables(&kt); return -1; }
    const int64_t M = kt.M;
    double *Fr = malloc(sizeof(double) * M), *Fi = malloc(sizeof(double) * M);
    oracle_dft(p->d, p->N, F, Fr, Fi);
    for (int64_t m = 0; m < M; ++m) {
        double b = bsig(&kt, m, m);
        Fr[m] *= b; Fi[m] *= b;
    }
    oracle_idft_real(p->d, p->N, Fr, Fi, nu);
    free(Fr); free(Fi); free_tables(&kt);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
