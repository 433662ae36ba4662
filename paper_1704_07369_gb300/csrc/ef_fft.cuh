// ef_fft.cuh -- register-resident mixed-radix FFTs of small compile-time length (N <= 64,
// factors 2, 3, 4, 5) for one thread, plus two-for-one real<->half-complex transforms.
//
// Convention: fft<L, SIGN> computes X[k] = sum_n x[n] exp(SIGN 2 pi i n k / L) in place, input
// and output in natural order.  Twiddles exp(-2 pi i j / NTOP) of the top-level length come from a
// constant-memory table built at compile time; every index is known after unrolling, so each
// twiddle is a constant-bank operand of the multiply (no shared-memory table, no loads).
#pragma once

#include <cuda_runtime.h>

namespace ef {

template <typename T>
struct C2 {
    T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> c2(T x, T y) { return C2<T>{x, y}; }
template <typename T>
__device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return C2<T>{a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return C2<T>{a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) { return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename T>
__device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return C2<T>{a.x * s, a.y * s}; }
template <typename T>
__device__ __forceinline__ C2<T> cconj(C2<T> a) { return C2<T>{a.x, -a.y}; }
// multiply by SIGN * i
template <int SIGN, typename T>
__device__ __forceinline__ C2<T> mul_si(C2<T> a) { return SIGN > 0 ? C2<T>{-a.y, a.x} : C2<T>{a.y, -a.x}; }

__host__ __device__ constexpr int first_radix(int L) { return (L % 4 == 0) ? 4 : (L % 2 == 0) ? 2 : (L % 3 == 0) ? 3 : 5; }

// ---- compile-time twiddle table: exp(-2 pi i j / n) for the built lengths n, j < n
constexpr int kTwLens[8] = {8, 12, 16, 24, 32, 40, 48, 64};
constexpr int kTwTotal = 8 + 12 + 16 + 24 + 32 + 40 + 48 + 64;
__host__ __device__ constexpr int tw_offset(int n)
{
    int off = 0;
    for (int a = 0; a < 8 && kTwLens[a] != n; ++a) off += kTwLens[a];
    return off;
}
struct TwTable {
    double c[kTwTotal], s[kTwTotal];     // cos, -sin
    float cf[kTwTotal], sf[kTwTotal];
};
// cos and sin of x in [0, pi/4] by their Taylor series (30 terms: converged in double)
constexpr void taylor_cs(double x, double &c, double &s)
{
    double x2 = x * x, tc = 1.0, ts = x;
    c = 0.0;
    s = 0.0;
    for (int k = 0; k < 30; ++k) {
        c += tc;
        s += ts;
        tc *= -x2 / ((2.0 * k + 1.0) * (2.0 * k + 2.0));
        ts *= -x2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
}
// cos and sin of 2 pi num / den: exact integer reduction to an octant, then the series on the
// distance r in [0, pi/4] to the octant's even boundary (cos / sin swapped on odd octants)
constexpr void cs_turn(long num, long den, double &c, double &s)
{
    constexpr double pi = 3.14159265358979323846264338327950288;
    num %= den;
    if (num < 0) num += den;
    const long o = (8 * num) / den;
    const long rnum = (o % 2 == 0) ? 8 * num - o * den : (o + 1) * den - 8 * num;
    double c0 = 0.0, s0 = 0.0;
    taylor_cs(2.0 * pi * (double)rnum / (8.0 * (double)den), c0, s0);
    switch (o) {
    case 0: c = c0; s = s0; break;
    case 1: c = s0; s = c0; break;
    case 2: c = -s0; s = c0; break;
    case 3: c = -c0; s = s0; break;
    case 4: c = -c0; s = -s0; break;
    case 5: c = -s0; s = -c0; break;
    case 6: c = s0; s = -c0; break;
    default: c = c0; s = -s0; break;
    }
}
constexpr TwTable make_tw_table()
{
    TwTable t{};
    int off = 0;
    for (int a = 0; a < 8; ++a) {
        for (int j = 0; j < kTwLens[a]; ++j) {
            double c = 0.0, s = 0.0;
            cs_turn(j, kTwLens[a], c, s);
            t.c[off + j] = c;
            t.s[off + j] = -s;
            t.cf[off + j] = (float)c;
            t.sf[off + j] = (float)(-s);
        }
        off += kTwLens[a];
    }
    return t;
}
static __constant__ TwTable c_tw = make_tw_table();

template <int NTOP, typename T>
__device__ __forceinline__ C2<T> tw_value(int j)
{
    constexpr int off = tw_offset(NTOP);
    static_assert(off < kTwTotal, "twiddle length not in the table");
    if constexpr (sizeof(T) == 4) return C2<T>{c_tw.cf[off + j], c_tw.sf[off + j]};
    else return C2<T>{c_tw.c[off + j], c_tw.s[off + j]};
}

// exp(SIGN 2 pi i e / L) with L | NTOP and 0 <= e < L
template <int L, int SIGN, int NTOP, typename T>
__device__ __forceinline__ C2<T> twiddle_mul(C2<T> v, int e)
{
    const int j = e * (NTOP / L);
    if (j == 0) return v;
    if (2 * j == NTOP) return C2<T>{-v.x, -v.y};
    if (4 * j == NTOP) return mul_si<SIGN>(v);            // exp(SIGN i pi/2) = SIGN i
    if (4 * j == 3 * NTOP) return mul_si<-SIGN>(v);
    C2<T> w = tw_value<NTOP, T>(j);
    if (SIGN > 0) w.y = -w.y;
    return cmul(v, w);
}

// In-place length-P DFT with exp(SIGN 2 pi i / P), P in {2, 3, 4, 5}
template <int P, int SIGN, typename T>
__device__ __forceinline__ void butterfly(C2<T> (&t)[P])
{
    if constexpr (P == 2) {
        C2<T> a = t[0], b = t[1];
        t[0] = a + b;
        t[1] = a - b;
    } else if constexpr (P == 4) {
        C2<T> s02 = t[0] + t[2], d02 = t[0] - t[2];
        C2<T> s13 = t[1] + t[3], d13 = mul_si<SIGN>(t[1] - t[3]);
        t[0] = s02 + s13;
        t[2] = s02 - s13;
        t[1] = d02 + d13;
        t[3] = d02 - d13;
    } else if constexpr (P == 3) {
        const T h = T(-0.5);
        const T s3 = T(SIGN) * T(0.86602540378443864676372317075294);   // sin(2 pi / 3)
        C2<T> a = t[0], s = t[1] + t[2], d = t[1] - t[2];
        C2<T> m = C2<T>{a.x + h * s.x, a.y + h * s.y};
        C2<T> r = C2<T>{-s3 * d.y, s3 * d.x};                           // i s3 d
        t[0] = a + s;
        t[1] = m + r;
        t[2] = m - r;
    } else {  // P == 5
        const T c1 = T(0.30901699437494742410229341718282);    // cos(2 pi / 5)
        const T c2v = T(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
        const T s1 = T(SIGN) * T(0.95105651629515357211643933337938);  // sin(2 pi / 5)
        const T s2 = T(SIGN) * T(0.58778525229247312916870595463907);  // sin(4 pi / 5)
        C2<T> a = t[0];
        C2<T> t1 = t[1] + t[4], u1 = t[1] - t[4];
        C2<T> t2 = t[2] + t[3], u2 = t[2] - t[3];
        C2<T> m1 = C2<T>{a.x + c1 * t1.x + c2v * t2.x, a.y + c1 * t1.y + c2v * t2.y};
        C2<T> m2 = C2<T>{a.x + c2v * t1.x + c1 * t2.x, a.y + c2v * t1.y + c1 * t2.y};
        C2<T> v1 = C2<T>{s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y};
        C2<T> v2 = C2<T>{s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y};
        // multiply by i
        C2<T> iv1 = C2<T>{-v1.y, v1.x}, iv2 = C2<T>{-v2.y, v2.x};
        t[0] = C2<T>{a.x + t1.x + t2.x, a.y + t1.y + t2.y};
        t[1] = m1 + iv1;
        t[4] = m1 - iv1;
        t[2] = m2 + iv2;
        t[3] = m2 - iv2;
    }
}

// Decimation in time: X[k1 + Q k2] = sum_p W_L^{p k1} W_P^{p k2} Y_p[k1], Y_p = DFT_Q(x[p + P m]).
template <int L, int SIGN, int NTOP, typename T>
__device__ __forceinline__ void fft(C2<T> (&x)[L])
{
    if constexpr (L == 1) {
        return;
    } else {
        constexpr int P = first_radix(L);
        constexpr int Qn = L / P;
        if constexpr (Qn == 1) {
            butterfly<P, SIGN>(x);
        } else {
            C2<T> y[P][Qn];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int m = 0; m < Qn; ++m) y[p][m] = x[p + P * m];
#pragma unroll
            for (int p = 0; p < P; ++p) fft<Qn, SIGN, NTOP>(y[p]);
#pragma unroll
            for (int k1 = 0; k1 < Qn; ++k1) {
                C2<T> t[P];
#pragma unroll
                for (int p = 0; p < P; ++p) t[p] = twiddle_mul<L, SIGN, NTOP>(y[p][k1], p * k1);
                butterfly<P, SIGN>(t);
#pragma unroll
                for (int k2 = 0; k2 < P; ++k2) x[k1 + Qn * k2] = t[k2];
            }
        }
    }
}

// Two real rows -> their half spectra (k = 0 .. N/2), forward sign, unscaled.
template <int N, typename T>
__device__ __forceinline__ void r2c_pair(const T (&r1)[N], const T (&r2)[N], C2<T> (&X1)[N / 2 + 1],
                                         C2<T> (&X2)[N / 2 + 1])
{
    C2<T> z[N];
#pragma unroll
    for (int n = 0; n < N; ++n) z[n] = C2<T>{r1[n], r2[n]};
    fft<N, -1, N>(z);
#pragma unroll
    for (int k = 0; k <= N / 2; ++k) {
        C2<T> a = z[k], b = cconj(z[(N - k) % N]);
        C2<T> s = a + b, d = a - b;
        X1[k] = C2<T>{T(0.5) * s.x, T(0.5) * s.y};
        X2[k] = C2<T>{T(0.5) * d.y, T(-0.5) * d.x};
    }
}

// Two Hermitian half spectra (k = 0 .. N/2) -> two real rows, inverse sign, unscaled.  The
// imaginary parts of the k = 0 and k = N/2 entries are ignored, as for any real inverse.
template <int N, typename T>
__device__ __forceinline__ void c2r_pair(const C2<T> (&X1)[N / 2 + 1], const C2<T> (&X2)[N / 2 + 1], T (&r1)[N],
                                         T (&r2)[N])
{
    C2<T> z[N];
    z[0] = C2<T>{X1[0].x, X2[0].x};
#pragma unroll
    for (int k = 1; k < N / 2; ++k) {
        z[k] = C2<T>{X1[k].x - X2[k].y, X1[k].y + X2[k].x};
        z[N - k] = C2<T>{X1[k].x + X2[k].y, X2[k].x - X1[k].y};
    }
    z[N / 2] = C2<T>{X1[N / 2].x, X2[N / 2].x};
    fft<N, 1, N>(z);
#pragma unroll
    for (int n = 0; n < N; ++n) {
        r1[n] = z[n].x;
        r2[n] = z[n].y;
    }
}

}  // namespace ef
