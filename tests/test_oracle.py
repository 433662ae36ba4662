"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped gain or loss term, a
wrong sign, a wrong aliasing index, a wrong kernel constant or filter) fails at least one:

* the modified Jackson filter against an independent closed form (autocorrelation of a sine
  sequence, Fejer-Riesz), which also proves chi^sigma >= 0 (Sec. 3.2.2);
* Tables 1 and 2 of the paper (2D BKW, Sec. 4.2, Example 1) reproduced from the printed values;
* the DVM form (eq. Qsr with A^sigma of eq. A_simplified) equal to the Fourier form (eq. Qsk) by
  brute force on tiny grids, with A^sigma >= 0 and symmetric (Sec. 3.2);
* the unfiltered kernel G taking negative values while the filtered one does not (Fig. 1);
* mass conservation, the discrete H-theorem and non-negativity (Theorem 1);
* closed-form loss frequencies: nu = mass for Maxwell molecules, nu(0) = sqrt(8/pi) for hard
  spheres against a unit Maxwellian;
* the BKW solution as an exact solution: Q[f_BKW] -> d f_BKW / dt as N grows;
* grid symmetries (translation, reflection, axis swap).
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
T_PAPER = (3.0 * np.sqrt(2.0) + 1.0) * 6.0 / 4.0   # T = (3 sqrt 2 + 1) R / 4 with R = 6


def _load_table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return {int(r[0]): r[1:] for r in rows}


def _within_print(ours, printed, sig):
    unit = 10.0 ** (np.floor(np.log10(abs(printed))) - (sig - 1))
    return abs(ours - printed) <= unit * 1.0001


# ------------------------------------------------------------------ filter --------------

@pytest.mark.parametrize("N", [7, 8, 9, 16, 17, 24, 32, 48, 64])
def test_jackson_filter_equals_sine_autocorrelation(N):
    n = (N - 1) // 2 if N % 2 else N // 2
    a = np.sin(np.pi * (np.arange(n) + 1) / (n + 1))
    ac = [(a[: n - k] * a[k:]).sum() / (a * a).sum() for k in range(n)] + [0.0]
    for k in range(n + 1):
        assert abs(oracle.sigma1(N, k) - ac[k]) < 1e-14
        assert abs(oracle.sigma1(N, -k) - ac[k]) < 1e-14
    assert oracle.sigma1(N, 0) == pytest.approx(1.0, abs=1e-15)
    assert oracle.sigma1(N, 1) == pytest.approx(np.cos(np.pi / (n + 1)), abs=1e-14)
    if N % 2 == 0:
        assert oracle.sigma1(N, -N // 2) == 0.0
    # chi^sigma(x) = sum_k sigma(k) e^{ikx} >= 0 everywhere (dense x)
    x = np.linspace(-np.pi, np.pi, 2001)
    k = np.arange(-n, n + 1)
    s = np.array([oracle.sigma1(N, int(kk)) for kk in k])
    chi = (s[None, :] * np.cos(np.outer(x, k))).sum(1)
    assert chi.min() > -1e-12


# --------------------------------------------------------------- paper tables ----------

def _bkw2d_errors(N, M):
    p = oracle.Params(d=2, N=N, T=T_PAPER, kernel=oracle.KERNEL_MAXWELL, R=2 * M, Rtr=6.0)
    V = oracle.grid(2, N, T_PAPER)
    F = oracle.ssp_rk3(p, oracle.bkw2d(0.0, V), 0.01)
    return oracle.rel_errors(F, oracle.bkw2d(0.01, V))


@pytest.mark.parametrize("N", [16, 32, 64])
def test_table2_fast_algorithm_l1(N):
    """Table 2: every printed entry for N <= 64, to the printed 5 significant figures."""
    tab = _load_table("table2_fast_l1.txt")
    for M, printed in zip((2, 3, 32), tab[N]):
        l1 = _bkw2d_errors(N, M)[0]
        assert _within_print(l1, printed, 5), (N, M, l1, printed)


def test_table2_n128_m2():
    tab = _load_table("table2_fast_l1.txt")
    l1 = _bkw2d_errors(128, 2)[0]
    assert _within_print(l1, tab[128][0], 5), l1


@pytest.mark.parametrize("N", [16, 32, 64])
def test_table1_bkw2d_errors(N):
    """Table 1: l1, l2, l_inf to the printed 3 significant figures (M = 32 angular samples)."""
    tab = _load_table("table1_bkw2d.txt")
    errs = _bkw2d_errors(N, 32)
    for e, printed in zip(errs, tab[N]):
        assert _within_print(e, printed, 3), (N, e, printed)


def test_table2_rejects_other_even_n_readings():
    """The reading matters: truncating F's -N/2 modes in the loss term (instead of multiplying the
    grid value F_r) or using T = 8 both miss Table 2 at N = 16."""
    tab = _load_table("table2_fast_l1.txt")
    p = oracle.Params(d=2, N=16, T=8.0, kernel=oracle.KERNEL_MAXWELL, R=4, Rtr=6.0)
    V = oracle.grid(2, 16, 8.0)
    F = oracle.ssp_rk3(p, oracle.bkw2d(0.0, V), 0.01)
    l1 = oracle.rel_errors(F, oracle.bkw2d(0.01, V))[0]
    assert not _within_print(l1, tab[16][0], 5)


# ------------------------------------------------------------- DVM equivalence ----------

CASES_TINY = [
    dict(d=2, N=6, kernel=0, R=8),
    dict(d=2, N=7, kernel=0, R=4),
    dict(d=2, N=8, kernel=0, R=4),
    dict(d=3, N=4, kernel=1, R=16),
    dict(d=3, N=4, kernel=2, R=16, J=3),
]


@pytest.mark.parametrize("case", CASES_TINY)
def test_dvm_form_equals_fourier_form(case):
    rng = np.random.default_rng(7)
    p = oracle.Params(T=T_PAPER, Rtr=6.0, **case)
    F = rng.random((case["N"],) * case["d"]) + 0.05
    Q = oracle.collide(p, F)
    Qd, gmin, asym = oracle.dvm(p, F)
    scale = np.abs(Q).max()
    assert np.abs(Q - Qd).max() <= 1e-13 * scale
    # A^sigma >= 0 (eq. tildetildeA) up to round-off, and symmetric (eq. symA)
    # G sums N^{2d} kernel modes of size up to B(0,0), so round-off is relative to that sum
    G0 = oracle.G_slice(p, 0)
    w, b, g = oracle.factors(p)
    bscale = float((w * b[:, 0] * g[:, 0]).sum()) * case["N"] ** case["d"]
    assert gmin >= -1e-13 * bscale
    assert asym <= 1e-13 * bscale / float(case["N"] ** (2 * case["d"]))
    # the rank-separated point form agrees too
    idx = np.arange(F.size)
    Qp = oracle.collide_points(p, F, idx)
    assert np.abs(Q.ravel() - Qp).max() <= 1e-13 * scale


@pytest.mark.parametrize("d,N", [(2, 6), (2, 8), (2, 12), (2, 7), (3, 6), (3, 8), (3, 12)])
def test_fft_helper_equals_direct_dft(d, N):
    """The NumPy-FFT helper used for large grids (dft_fft, with the phase of the centred index
    j = i - N/2) equals the direct sum of eq. DFT, and both equal the closed form of a point mass:
    F = delta at j0 gives Fh_k = N^-d exp(-2 pi i k.j0 / N)."""
    rng = np.random.default_rng(N + 10 * d)
    F = rng.random((N,) * d)
    a = oracle.dft(F)
    b = oracle.dft_fft(F)
    assert np.abs(a - b).max() <= 1e-15 * np.abs(F).sum()
    i0 = tuple(int(x) for x in rng.integers(0, N, d))
    D = np.zeros((N,) * d)
    D[i0] = 1.0
    k = [((np.arange(N) + N // 2) % N) - N // 2] * d       # k in FFT order: 0..N/2-1, -N/2..-1
    kk = np.meshgrid(*k, indexing="ij")
    j0 = [i - N // 2 for i in i0]
    exact = np.exp(-2j * np.pi * sum(kk[a_] * j0[a_] for a_ in range(d)) / N) / N ** d
    assert np.abs(oracle.dft(D) - exact).max() <= 1e-15
    assert np.abs(oracle.dft_fft(D) - exact).max() <= 1e-15


@pytest.mark.parametrize("case", [dict(d=2, N=12, kernel=0, R=8), dict(d=3, N=8, kernel=1, R=16),
                                  dict(d=3, N=6, kernel=2, R=16, J=3)])
def test_sampled_evaluators_equal_the_full_sum(case):
    """The point evaluators used at large N (rank-separated form, with Fh from the direct DFT or from
    the FFT helper) equal the direct double sum of eq. Qsk at every grid point."""
    rng = np.random.default_rng(11)
    p = oracle.Params(T=8.0, **case)
    F = rng.random((case["N"],) * case["d"]) + 0.05
    Q = oracle.collide(p, F).ravel()
    idx = np.arange(F.size)
    scale = np.abs(Q).max()
    assert np.abs(oracle.collide_points(p, F, idx) - Q).max() <= 1e-13 * scale
    assert np.abs(oracle.collide_points_fft(p, F, idx) - Q).max() <= 1e-13 * scale


@pytest.mark.parametrize("case", [dict(d=2, N=12, kernel=0, R=8, filter=False), dict(d=2, N=12, kernel=0, R=8, filter=True),
                                  dict(d=3, N=8, kernel=1, R=16, filter=False)])
def test_galerkin_sum_equals_collocation_for_band_limited_data(case):
    """The Fourier Galerkin sum (eq. FGM_Q) differs from the collocation sum (eq. Qsk) only by the
    products l + m that leave the mode set and wrap mod N.  For F whose spectrum lies in
    |k_a| <= N/4 - 1 no product wraps, so the two must agree; for generic F they must not."""
    rng = np.random.default_rng(21)
    N, d = case["N"], case["d"]
    p = oracle.Params(T=8.0, **case)
    X = np.zeros((N,) * d, dtype=complex)
    band = N // 4 - 1
    ks = [list(range(0, band + 1)) + list(range(N - band, N))] * d
    for idx in np.ndindex(*[len(k) for k in ks]):
        X[tuple(ks[a][i] for a, i in enumerate(idx))] = rng.normal() + 1j * rng.normal()
    F = np.real(np.fft.ifftn(X)) * N ** d + 3.0
    Qg = oracle.collide_galerkin(p, F)
    Qc = oracle.collide(p, F)
    assert np.abs(Qg - Qc).max() <= 1e-12 * np.abs(Qc).max()
    G = rng.random((N,) * d) + 0.1                          # generic data: aliasing present
    Qg, Qc = oracle.collide_galerkin(p, G), oracle.collide(p, G)
    assert np.abs(Qg - Qc).max() >= 1e-4 * np.abs(Qc).max()
    # mass is conserved exactly (B(l,-l) = B(-l,-l) by eq. sym_B) and translation commutes
    assert abs(Qg.sum()) <= 1e-13 * np.abs(Qg).sum()
    shift = tuple(range(d))
    Qs = oracle.collide_galerkin(p, np.roll(G, 1, axis=shift))
    assert np.abs(Qs - np.roll(Qg, 1, axis=shift)).max() <= 1e-12 * np.abs(Qg).max()


def test_unfiltered_kernel_is_not_positive_fig1():
    """Fig. 1: 2D, B~ = 1/pi, R = 6, N = 32, z = (T/2, T/2): G takes negative values without the
    filter and is non-negative with it (Sec. 3.2.1 / 3.2.2)."""
    N = 32
    z = (N // 2 + N // 4) * N + (N // 2 + N // 4)   # j = (N/4, N/4)  ->  v = (T/2, T/2)
    pf = oracle.Params(d=2, N=N, T=T_PAPER, kernel=0, R=64, Rtr=6.0, filter=False)
    ps = oracle.Params(d=2, N=N, T=T_PAPER, kernel=0, R=64, Rtr=6.0, filter=True)
    G = oracle.G_slice(pf, z)
    Gs = oracle.G_slice(ps, z)
    assert G.min() < -1e-2 * G.max()
    assert Gs.min() >= -1e-12 * Gs.max()


# --------------------------------------------------------------- Theorem 1 --------------

CASES_SMALL = [
    dict(d=2, N=16, kernel=0, R=16, T=8.0),
    dict(d=2, N=15, kernel=0, R=8, T=8.0),
    dict(d=3, N=8, kernel=1, R=32, T=8.0),
    dict(d=3, N=8, kernel=2, R=16, T=8.0, J=4),
]


def _bumpy(d, N, T, seed):
    rng = np.random.default_rng(seed)
    V = oracle.grid(d, N, T)
    F = np.zeros((N,) * d)
    for _ in range(3):
        c = rng.uniform(-2, 2, d)
        w = rng.uniform(0.6, 1.5)
        F += rng.uniform(0.3, 1.0) * np.exp(-sum((x - ci) ** 2 for x, ci in zip(V, c)) / (2 * w * w))
    return F


@pytest.mark.parametrize("case", CASES_SMALL)
def test_mass_conservation_and_h_theorem(case):
    p = oracle.Params(**case)
    F = _bumpy(case["d"], case["N"], case["T"], 3)
    Q = oracle.collide(p, F)
    gain_scale = np.abs(Q).sum() + np.abs(F * oracle.nu(p, F)).sum()
    assert abs(Q.sum()) <= 1e-13 * gain_scale
    prod = (Q * np.log(F)).sum()
    assert prod < 0.0


@pytest.mark.parametrize("case", CASES_SMALL)
def test_positivity_under_small_euler_steps(case):
    """With gain >= 0 and nu >= 0 the forward Euler update F + dt Q stays >= 0 whenever
    dt max(nu) <= 1, even where F is exactly 0 (proof of Theorem 1)."""
    p = oracle.Params(**case)
    F = _bumpy(case["d"], case["N"], case["T"], 5)
    F[F < 0.2 * F.max()] = 0.0
    nu = oracle.nu(p, F)
    assert nu.min() >= -1e-12 * nu.max()
    dt = 1.0 / nu.max()
    Q = oracle.collide(p, F)
    Fn = F + dt * Q
    assert Fn.min() >= -1e-12 * F.max()
    gain = Q + F * nu
    assert gain.min() >= -1e-12 * np.abs(gain).max()


# --------------------------------------------------------- closed-form pins ---------------

def test_loss_frequency_maxwell_2d_equals_mass():
    """For Maxwell molecules nu(v) = int B domega dv* f = mass (unit mass here)."""
    T = 8.0
    for N, tol in ((16, 6e-3), (32, 1e-3)):
        p = oracle.Params(d=2, N=N, T=T, kernel=0, R=16)
        V = oracle.grid(2, N, T)
        F = np.exp(-sum(x * x for x in V) / 2) / (2 * np.pi)
        nu = oracle.nu(p, F)
        core = sum(x * x for x in V) < 4
        assert np.abs(nu[core] - 1.0).max() < tol


def test_loss_frequency_hard_sphere_3d():
    """For B = |g|/(4 pi): nu(v) = int |v - v*| f(v*) dv*; at v = 0 for a unit Maxwellian this is
    sqrt(8/pi).  The filter smooths nu at second order, so check the unfiltered collocation kernel
    (filter off) at the centre and the filtered one converging to it."""
    T = 8.0
    exact = np.sqrt(8.0 / np.pi)
    vals = {}
    for N, filt in ((24, False), (16, True), (24, True)):
        p = oracle.Params(d=3, N=N, T=T, kernel=1, R=32, filter=filt)
        V = oracle.grid(3, N, T)
        F = np.exp(-sum(x * x for x in V) / 2) / (2 * np.pi) ** 1.5
        vals[(N, filt)] = oracle.nu(p, F)[N // 2, N // 2, N // 2]
    assert abs(vals[(24, False)] - exact) < 1e-3 * exact
    e16, e24 = abs(vals[(16, True)] - exact), abs(vals[(24, True)] - exact)
    assert e24 < e16 * (16.0 / 24.0) ** 1.2


def test_loss_frequency_maxwell_3d_equals_mass():
    T = 8.0
    p = oracle.Params(d=3, N=16, T=T, kernel=2, R=32, J=8, filter=False)
    V = oracle.grid(3, 16, T)
    F = np.exp(-sum(x * x for x in V) / 2) / (2 * np.pi) ** 1.5
    assert abs(oracle.nu(p, F)[8, 8, 8] - 1.0) < 3e-3


def _dfdt(fn, t, V, h=1e-4):
    return (fn(t + h, V) - fn(t - h, V)) / (2 * h)


def test_bkw2d_is_a_fixed_point_of_the_discrete_dynamics_in_the_limit():
    """Q^sigma[f_BKW] approaches d f_BKW/dt at second order in N (Sec. 3.4)."""
    T = 8.0
    errs = []
    for N in (16, 32, 64):
        p = oracle.Params(d=2, N=N, T=T, kernel=0, R=16)
        V = oracle.grid(2, N, T)
        f = oracle.bkw2d(1.0, V)
        Q = oracle.collide(p, f)
        ex = _dfdt(oracle.bkw2d, 1.0, V)
        errs.append(np.abs(Q - ex).max() / np.abs(ex).max())
    assert errs[1] < errs[0] / 2.2 and errs[2] < errs[1] / 2.8, errs


def test_bkw3d_maxwell_consistency():
    """3D Maxwell molecules: Q^sigma[f_BKW(0)] approaches d f_BKW/dt(0) as N grows (max norm)."""
    T = 8.0
    errs = []
    for N in (12, 16):
        p = oracle.Params(d=3, N=N, T=T, kernel=2, R=32, J=6)
        V = oracle.grid(3, N, T)
        Q = oracle.collide(p, oracle.bkw3d(0.0, V))
        ex = (oracle.bkw3d(2e-4, V) - oracle.bkw3d(0.0, V)) / 2e-4
        errs.append(np.abs(Q - ex).max() / np.abs(ex).max())
    assert errs[1] < 0.8 * errs[0] and errs[1] < 0.45, errs


def test_unfiltered_collocation_maxwellian_is_near_equilibrium():
    """Without the filter (Fourier collocation) a Maxwellian is an equilibrium to spectral
    accuracy; with it, to second order in N.  A wrong sign or a dropped gain/loss term fails."""
    T = 8.0
    res = {}
    for N in (16, 32):
        V = oracle.grid(2, N, T)
        F = np.exp(-sum(x * x for x in V) / 2) / (2 * np.pi)
        for filt in (False, True):
            p = oracle.Params(d=2, N=N, T=T, kernel=0, R=16, filter=filt)
            loss = np.abs(F * oracle.nu(p, F)).max()
            res[(N, filt)] = np.abs(oracle.collide(p, F)).max() / loss
    assert res[(32, False)] < 1e-7
    assert res[(32, True)] < 0.2 and res[(32, True)] < res[(16, True)] / 2.2


# ---------------------------------------------------------------- symmetries --------------

def test_translation_reflection_and_axis_swap_equivariance():
    T = 8.0
    rng = np.random.default_rng(11)
    F = rng.random((12, 12)) + 0.1
    p = oracle.Params(d=2, N=12, T=T, kernel=0, R=8)
    Q = oracle.collide(p, F)
    Qs = oracle.collide(p, np.roll(F, (3, -2), axis=(0, 1)))
    assert np.abs(Qs - np.roll(Q, (3, -2), axis=(0, 1))).max() < 1e-13 * np.abs(Q).max()
    refl = lambda A: np.roll(A[::-1, :], 1, axis=0)          # j -> -j (mod N) on axis 0
    assert np.abs(oracle.collide(p, refl(F)) - refl(Q)).max() < 1e-13 * np.abs(Q).max()
    assert np.abs(oracle.collide(p, F.T.copy()) - Q.T).max() < 1e-13 * np.abs(Q).max()
    F3 = rng.random((6, 6, 6)) + 0.1
    p3 = oracle.Params(d=3, N=6, T=T, kernel=1, R=16)
    Q3 = oracle.collide(p3, F3)
    Q3s = oracle.collide(p3, np.roll(F3, (1, 2, -1), axis=(0, 1, 2)))
    assert np.abs(Q3s - np.roll(Q3, (1, 2, -1), axis=(0, 1, 2))).max() < 1e-13 * np.abs(Q3).max()


# ------------------------------------------------ classical form, Table 3 ------------------

T_CLASSICAL = (3.0 + np.sqrt(2.0)) * 6.0 / 4.0   # T = (3 + sqrt 2) R / 4 with R = 6 (classical form)


def test_classical_radial_integral_closed_form():
    """int_0^R r^2 sinc(ar) sinc(br) dr: closed form against composite Gauss-Legendre, including the
    limits a = 0, b = 0, a = b and a close to b."""
    x, w = np.polynomial.legendre.leggauss(40)
    R = 6.0
    edges = np.linspace(0.0, R, 41)
    r = np.concatenate([0.5 * (e1 - e0) * x + 0.5 * (e0 + e1) for e0, e1 in zip(edges[:-1], edges[1:])])
    wr = np.concatenate([0.5 * (e1 - e0) * w for e0, e1 in zip(edges[:-1], edges[1:])])
    for a, b in ((0.0, 0.0), (0.0, 1.3), (0.7, 0.0), (1.1, 1.1), (0.9, 0.9 + 1e-9), (0.4, 2.5), (3.0, 1.7)):
        f = r ** 2 * np.sinc(a * r / np.pi) * np.sinc(b * r / np.pi)
        assert oracle.classical_radial(a, b, R) == pytest.approx(float((f * wr).sum()), rel=1e-12, abs=1e-12)


def test_classical_bhat_against_the_defining_integral():
    """B_hat(l, m) of eq. classical_hatB (B = 1/(4 pi)) against a product quadrature of the
    5-dimensional integral over g in the ball and omega on the sphere, without the closed forms."""
    T, R = T_CLASSICAL, 6.0
    xr, wr = np.polynomial.legendre.leggauss(40)
    r, wr = 0.5 * R * (xr + 1.0), 0.5 * R * wr
    xm, wm = np.polynomial.legendre.leggauss(24)
    nphi = 24
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    wphi = np.full(nphi, 2.0 * np.pi / nphi)
    st = np.sqrt(1.0 - xm ** 2)
    dirs = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                     np.repeat(xm, nphi)], axis=1)                       # unit vectors
    wdir = np.outer(wm, wphi).ravel()
    for l, m in (((1, 0, 0), (0, 2, 1)), ((2, -1, 0), (-1, 0, 3)), ((0, 0, 0), (1, 1, 1)), ((3, 2, -2), (3, 2, -2))):
        l, m = np.array(l, float), np.array(m, float)
        c = np.pi / (2.0 * T)
        tot = 0.0
        for ri, wri in zip(r, wr):
            g = ri * dirs                                                 # g over the ball
            ph_g = c * (g @ (l + m))
            ph_w = c * ri * (dirs @ (l - m))                              # |g| omega . (l - m)
            s = np.exp(1j * ph_g).dot(wdir) * np.exp(1j * ph_w).dot(wdir)
            tot += wri * ri ** 2 * s.real
        ref = tot / (4.0 * np.pi)
        assert oracle.classical_bhat(l.astype(int), m.astype(int), T, R) == pytest.approx(ref, rel=1e-7)


def _bkw3d_classical_errors(N):
    p = oracle.Params(d=3, N=N, T=T_CLASSICAL, kernel=oracle.KERNEL_MAXWELL, R=32, Rtr=6.0)
    V = oracle.grid(3, N, T_CLASSICAL)
    F = oracle.ssp_rk3_with(lambda X: oracle.collide_classical(p, X), oracle.bkw3d(0.0, V), 0.01)
    return oracle.rel_errors(F, oracle.bkw3d(0.01, V))


def test_table3_classical_form_n16():
    """Table 3 at N = 16: l2 and l_inf to the printed 3 figures; l1 = 4.0675e-3 against the printed
    4.08e-3 (0.3%, 1.25 units of the last printed digit)."""
    tab = _load_table("table3_bkw3d.txt")
    l1, l2, linf = _bkw3d_classical_errors(16)
    assert _within_print(l2, tab[16][1], 3) and _within_print(linf, tab[16][2], 3), (l2, linf)
    assert abs(l1 - tab[16][0]) <= 0.0035 * tab[16][0], l1


def test_table3_classical_form_n32():
    """Table 3 at N = 32: all three errors to the printed 3 significant figures."""
    tab = _load_table("table3_bkw3d.txt")
    for e, printed in zip(_bkw3d_classical_errors(32), tab[32]):
        assert _within_print(e, printed, 3), (e, printed)


def test_classical_form_conserves_mass_and_dissipates_entropy():
    N = 12
    p = oracle.Params(d=3, N=N, T=T_CLASSICAL, kernel=oracle.KERNEL_MAXWELL, R=32, Rtr=6.0)
    V = oracle.grid(3, N, T_CLASSICAL)
    F = oracle.bkw3d(0.0, V)
    Q = oracle.collide_classical(p, F)
    assert abs(Q.sum()) <= 1e-13 * np.abs(Q).sum()
    assert (Q[F > 0] * np.log(F[F > 0])).sum() < 0


# ---------------------------------------------- spatially inhomogeneous coupling (Sec. 5) -------

def _cells(M, N, d, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.1, 1.0, size=(M,) + (N,) * d)


def test_transport_keeps_a_spatially_uniform_state():
    F = np.stack([_cells(1, 8, 2, 3)[0]] * 5)
    out = oracle.transport_upwind(F, 4.0, 0.5, 0.1)
    assert np.array_equal(out, F)


def test_transport_at_courant_one_is_the_exact_shift():
    """N = 8, T = 4: h = 1, the first-axis indices 7 and 1 carry v = +3 and -3.  With dt / dx = 1/3
    their Courant numbers are +1 and -1: those slices move one cell up and one cell down; index 4
    (v = 0) stays."""
    F = _cells(6, 8, 2, 5)
    out = oracle.transport_upwind(F, 4.0, 3.0, 1.0)
    assert np.allclose(out[:, 7], np.roll(F, 1, axis=0)[:, 7], rtol=0, atol=1e-15)
    assert np.allclose(out[:, 1], np.roll(F, -1, axis=0)[:, 1], rtol=0, atol=1e-15)
    assert np.array_equal(out[:, 4], F[:, 4])


def test_transport_conserves_mass_per_velocity_and_keeps_positivity_below_courant_one():
    F = _cells(9, 8, 3, 7)
    T, dx = 4.0, 1.0
    vmax = 4.0                                   # |v| <= (N/2) h
    out = oracle.transport_upwind(F, T, dx, 0.9 * dx / vmax)
    assert np.allclose(out.sum(axis=0), F.sum(axis=0), rtol=1e-14, atol=0)
    assert out.min() >= 0.0
    # beyond Courant number one the upwind step is no longer a convex combination
    G = np.zeros_like(F)
    G[4] = 1.0
    bad = oracle.transport_upwind(G, T, dx, 2.0 * dx / vmax)
    assert bad.min() < 0.0


def test_transport_converges_at_first_order_to_the_exact_shift():
    """A smooth periodic profile in x, carried by each velocity: the upwind error at a fixed time,
    with dt / dx fixed, halves when dx halves."""
    N, T, Lx, t_end = 8, 4.0, 1.0, 0.125
    h = 2.0 * T / N
    v = (np.arange(N) - N // 2) * h

    def err(M):
        dx = Lx / M
        dt = 0.5 * dx / np.abs(v).max()
        steps = int(round(t_end / dt))
        x = np.arange(M) * dx
        F = np.stack([1.0 + 0.5 * np.sin(2 * np.pi * xi / Lx) * np.ones((N, N)) for xi in x])
        for _ in range(steps):
            F = oracle.transport_upwind(F, T, dx, dt)
        exact = 1.0 + 0.5 * np.sin(2 * np.pi * (x[:, None] - v[None, :] * steps * dt) / Lx)
        return np.abs(F[:, :, 0] - exact).max()

    e1, e2, e3 = err(64), err(128), err(256)
    assert 1.8 < e1 / e2 < 2.2 and 1.8 < e2 / e3 < 2.2, (e1, e2, e3)


def test_lie_splitting_conserves_total_mass():
    p = oracle.Params(d=2, N=8, T=4.0, kernel=oracle.KERNEL_MAXWELL, R=16)
    F = _cells(4, 8, 2, 11)
    out = oracle.inhomogeneous_lie(p, F, 0.5, 0.02, steps=2)
    assert abs(out.sum() - F.sum()) <= 1e-13 * F.sum()
    assert out.min() >= 0.0
