"""FP64 CPU oracle for the entropic Fourier method (EFM) collision operator.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  The library's product path never
imports, links or executes anything here, and nothing here imports the product package.

The arithmetic lives in ``ef_oracle.c`` (plain C, double precision, OpenMP), built into
``liboracle.so`` by :func:`build`.  This module adds the parts that are plain NumPy:

* the BKW closed-form solutions in 2D and 3D (Sec. 4.2, Examples 1 and 4);
* the relative l_p errors of Sec. 4.2, the positivity error epsilon and the discrete entropy
  eta = (2T/N)^d sum F ln F;
* third-order SSP Runge-Kutta and forward Euler steppers over the oracle operator (Sec. 4.1);
* moments and entropy production of a grid function;
* the spatially inhomogeneous coupling (left to future work in Sec. 5): first-order upwind free
  transport between cells that are the points of a periodic 1D spatial grid, and Lie splitting of
  transport and collision.

Kernel numbering follows the library's C header: 0 = Maxwell molecules (2D, B = 1/(2 pi)),
1 = hard spheres (3D, B = |g|/(4 pi)), 2 = Maxwell molecules (3D, B = 1/(4 pi)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ef_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KERNEL_MAXWELL = 0
KERNEL_HARD_SPHERE = 1


def build(force: bool = False) -> str:
    """Compile ``ef_oracle.c`` into ``liboracle.so`` beside it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("kernel", ctypes.c_int), ("R", ctypes.c_int),
        ("nmu", ctypes.c_int), ("nphi", ctypes.c_int), ("nc", ctypes.c_int), ("J", ctypes.c_int),
        ("filter", ctypes.c_int), ("pad", ctypes.c_int),
        ("T", ctypes.c_double), ("Rtr", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.oracle_sigma1.restype = ctypes.c_double
        lib.oracle_sigma1.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_nterms.argtypes = [pp]
        lib.oracle_factors.argtypes = [pp, dp, dp, dp]
        lib.oracle_dft.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.oracle_idft_real.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.oracle_collide.argtypes = [pp, dp, dp]
        lib.oracle_collide_points.argtypes = [pp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp]
        lib.oracle_collide_points_hat.argtypes = [pp, dp, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp]
        lib.oracle_G.argtypes = [pp, ctypes.c_int64, dp]
        lib.oracle_dvm.argtypes = [pp, dp, dp, dp, dp]
        lib.oracle_nu.argtypes = [pp, dp, dp]
        lib.oracle_classical_radial.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_classical_radial.restype = ctypes.c_double
        lib.oracle_classical_bhat.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_double, ctypes.c_double]
        lib.oracle_classical_bhat.restype = ctypes.c_double
        lib.oracle_collide_classical.argtypes = [pp, dp, dp]
        lib.oracle_collide_galerkin.argtypes = [pp, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def default_rtr(T: float) -> float:
    """Largest truncation radius allowed by T >= (3 sqrt(2) + 1) R / 4 (Sec. 1.2)."""
    return 4.0 * T / (3.0 * np.sqrt(2.0) + 1.0)


def default_angular(R: int):
    """(n_mu, n_phi, n_c) with 2 n_mu n_phi n_c = R for the 3D angular quadrature."""
    table = {8: (1, 2, 2), 16: (1, 4, 2), 32: (2, 4, 2), 64: (2, 4, 4), 128: (4, 4, 4)}
    if R not in table:
        raise ValueError("no default 3D angular factorisation for R=%d" % R)
    return table[R]


@dataclass
class Params:
    """Discretisation of one EFM operator (mirrors the library's plan description)."""
    d: int
    N: int
    T: float
    kernel: int
    R: int
    Rtr: float | None = None
    J: int = 4
    filter: bool = True
    angular: tuple | None = None

    def c(self) -> _Params:
        p = _Params()
        p.d, p.N, p.R, p.J = self.d, self.N, self.R, self.J
        if self.d == 2:
            if self.kernel != KERNEL_MAXWELL:
                raise ValueError("2D supports Maxwell molecules only")
            p.kernel = 0
        else:
            p.kernel = 1 if self.kernel == KERNEL_HARD_SPHERE else 2
            nmu, nphi, nc = self.angular or default_angular(self.R)
            if 2 * nmu * nphi * nc != self.R:
                raise ValueError("angular factorisation does not match R")
            p.nmu, p.nphi, p.nc = nmu, nphi, nc
        p.filter = 1 if self.filter else 0
        p.T = float(self.T)
        p.Rtr = float(self.Rtr if self.Rtr is not None else default_rtr(self.T))
        return p


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sigma1(N: int, k: int) -> float:
    return _load().oracle_sigma1(N, k)


def factors(p: Params):
    """(w[t], beta[t, modes], gamma[t, modes]) of B_fast = sum_t w_t beta_t(l) gamma_t(m)."""
    lib = _load()
    cp = p.c()
    T = lib.oracle_nterms(ctypes.byref(cp))
    M = p.N ** p.d
    w = np.zeros(T)
    b = np.zeros((T, M))
    g = np.zeros((T, M))
    if lib.oracle_factors(ctypes.byref(cp), _dp(w), _dp(b), _dp(g)):
        raise ValueError("bad parameters")
    return w, b, g


def dft(F: np.ndarray):
    F = np.ascontiguousarray(F, dtype=np.float64)
    d, N = F.ndim, F.shape[0]
    re = np.zeros(F.size)
    im = np.zeros(F.size)
    _load().oracle_dft(d, N, _dp(F), _dp(re), _dp(im))
    return (re + 1j * im).reshape(F.shape)


def idft_real(Fh: np.ndarray):
    re = np.ascontiguousarray(Fh.real, dtype=np.float64)
    im = np.ascontiguousarray(Fh.imag, dtype=np.float64)
    out = np.zeros(Fh.size)
    _load().oracle_idft_real(Fh.ndim, Fh.shape[0], _dp(re), _dp(im), _dp(out))
    return out.reshape(Fh.shape)


def collide(p: Params, F: np.ndarray) -> np.ndarray:
    """Q^sigma[F] on the grid by the direct O(R N^{2d}) double sum (eq. Qsk)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    assert F.shape == (p.N,) * p.d
    Q = np.zeros_like(F)
    if _load().oracle_collide(ctypes.byref(p.c()), _dp(F), _dp(Q)):
        raise ValueError("bad parameters")
    return Q


def classical_radial(a: float, b: float, R: float) -> float:
    """int_0^R r^2 sinc(a r) sinc(b r) dr in closed form (the radial factor of eq. classical_hatB)."""
    return _load().oracle_classical_radial(float(a), float(b), float(R))


def classical_bhat(l, m, T: float, R: float) -> float:
    """B_hat(l, m) of eq. classical_hatB for 3D Maxwell molecules (B = 1/(4 pi))."""
    la = (ctypes.c_int * 3)(*[int(x) for x in l])
    ma = (ctypes.c_int * 3)(*[int(x) for x in m])
    return _load().oracle_classical_bhat(la, ma, float(T), float(R))


def collide_classical(p: Params, F: np.ndarray) -> np.ndarray:
    """Q^sigma of the entropic Fourier method on the classical form of the operator (remark after
    eq. EFMk), 3D Maxwell molecules, by the direct double sum; uses p.N, p.T, p.Rtr, p.filter."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    assert p.d == 3 and F.shape == (p.N,) * 3
    Q = np.zeros_like(F)
    if _load().oracle_collide_classical(ctypes.byref(p.c()), _dp(F), _dp(Q)):
        raise ValueError("bad parameters")
    return Q


def collide_galerkin(p: Params, F: np.ndarray) -> np.ndarray:
    """The Fourier Galerkin method's collision term (eq. FGM_Q) on the grid: the unaliased sum over
    l + m = k in K (even N: modes with a component -N/2 dropped), the plan's low-rank kernel, the
    filter only if p.filter; Fh from the DFT of the grid values."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    assert F.shape == (p.N,) * p.d
    Q = np.zeros_like(F)
    if _load().oracle_collide_galerkin(ctypes.byref(p.c()), _dp(F), _dp(Q)):
        raise ValueError("bad parameters")
    return Q


def ssp_rk3_with(collide_fn, F: np.ndarray, dt: float, steps: int = 1):
    """SSP-RK3 (as ssp_rk3) for any operator F -> Q."""
    for _ in range(steps):
        F1 = F + dt * collide_fn(F)
        F2 = 0.75 * F + 0.25 * (F1 + dt * collide_fn(F1))
        F = F / 3.0 + 2.0 / 3.0 * (F2 + dt * collide_fn(F2))
    return F


def collide_points(p: Params, F: np.ndarray, idx) -> np.ndarray:
    """Q^sigma[F] at flat grid indices ``idx`` (rank-separated collocation form)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    Q = np.zeros(idx.size)
    if _load().oracle_collide_points(ctypes.byref(p.c()), _dp(F), int(idx.size),
                                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(Q)):
        raise ValueError("bad parameters")
    return Q


def dft_fft(F: np.ndarray) -> np.ndarray:
    """The DFT of eq. DFT computed with NumPy's FFT (a library primitive) for large grids:
    Fh_k = N^{-d} sum_j F_j exp(-2 pi i k.j / N) with j = i - N/2, i.e. the FFT over array
    indices times the phase (-1)^{sum k}."""
    F = np.asarray(F, dtype=np.float64)
    d, N = F.ndim, F.shape[0]
    Fh = np.fft.fftn(F) / F.size
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    ph = np.ones(())
    for a in range(d):
        shape = [1] * d
        shape[a] = N
        ph = ph * np.exp(1j * np.pi * k * (N // 2) * 2.0 / N).reshape(shape)
    return Fh * ph


def collide_points_fft(p: Params, F: np.ndarray, idx) -> np.ndarray:
    """Q^sigma[F] at flat grid indices ``idx``, rank-separated form, with Fh from NumPy's FFT."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    Fh = dft_fft(F)
    re = np.ascontiguousarray(Fh.real.ravel())
    im = np.ascontiguousarray(Fh.imag.ravel())
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    Q = np.zeros(idx.size)
    if _load().oracle_collide_points_hat(ctypes.byref(p.c()), _dp(re), _dp(im), _dp(F), int(idx.size),
                                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(Q)):
        raise ValueError("bad parameters")
    return Q


def nu(p: Params, F: np.ndarray) -> np.ndarray:
    """Loss frequency nu on the grid: the loss part of Q^sigma is F * nu."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros_like(F)
    if _load().oracle_nu(ctypes.byref(p.c()), _dp(F), _dp(out)):
        raise ValueError("bad parameters")
    return out


def G_slice(p: Params, z_index: int) -> np.ndarray:
    """G(y, z) for every grid point y at the grid point with flat index z_index."""
    out = np.zeros(p.N ** p.d)
    if _load().oracle_G(ctypes.byref(p.c()), int(z_index), _dp(out)):
        raise ValueError("bad parameters")
    return out.reshape((p.N,) * p.d)


def dvm(p: Params, F: np.ndarray):
    """DVM-form brute force (eq. Qsr).  Returns (Q, min G, max asymmetry of A)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    Q = np.zeros_like(F)
    gmin = ctypes.c_double()
    asym = ctypes.c_double()
    if _load().oracle_dvm(ctypes.byref(p.c()), _dp(F), _dp(Q), ctypes.byref(gmin), ctypes.byref(asym)):
        raise ValueError("bad parameters")
    return Q, gmin.value, asym.value


def num_threads() -> int:
    return _load().oracle_num_threads()


# ----------------------------------------------------------------- grid helpers ----------

def grid(d: int, N: int, T: float):
    """Velocity coordinates v = h j, j = -N/2 .. N/2-1, h = 2T/N (array index i = j + N/2)."""
    h = 2.0 * T / N
    v1 = (np.arange(N) - N // 2) * h
    return np.meshgrid(*([v1] * d), indexing="ij")


def bkw2d(t: float, V) -> np.ndarray:
    """2D BKW solution for Maxwell molecules, S = 1 - exp(-t/8)/2 (Sec. 4.2, Example 1)."""
    S = 1.0 - np.exp(-t / 8.0) / 2.0
    v2 = sum(x * x for x in V)
    return np.exp(-v2 / (2 * S)) / (2 * np.pi * S) * ((2 * S - 1) / S + (1 - S) / (2 * S * S) * v2)


def bkw3d(t: float, V) -> np.ndarray:
    """3D BKW solution for Maxwell molecules, S = 1 - 2 exp(-t/6)/5 (Sec. 4.2, Example 4)."""
    S = 1.0 - 2.0 * np.exp(-t / 6.0) / 5.0
    v2 = sum(x * x for x in V)
    return (np.exp(-v2 / (2 * S)) / (2 * np.pi * S) ** 1.5
            * ((5 * S - 3) / (2 * S) + (1 - S) / (2 * S * S) * v2))


def rel_errors(F: np.ndarray, f: np.ndarray):
    """Relative l1, l2, l_inf errors on the grid (Sec. 4.2)."""
    e = F - f
    return (np.abs(e).sum() / np.abs(f).sum(),
            np.sqrt((e * e).sum() / (f * f).sum()),
            np.abs(e).max() / np.abs(f).max())


def positivity_error(F: np.ndarray) -> float:
    """epsilon = (sum |F| - sum F) / sum |F|  (Sec. 4.2, Example 1)."""
    a = np.abs(F).sum()
    return float((a - F.sum()) / a)


def entropy(F: np.ndarray, T: float) -> float:
    """eta = (2T/N)^d sum F ln F with 0 ln 0 = 0 (Sec. 4.2)."""
    h = 2.0 * T / F.shape[0]
    Fp = F[F > 0]
    return float(h ** F.ndim * (Fp * np.log(Fp)).sum())


def moments(F: np.ndarray, T: float, Q: np.ndarray | None = None):
    """[mass, momentum_1..d, energy, eta, sum Q ln F, min F] with h^d quadrature weights.
    Momentum and energy use the grid velocities v = h j; energy is (1/2) sum |v|^2 F h^d."""
    d, N = F.ndim, F.shape[0]
    h = 2.0 * T / N
    V = grid(d, N, T)
    w = h ** d
    out = [w * F.sum()]
    out += [w * (F * v).sum() for v in V]
    out.append(0.5 * w * (F * sum(v * v for v in V)).sum())
    out.append(entropy(F, T))
    if Q is not None:
        pos = F > 0
        out.append(float((Q[pos] * np.log(F[pos])).sum()))
    else:
        out.append(0.0)
    out.append(float(F.min()))
    return np.array(out)


def ssp_rk3(p: Params, F: np.ndarray, dt: float, steps: int = 1):
    """Third-order SSP Runge-Kutta of Gottlieb, Shu & Tadmor, as used in Sec. 4.1."""
    for _ in range(steps):
        F1 = F + dt * collide(p, F)
        F2 = 0.75 * F + 0.25 * (F1 + dt * collide(p, F1))
        F = F / 3.0 + 2.0 / 3.0 * (F2 + dt * collide(p, F2))
    return F


def euler(p: Params, F: np.ndarray, dt: float, steps: int = 1):
    """Forward Euler F <- F + dt Q^sigma[F]."""
    for _ in range(steps):
        F = F + dt * collide(p, F)
    return F


# ------------------------------------------------- spatially inhomogeneous coupling ----------
# The paper leaves the spatially inhomogeneous equation to future work (Sec. 5).  Reading used here:
# the cells of a batch are the points x_i = i dx of a periodic 1D spatial grid, F moves along x with
# the velocity component of the first array axis, and free transport is discretised by first-order
# upwinding; transport and collision are combined by Lie splitting.

def transport_upwind(F: np.ndarray, T: float, dx: float, dt: float) -> np.ndarray:
    """One upwind step of dF/dt + v dF/dx = 0 on cells F[i] (shape [M, N, ...]), periodic in i, with
    v = h (j - N/2) the velocity of the first velocity axis and nu = v dt / dx:
    F_i - nu (F_i - F_{i-1}) where nu > 0, F_i - nu (F_{i+1} - F_i) where nu < 0."""
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[1]
    h = 2.0 * T / N
    nu = (np.arange(N) - N // 2) * h * dt / dx
    nu = nu.reshape([1, N] + [1] * (F.ndim - 2))
    left = np.roll(F, 1, axis=0)        # F_{i-1}
    right = np.roll(F, -1, axis=0)      # F_{i+1}
    return np.where(nu > 0, F - nu * (F - left), F - nu * (right - F))


def inhomogeneous_lie(p: Params, F: np.ndarray, dx: float, dt: float, steps: int = 1, rk3: bool = False):
    """Lie splitting: each step one upwind transport step, then one collision step (forward Euler or
    SSP-RK3 of the oracle operator) in every cell."""
    F = np.asarray(F, dtype=np.float64)
    for _ in range(steps):
        F = transport_upwind(F, p.T, dx, dt)
        F = np.stack([(ssp_rk3 if rk3 else euler)(p, c, dt) for c in F])
    return F
