"""Parity of the CUDA path (through the C ABI) against the FP64 oracle, on seeded inputs.

Bars: FP64 rel-L2 <= 1e-12; FP32 max |Q_gpu - Q_oracle| <= 2e-5 max |Q_oracle| (the same
tolerances for the sampled full-size cases, over the sampled points).  Sizes span several cells,
clusters of 1 to 16 CTAs, ragged batches and the largest built N.
"""
import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _dtype(prec):
    return torch.float32 if prec == ef.EF_PREC_F32 else torch.float64


def gpu_collide(d, N, L, kernel, R, prec, cells, **ex):
    plan = ef.Plan(d, N, L, kernel, R, prec, **ex)
    F = torch.tensor(np.stack(cells), dtype=_dtype(prec), device="cuda").contiguous()
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=len(cells))
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    return Q.double().cpu().numpy(), plan


def rel_l2(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def check(prec, got, ref):
    if prec == ef.EF_PREC_F64:
        assert rel_l2(got, ref) <= F64_TOL, rel_l2(got, ref)
    else:
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= F32_TOL, err


def oparams(d, N, L, kernel, R, **ex):
    return oracle.Params(d=d, N=N, T=L, kernel=kernel, R=R, J=ex.get("J", 6),
                         filter=ex.get("sigma_enabled", 1) != 0)


# -------------------------------------------------------------- 2D (config 1 family) --------

def test_config1_2d_collide_and_100_euler_steps_fp64():
    """2D, N=16, L=8, Maxwell, R=16, FP64, bi-Gaussian at +-1.5: one Q evaluation and 100 forward
    Euler steps (dt = 0.01), against the oracle; FP64 diagnostics against the oracle's."""
    N, L, R = 16, 8.0, 16
    F0 = inputs.bigauss2d(N, L)
    p = oparams(2, N, L, 0, R)
    Q, plan = gpu_collide(2, N, L, ef.EF_KERNEL_MAXWELL, R, ef.EF_PREC_F64, [F0])
    check(ef.EF_PREC_F64, Q[0], oracle.collide(p, F0))

    F = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
    diag = torch.zeros(100, 1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.euler(F, 0.01, nsteps=100, diag=diag, ncells=1)
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    Fo = F0.copy()
    ref_diag = []
    for _ in range(100):
        Qo = oracle.collide(p, Fo)
        ref_diag.append(oracle.moments(Fo, L, Qo))
        Fo = Fo + 0.01 * Qo
    got = F[0].cpu().numpy()
    assert rel_l2(got, Fo) <= F64_TOL
    dg = diag.cpu().numpy()[:, 0, :]
    ref = np.array(ref_diag)
    # [mass, mom0, mom1, (mom2), energy, eta, production, min F] of the oracle's moments()
    for k_gpu, k_ref in ((0, 0), (1, 1), (2, 2), (4, 3), (5, 4), (6, 5), (7, 6)):
        scale = np.abs(ref[:, k_ref]).max() + 1e-300
        assert np.abs(dg[:, k_gpu] - ref[:, k_ref]).max() <= 1e-11 * max(scale, 1e-3), (k_gpu,)
    # mass conserved, entropy production <= 0, positivity kept (Theorem 1)
    assert np.abs(dg[:, 0] - dg[0, 0]).max() <= 1e-13
    assert (dg[:, 6] <= 0).all()
    assert dg[:, 9].min() >= -1e-14 * F0.max()


@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64])
@pytest.mark.parametrize("prec", [ef.EF_PREC_F64, ef.EF_PREC_F32])
def test_2d_sizes(N, prec):
    L, R = 8.0, 16
    rng = np.random.default_rng(N)
    cells = [inputs.bigauss2d(N, L, shift=s) for s in rng.uniform(0.5, 2.0, 3)]
    Q, _ = gpu_collide(2, N, L, ef.EF_KERNEL_MAXWELL, R, prec, cells)
    p = oparams(2, N, L, 0, R)
    for i, c in enumerate(cells):
        check(prec, Q[i], oracle.collide(p, c))


# ----------------------------------------------------------------------- 3D ------------------

@pytest.mark.parametrize("N", [8, 12, 16])
@pytest.mark.parametrize("prec", [ef.EF_PREC_F64, ef.EF_PREC_F32])
def test_3d_hard_sphere_cells(N, prec):
    L, R = 8.0, 32
    cells = [inputs.mixture_cell(3, N, L, 100 + i) for i in range(3)]
    Q, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, prec, cells)
    p = oparams(3, N, L, 1, R)
    for i, c in enumerate(cells):
        check(prec, Q[i], oracle.collide(p, c))


@pytest.mark.parametrize("N", [8, 12])
@pytest.mark.parametrize("prec", [ef.EF_PREC_F64, ef.EF_PREC_F32])
def test_3d_maxwell_cells(N, prec):
    L, R = 8.0, 32
    cells = [inputs.bkw(3, N, L, 5.5), inputs.mixture_cell(3, N, L, 7)]
    Q, _ = gpu_collide(3, N, L, ef.EF_KERNEL_MAXWELL, R, prec, cells)
    p = oparams(3, N, L, 0, R)
    for i, c in enumerate(cells):
        check(prec, Q[i], oracle.collide(p, c))


def test_3d_unfiltered_and_custom_quadrature():
    """sigma off (Fourier collocation) and an explicit (n_mu, n_phi, n_c) and R_tr."""
    N, L = 8, 8.0
    cells = [inputs.mixture_cell(3, N, L, 3)]
    Q, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 24, ef.EF_PREC_F64, cells,
                       n_mu=3, n_phi=2, n_c=2, R_tr=5.0, sigma_enabled=0)
    p = oracle.Params(d=3, N=N, T=L, kernel=1, R=24, Rtr=5.0, filter=False, angular=(3, 2, 2))
    check(ef.EF_PREC_F64, Q[0], oracle.collide(p, cells[0]))


def _sample_idx(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, k)]))


def _check_sampled(prec, Q, p, F, seed, k=24):
    idx = _sample_idx(F.size, k, seed)
    ref = oracle.collide_points_fft(p, F, idx)
    got = Q.ravel()[idx]
    if prec == ef.EF_PREC_F64:
        assert rel_l2(got, ref) <= F64_TOL, rel_l2(got, ref)
    else:
        # the bar is relative to max |Q| over the cell; GPU FP64 supplies the scale
        return got, ref, idx


@pytest.mark.parametrize("N", [24, 32, 40, 48, 64])
def test_3d_hard_sphere_large_sizes_sampled(N):
    """FP64 against the oracle at sampled points; FP32 against FP64 over the whole cell."""
    L, R = 8.0, 32
    cells = [inputs.mixture_cell(3, N, L, 11)]
    Q64, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F64, cells)
    p = oparams(3, N, L, 1, R)
    _check_sampled(ef.EF_PREC_F64, Q64[0], p, cells[0], N)
    Q32, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32, cells)
    err = np.abs(Q32[0] - Q64[0]).max() / np.abs(Q64[0]).max()
    assert err <= F32_TOL, err
    # mass conservation over the whole cell
    assert abs(Q64[0].sum()) <= 1e-12 * np.abs(Q64[0]).sum()


def test_batched_ragged_cells_against_oracle():
    L, R = 8.0, 32
    Ns = [8, 12, 16, 12, 8, 16, 8, 12]
    cells = [inputs.mixture_cell(3, n, L, 500 + i) for i, n in enumerate(Ns)]
    for prec in (ef.EF_PREC_F64, ef.EF_PREC_F32):
        plan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, R, prec, batched_N=Ns)
        F = torch.tensor(inputs.pack(cells), dtype=_dtype(prec), device="cuda")
        Q = torch.empty_like(F)
        plan.collide(F, Q)
        torch.cuda.synchronize()
        assert plan.status() == ef.EF_OK
        Qh = Q.double().cpu().numpy()
        off = 0
        for n, c in zip(Ns, cells):
            ref = oracle.collide(oparams(3, n, L, 1, R), c)
            check(prec, Qh[off:off + n ** 3].reshape(c.shape), ref)
            off += n ** 3
        # graph replay gives the same bits
        plan.set_graph(True)
        Q2 = torch.empty_like(F)
        plan.collide(F, Q2)
        plan.collide(F, Q2)
        torch.cuda.synchronize()
        assert torch.equal(Q, Q2)


# --------------------------------------------------------------- full-size configurations ----

def test_config3_batched_4096_ragged_cells_sampled():
    """4096 cells, N ~ U{24,32,40,48}, L=8, hard spheres, R=32, FP32 (the benchmark's launch,
    graph-captured): sampled points of one cell per N against the oracle, and mass conservation
    plus the sign of the entropy production on every cell."""
    L, R = 8.0, 32
    Ns = inputs.ragged_sizes(4096, seed=1234)
    plan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32, batched_N=Ns)
    plan.set_graph(True)
    offs = np.concatenate([[0], np.cumsum(Ns.astype(np.int64) ** 3)])
    F = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    picks = {}
    for i, n in enumerate(Ns):
        c = inputs.mixture_cell(3, int(n), L, 1234 + i)
        F[offs[i]:offs[i + 1]] = torch.from_numpy(c.ravel()).float()
        if int(n) not in picks:
            picks[int(n)] = (i, c)
    Q = torch.empty_like(F)
    plan.collide(F, Q)
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    for n, (i, c) in sorted(picks.items()):
        q = Q[offs[i]:offs[i + 1]].double().cpu().numpy()
        # the FP32 bar is relative to max |Q| of the cell; take the scale from the GPU cell
        idx = _sample_idx(c.size, 24, n)
        ref = oracle.collide_points_fft(oparams(3, n, L, 1, R), c.astype(np.float32).astype(np.float64), idx)
        err = np.abs(q[idx] - ref).max() / np.abs(q).max()
        assert err <= F32_TOL, (n, err)
    # every cell: sum Q = 0 (FP32 round-off) and sum Q ln F <= 0
    out = torch.zeros(4096, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.moments(F, Q, out)
    torch.cuda.synchronize()
    prod = out[:, 6].cpu().numpy()
    assert (prod < 0).all()
    Qd = Q.double()
    sums = torch.stack([Qd[offs[i]:offs[i + 1]].sum() for i in range(0, 4096, 64)]).cpu().numpy()
    absums = torch.stack([Qd[offs[i]:offs[i + 1]].abs().sum() for i in range(0, 4096, 64)]).cpu().numpy()
    assert (np.abs(sums) <= 1e-5 * absums).all()


def test_config2_bkw_trajectory_fp64_and_fp32():
    """3D, N=32, L=8, Maxwell molecules, R=32: BKW at t0 = 5.5; sampled FP64 parity; 200 Euler
    steps (dt = 0.01) in FP64 and FP32, compared with BKW(t0 + n dt) along the way; mass
    conserved, F >= 0 and sum Q ln F <= 0 at every step, FP32 tracking FP64.

    BKW at t0 = 5.5 is close to equilibrium, where the filter's second-order smoothing dominates
    Q^sigma (Sec. 3.4): the discrete solution relaxes towards the scheme's own equilibrium and its
    distance to BKW grows about linearly in time (about 0.14 per unit time at N = 32); the check
    is that it stays on that line (no instability), not that it vanishes."""
    N, L, R, dt = 32, 8.0, 32, 0.01
    F0 = inputs.bkw(3, N, L, 5.5)
    Q64, plan64 = gpu_collide(3, N, L, ef.EF_KERNEL_MAXWELL, R, ef.EF_PREC_F64, [F0])
    _check_sampled(ef.EF_PREC_F64, Q64[0], oparams(3, N, L, 0, R), F0, 2, k=12)
    plan32 = ef.Plan(3, N, L, ef.EF_KERNEL_MAXWELL, R, ef.EF_PREC_F32)
    F64 = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
    F32 = F64.float()
    d64 = torch.zeros(200, 1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    d32 = torch.zeros_like(d64)
    errs = []
    for n in range(200):
        plan64.euler(F64, dt, 1, d64[n:n + 1], ncells=1)
        plan32.euler(F32, dt, 1, d32[n:n + 1], ncells=1)
        if n % 20 == 19:
            ex = inputs.bkw(3, N, L, 5.5 + (n + 1) * dt)
            errs.append(rel_l2(F64[0].cpu().numpy(), ex))
    torch.cuda.synchronize()
    assert plan64.status() == ef.EF_OK and plan32.status() == ef.EF_OK
    dg = d64.cpu().numpy()[:, 0]
    assert np.abs(dg[:, 0] - dg[0, 0]).max() <= 1e-12 * dg[0, 0]
    assert (dg[:, 9] >= -1e-14 * F0.max()).all() and (dg[:, 6] <= 0).all()
    errs = np.array(errs)
    slope = errs[0]
    assert (np.diff(errs) > 0).all() and (np.diff(errs) < 1.5 * slope).all(), errs
    assert errs[-1] < 12 * slope, errs
    a, b = F32[0].double(), F64[0]
    assert ((a - b).abs().max() / b.abs().max()).item() <= 1e-4


def test_config4_n64_hard_sphere_precision():
    """3D, N=64, L=10, hard spheres, R=64 (config-2 family cells): FP64 against the oracle at
    sampled points, FP32 against FP64 over whole cells, mass and entropy production per cell."""
    N, L, R = 64, 10.0, 64
    cells = list(inputs.bkw_family_cells(3, N, L, 4, seed=99))
    Q64, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F64, cells)
    Q32, _ = gpu_collide(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32, cells)
    _check_sampled(ef.EF_PREC_F64, Q64[0], oparams(3, N, L, 1, R), cells[0], 64, k=8)
    for i in range(len(cells)):
        err = np.abs(Q32[i] - Q64[i]).max() / np.abs(Q64[i]).max()
        assert err <= F32_TOL, err
        assert abs(Q64[i].sum()) <= 1e-12 * np.abs(Q64[i]).sum()


# --------------------------------------------------------------------- edge cases ------------

def test_edge_cases_and_errors():
    N, L = 8, 8.0
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64)
    F = torch.zeros(2, N, N, N, dtype=torch.float64, device="cuda")
    Q = torch.full_like(F, 7.0)
    plan.collide(F, Q, ncells=0)                 # empty batch: nothing written
    torch.cuda.synchronize()
    assert (Q == 7.0).all()
    plan.collide(F, Q, ncells=2)                 # F = 0 -> Q = 0
    torch.cuda.synchronize()
    assert (Q == 0).all()
    F.fill_(0.25)                                # constant F: only the zero mode, Q = 0
    plan.collide(F, Q, ncells=2)
    torch.cuda.synchronize()
    # gain and loss are each B(0,0) Fh_0^2 ~ 5e2 here; they cancel to round-off
    assert Q.abs().max().item() <= 1e-14 * 8721.3 * 0.25 ** 2 * 8
    F.zero_()                                    # a single point mass: gain >= 0 everywhere else
    F[0, 3, 4, 5] = 1.0
    plan.collide(F, Q, ncells=2)
    torch.cuda.synchronize()
    q = Q[0].cpu().numpy()
    ref = oracle.collide(oparams(3, N, L, 1, 32), F[0].cpu().numpy())
    assert rel_l2(q, ref) <= F64_TOL
    with pytest.raises(ef.EfError):
        ef.Plan(3, 36, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)      # not a built size
    with pytest.raises(ef.EfError):
        ef.Plan(3, 7, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)       # odd N
    with pytest.raises(ef.EfError):
        ef.Plan(2, 16, L, ef.EF_KERNEL_MAXWELL, 15, ef.EF_PREC_F32)          # odd R in 2D
    with pytest.raises(ef.EfError):
        ef.Plan(2, 16, L, ef.EF_KERNEL_HARD_SPHERE, 16, ef.EF_PREC_F32)      # 2D hard spheres
    with pytest.raises(ef.EfError):
        ef.Plan(3, 16, -1.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)   # L <= 0
    with pytest.raises(ef.EfError):
        ef.ef_collide(plan.handle, None, Q, 1)
    with pytest.raises(ef.EfError):
        ef.ef_collide(plan.handle, F, F, 1)                                   # aliasing
    bplan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64, batched_N=[8, 12])
    with pytest.raises(ef.EfError):
        ef.ef_collide(bplan.handle, F, Q, 3)                                  # wrong cell count


def test_status_word_positivity_and_nan():
    N, L = 8, 8.0
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64)
    F = torch.tensor(inputs.mixture_cell(3, N, L, 1)[None], dtype=torch.float64, device="cuda")
    F[0, F[0] < 0.2 * F.max()] = 0.0
    plan.euler(F, 50.0, nsteps=1, ncells=1)      # dt max nu >> 1: positivity not guaranteed
    assert plan.status(sync=1, reset=1) == ef.EF_ERR_POSITIVITY
    assert plan.status(sync=1) == ef.EF_OK
    F.fill_(float("nan"))
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=1)
    assert plan.status(sync=1, reset=1) == ef.EF_ERR_NOT_FINITE


def test_moments_kernel_against_oracle():
    L = 8.0
    for d, N, prec in ((3, 16, ef.EF_PREC_F64), (2, 32, ef.EF_PREC_F64), (3, 12, ef.EF_PREC_F32)):
        cells = [inputs.mixture_cell(d, N, L, 40 + i) for i in range(2)]
        kern = ef.EF_KERNEL_HARD_SPHERE if d == 3 else ef.EF_KERNEL_MAXWELL
        plan = ef.Plan(d, N, L, kern, 32 if d == 3 else 16, prec)
        F = torch.tensor(np.stack(cells), dtype=_dtype(prec), device="cuda")
        Q = torch.empty_like(F)
        plan.collide(F, Q, ncells=2)
        out = torch.zeros(2, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
        plan.moments(F, Q, out, ncells=2)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for i in range(2):
            Fi = F[i].double().cpu().numpy()
            ref = oracle.moments(Fi, L, Q[i].double().cpu().numpy())
            k_gpu = [0, 1, 2] + ([3] if d == 3 else []) + [4, 5, 6, 7]
            # FP32 input: each lane sums runs of at most 32 float4 partials, keeps the runs' total in
            # a compensated FP32 pair, and a warp adds its lanes in FP32: the error is at most about
            # (3 + 32 + 8) * 2^-24 of the sum of |terms| (a few times max(1, |ref|))
            tol = 1e-12 if prec == ef.EF_PREC_F64 else 1e-5
            for kg, kr in zip(k_gpu, range(len(ref))):
                assert abs(o[i, kg] - ref[kr]) <= tol * max(1.0, abs(ref[kr])), (d, kg)
            assert abs(o[i, 8] - oracle.positivity_error(Fi)) <= 1e-15
        # positivity error of Sec. 4.2 on cells with negative values
        Fn = F - 0.02 * F.amax()
        plan.moments(Fn, None, out, ncells=2)
        torch.cuda.synchronize()
        for i in range(2):
            eps = oracle.positivity_error(Fn[i].double().cpu().numpy())
            assert eps > 1e-3
            assert abs(out[i, 8].item() - eps) <= (1e-12 if prec == ef.EF_PREC_F64 else 1e-5) * eps, (d, N)
