"""Parity of the FP32 and FP64 CUDA paths against the FP64 oracle itself (never against the GPU's
own FP64 path) at the workload's sizes, and the boundary's no-allocation contract under stream
capture.

* Whole cells at N = 24 and 32 (3D hard spheres, R = 32): every grid point against the oracle's
  direct double sum of eq. Qsk, FP32 bar max |Q - Q_oracle| <= 2e-5 max |Q_oracle|.
* N = 40, 48 (L = 8, R = 32) and 64 (L = 10, R = 64): at least 400 sampled points, which include
  the points where the GPU's |Q| is largest, against the oracle's point evaluator; the scale of the
  FP32 bar is the oracle's largest |Q| over the sample.
* The entropy production sum Q ln F of the FP32 path near equilibrium (BKW cells at large t0 and a
  Maxwellian): the same sign as the oracle's, within the bound that the FP32 parity bar implies.
* Repeated ef_collide / ef_euler_step / ef_rk3_step calls captured into a CUDA graph: the capture
  succeeds (no allocation or synchronisation inside) and the replay reproduces the eager results.
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


def _gpu(N, L, R, prec, cells, kernel=ef.EF_KERNEL_HARD_SPHERE):
    plan = ef.Plan(3, N, L, kernel, R, prec)
    dt = torch.float32 if prec == ef.EF_PREC_F32 else torch.float64
    F = torch.tensor(np.stack(cells), dtype=dt, device="cuda")
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=len(cells))
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    return F.double().cpu().numpy(), Q.double().cpu().numpy()


@pytest.mark.parametrize("N", [24, 32])
def test_whole_cells_fp32_and_fp64_against_oracle(N):
    L, R = 8.0, 32
    cell = inputs.mixture_cell(3, N, L, 2024 + N)
    p = oracle.Params(d=3, N=N, T=L, kernel=oracle.KERNEL_HARD_SPHERE, R=R, J=6)
    # FP32: the oracle evaluates the FP32-rounded input, so only the arithmetic differs
    F32, Q32 = _gpu(N, L, R, ef.EF_PREC_F32, [cell])
    ref32 = oracle.collide(p, F32[0])
    err = np.abs(Q32[0] - ref32).max() / np.abs(ref32).max()
    assert err <= F32_TOL, err
    if N == 24:
        _, Q64 = _gpu(N, L, R, ef.EF_PREC_F64, [cell])
        ref = oracle.collide(p, cell)
        assert np.sqrt(((Q64[0] - ref) ** 2).sum() / (ref ** 2).sum()) <= F64_TOL


def _sample(Q_gpu, k, seed):
    rng = np.random.default_rng(seed)
    flat = np.abs(Q_gpu.ravel())
    top = np.argsort(flat)[-16:]                  # where |Q| peaks (the scale of the FP32 bar)
    return np.unique(np.concatenate([top, [0, flat.size - 1], rng.integers(0, flat.size, k)]))


@pytest.mark.parametrize("N,L,R", [(40, 8.0, 32), (48, 8.0, 32), (64, 10.0, 64)])
def test_sampled_points_fp32_against_oracle(N, L, R):
    cells = [inputs.mixture_cell(3, N, L, 77 + N)] if N < 64 else list(inputs.bkw_family_cells(3, N, L, 1, seed=5))
    F32, Q32 = _gpu(N, L, R, ef.EF_PREC_F32, cells)
    p = oracle.Params(d=3, N=N, T=L, kernel=oracle.KERNEL_HARD_SPHERE, R=R, J=6)
    idx = _sample(Q32[0], 400, N)
    assert idx.size >= 400
    ref = oracle.collide_points_fft(p, F32[0], idx)
    scale = np.abs(ref).max()
    assert scale >= 0.9 * np.abs(Q32[0]).max()   # the sample holds the peak of |Q|
    err = np.abs(Q32[0].ravel()[idx] - ref).max() / scale
    assert err <= F32_TOL, err
    if N == 40:
        _, Q64 = _gpu(N, L, R, ef.EF_PREC_F64, cells)
        ref64 = oracle.collide_points_fft(p, cells[0], idx)
        got = Q64[0].ravel()[idx]
        assert np.sqrt(((got - ref64) ** 2).sum() / (ref64 ** 2).sum()) <= F64_TOL


@pytest.mark.parametrize("kernel", [ef.EF_KERNEL_HARD_SPHERE, ef.EF_KERNEL_MAXWELL])
def test_fp32_entropy_production_sign_near_equilibrium(kernel):
    """sum Q ln F from the FP32 collide kernel's diagnostics (an Euler step with dt = 0) and from the
    FP32 moments kernel against the oracle's FP64 value on the same (FP32-rounded) cells: BKW at
    t0 = 10 and 40 and a Maxwellian.  The FP32 parity bar bounds the difference by
    2e-5 max|Q| sum |ln F| (plus FP32 summation error), which is below |P| here, so the sign is
    guaranteed and checked."""
    N, L, R = 24, 8.0, 32
    cells = [inputs.bkw(3, N, L, 10.0), inputs.bkw(3, N, L, 40.0), inputs.bkw(3, N, L, 1e9)]
    plan = ef.Plan(3, N, L, kernel, R, ef.EF_PREC_F32)
    F = torch.tensor(np.stack(cells), dtype=torch.float32, device="cuda")
    Fh = F.double().cpu().numpy()
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=3)
    diag = torch.zeros(1, 3, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.euler(F, 0.0, nsteps=1, diag=diag, ncells=3)
    mom = torch.zeros(3, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.moments(F, Q, mom, ncells=3)
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    p = oracle.Params(d=3, N=N, T=L, kernel=kernel, R=R, J=6)
    for i in range(3):
        Qo = oracle.collide(p, Fh[i])
        m = Fh[i] > 0
        lnF = np.log(Fh[i][m])
        P = float((Qo[m] * lnF).sum())
        bound = 2e-5 * np.abs(Qo).max() * np.abs(lnF).sum() + 1e-5 * np.abs(Qo[m] * lnF).sum()
        assert P < 0 and bound < abs(P)
        for got in (diag[0, i, 6].item(), mom[i, 6].item()):
            assert abs(got - P) <= bound, (i, got, P, bound)
            assert got < 0


def test_operations_capture_into_a_cuda_graph_without_allocation():
    """ef_collide, ef_euler_step and ef_rk3_step (after ef_plan_reserve) inside a stream capture:
    any allocation or device synchronisation would fail the capture.  The replayed graph gives the
    eager results bit for bit."""
    N, L, R = 16, 8.0, 32
    cells = [inputs.mixture_cell(3, N, L, 300 + i) for i in range(4)]
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32)
    plan.reserve(4)
    F0 = torch.tensor(np.stack(cells), dtype=torch.float32, device="cuda")
    Fa, Qa = F0.clone(), torch.empty_like(F0)
    Fb, Qb = F0.clone(), torch.empty_like(F0)

    def work(F, Q):
        plan.collide(F, Q, ncells=4)
        plan.euler(F, 0.01, nsteps=2, ncells=4)
        plan.rk3(F, 0.01, nsteps=1, ncells=4)

    work(Fa, Qa)                                  # eager
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            work(Fb, Qb)
    torch.cuda.current_stream().wait_stream(s)
    Fb.copy_(F0)
    g.replay()
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    assert torch.equal(Fa, Fb) and torch.equal(Qa, Qb)
    # a batched plan as well (two size classes)
    bplan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32, batched_N=[8, 12, 8])
    bplan.reserve()
    G0 = torch.tensor(inputs.pack([inputs.mixture_cell(3, n, L, 9 + n) for n in (8, 12, 8)]), dtype=torch.float32,
                      device="cuda")
    Ga, Gb = G0.clone(), G0.clone()
    bplan.rk3(Ga, 0.01)
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g2, stream=s):
            bplan.rk3(Gb, 0.01)
    torch.cuda.current_stream().wait_stream(s)
    Gb.copy_(G0)
    g2.replay()
    torch.cuda.synchronize()
    assert torch.equal(Ga, Gb)


def test_rk3_without_reserve_is_refused_before_any_launch():
    plan = ef.Plan(3, 8, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64)
    F = torch.zeros(2, 8, 8, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(ef.EfError) as e:
        ef.ef_rk3_step(plan.handle, F, 0.01, 1, None, 2)
    assert "ef_plan_reserve" in str(e.value)
    ef.ef_plan_reserve(plan.handle, 2)
    ef.ef_rk3_step(plan.handle, F, 0.01, 1, None, 2)
    with pytest.raises(ef.EfError):
        ef.ef_rk3_step(plan.handle, F, 0.01, 1, None, 3)      # more cells than reserved
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK


def test_kernel_function_fig1_on_the_gpu():
    """Fig. 1 from the GPU: 2D, B~ = 1/pi, R_tr = 6, T = (3 sqrt 2 + 1) R_tr / 4, N = 32, R = 64,
    z = (T/2, T/2).  G^sigma(y, z) of the plan's low-rank kernel takes negative values without the
    filter and none with it (Sec. 3.2.1 / 3.2.2), and equals the oracle's G to FP64 round-off."""
    N, R, Rtr = 32, 64, 6.0
    T = (3.0 * np.sqrt(2.0) + 1.0) * Rtr / 4.0
    z = (N // 2 + N // 4) * N + (N // 2 + N // 4)
    for sigma in (0, 1):
        plan = ef.Plan(2, N, T, ef.EF_KERNEL_MAXWELL, R, ef.EF_PREC_F64, R_tr=Rtr, sigma_enabled=sigma)
        G = torch.zeros(N * N, dtype=torch.float64, device="cuda")
        ef.ef_kernel_G(plan.handle, z, G)
        torch.cuda.synchronize()
        g = G.cpu().numpy()
        ref = oracle.G_slice(oracle.Params(d=2, N=N, T=T, kernel=0, R=R, Rtr=Rtr, filter=bool(sigma)), z).ravel()
        assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
        if sigma:
            assert g.min() >= -1e-12 * g.max()
        else:
            assert g.min() < -1e-2 * g.max()
    # 3D hard spheres, N = 8: the filtered G is non-negative and matches the oracle
    plan = ef.Plan(3, 8, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64)
    G = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    ef.ef_kernel_G(plan.handle, 3 * 64 + 5 * 8 + 2, G)
    torch.cuda.synchronize()
    ref = oracle.G_slice(oracle.Params(d=3, N=8, T=8.0, kernel=1, R=32, J=6), 3 * 64 + 5 * 8 + 2).ravel()
    g = G.cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    assert g.min() >= -1e-12 * g.max()
