"""GPU SSP-RK3 (ef_rk3_step) against the oracle's SSP-RK3, and the paper's Tables 1 and 2
reproduced from the GPU FP64 path: 2D BKW (Example 1), Maxwell molecules, truncation radius 6,
T = (3 sqrt 2 + 1) 6 / 4, one SSP-RK3 step of dt = 0.01 from t = 0, relative errors against the
closed form at t = 0.01; plus the positivity error of Sec. 4.2 on the GPU (zero for EFM)."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
T_PAPER = (3.0 * np.sqrt(2.0) + 1.0) * 6.0 / 4.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _table(name):
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


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_bkw_step(N, M):
    plan = ef.Plan(2, N, T_PAPER, ef.EF_KERNEL_MAXWELL, 2 * M, ef.EF_PREC_F64, R_tr=6.0)
    F = torch.tensor(inputs.bkw(2, N, T_PAPER, 0.0)[None], dtype=torch.float64, device="cuda")
    plan.rk3(F, 0.01, ncells=1)
    mom = torch.zeros(1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.moments(F, None, mom, ncells=1)
    torch.cuda.synchronize()
    assert plan.status(sync=1, reset=1) == ef.EF_OK
    V = oracle.grid(2, N, T_PAPER)
    return oracle.rel_errors(F[0].cpu().numpy(), oracle.bkw2d(0.01, V)), mom[0, 8].item()


@pytest.mark.parametrize("N", [16, 32, 64])
def test_table2_from_gpu(N):
    """Table 2 (l1 error for M = 2, 3, 32 angular samples) to the printed 5 significant figures."""
    tab = _table("table2_fast_l1.txt")
    for M, printed in zip((2, 3, 32), tab[N]):
        (l1, _, _), eps = _gpu_bkw_step(N, M)
        assert _within_print(l1, printed, 5), (N, M, l1, printed)
        assert eps == 0.0


@pytest.mark.parametrize("N", [16, 32, 64])
def test_table1_from_gpu(N):
    """Table 1 (l1, l2, l_inf for M = 32) to the printed 3 significant figures."""
    tab = _table("table1_bkw2d.txt")
    errs, _ = _gpu_bkw_step(N, 32)
    for e, printed in zip(errs, tab[N]):
        assert _within_print(e, printed, 3), (N, e, printed)


def test_rk3_matches_oracle_2d_and_3d():
    # 2D bi-Gaussian, Maxwell molecules, three steps
    N, L = 16, 8.0
    F0 = inputs.bigauss2d(N, L)
    plan = ef.Plan(2, N, L, ef.EF_KERNEL_MAXWELL, 16, ef.EF_PREC_F64)
    F = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
    diag = torch.zeros(3, 1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.rk3(F, 0.01, nsteps=3, diag=diag, ncells=1)
    torch.cuda.synchronize()
    p = oracle.Params(d=2, N=N, T=L, kernel=oracle.KERNEL_MAXWELL, R=16)
    ref = oracle.ssp_rk3(p, F0, 0.01, steps=3)
    assert _rel_l2(F[0].cpu().numpy(), ref) <= 1e-12
    # diagnostics of each step's first stage: the state before the step
    m0 = oracle.moments(F0, L, oracle.collide(p, F0))
    dg = diag.cpu().numpy()
    assert abs(dg[0, 0, 0] - m0[0]) <= 1e-12 * abs(m0[0])
    assert abs(dg[0, 0, 5] - m0[4]) <= 1e-12 * max(1.0, abs(m0[4]))
    assert np.abs(dg[:, 0, 0] - dg[0, 0, 0]).max() <= 1e-13        # mass conserved step to step
    assert (dg[:, 0, 6] <= 0).all()                                 # H-theorem at every step
    # 3D hard spheres, two ragged cells through a batched plan, FP64
    Ns = [8, 12]
    cells = [inputs.mixture_cell(3, n, L, 90 + i) for i, n in enumerate(Ns)]
    bplan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F64, batched_N=Ns)
    Fb = torch.tensor(inputs.pack(cells), dtype=torch.float64, device="cuda")
    bplan.rk3(Fb, 0.02, nsteps=1)
    torch.cuda.synchronize()
    got = Fb.cpu().numpy()
    off = 0
    for n, c in zip(Ns, cells):
        pc = oracle.Params(d=3, N=n, T=L, kernel=oracle.KERNEL_HARD_SPHERE, R=32)
        ref = oracle.ssp_rk3(pc, c, 0.02)
        assert _rel_l2(got[off:off + n ** 3].reshape(c.shape), ref) <= 1e-12, n
        off += n ** 3


def test_rk3_fp32_tracks_fp64():
    N, L = 24, 8.0
    c = inputs.mixture_cell(3, N, L, 7)
    out = {}
    for prec, dt in ((ef.EF_PREC_F64, torch.float64), (ef.EF_PREC_F32, torch.float32)):
        plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, prec)
        F = torch.tensor(c[None], dtype=dt, device="cuda")
        plan.rk3(F, 0.01, nsteps=5, ncells=1)
        torch.cuda.synchronize()
        out[prec] = F[0].double().cpu().numpy()
    assert np.abs(out[ef.EF_PREC_F32] - out[ef.EF_PREC_F64]).max() <= 1e-5 * np.abs(out[ef.EF_PREC_F64]).max()


def test_positivity_error_efm_zero_fcm_positive():
    """The contrast of Fig. 2 (Example 1): on the 2D BKW problem EFM keeps the positivity error of
    Sec. 4.2 at exactly zero, while the same collocation method without the filter (FCM, sigma = 1)
    produces negative values; the unfiltered GPU path matches the oracle's."""
    N, M, dt, steps = 32, 32, 0.05, 10
    F0 = inputs.bkw(2, N, T_PAPER, 0.0)
    eps = {}
    for filt in (1, 0):
        plan = ef.Plan(2, N, T_PAPER, ef.EF_KERNEL_MAXWELL, 2 * M, ef.EF_PREC_F64, R_tr=6.0, sigma_enabled=filt)
        F = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
        plan.rk3(F, dt, nsteps=steps, ncells=1)
        mom = torch.zeros(1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
        plan.moments(F, None, mom, ncells=1)
        torch.cuda.synchronize()
        eps[filt] = mom[0, 8].item()
        if not filt:
            p = oracle.Params(d=2, N=N, T=T_PAPER, kernel=oracle.KERNEL_MAXWELL, R=2 * M, Rtr=6.0, filter=False)
            ref = oracle.ssp_rk3(p, F0, dt, steps=steps)
            assert _rel_l2(F[0].cpu().numpy(), ref) <= 1e-12
            assert abs(eps[0] - oracle.positivity_error(ref)) <= 1e-12
    assert eps[1] == 0.0
    assert eps[0] > 1e-6
