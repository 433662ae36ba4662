"""The Fourier Galerkin method on the GPU (ef_galerkin_*, Sec. 1.2 eq. FGM_Q by zero padding)
against the oracle's unaliased double sum, and the FGM half of the Fig. 2 contrast: on the 2D BKW
problem (Example 1) EFM keeps the positivity error at zero while FGM, started from the
interpolated grid values (the "I" curves of Fig. 2), does not."""
import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu

T_PAPER = (3.0 * np.sqrt(2.0) + 1.0) * 6.0 / 4.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _rel_l2(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


@pytest.mark.parametrize("d,N,prec,sigma", [(2, 16, ef.EF_PREC_F64, 0), (2, 12, ef.EF_PREC_F64, 1), (2, 32, ef.EF_PREC_F32, 0),
                                            (3, 8, ef.EF_PREC_F64, 0), (3, 16, ef.EF_PREC_F32, 0), (3, 12, ef.EF_PREC_F64, 1)])
def test_galerkin_against_oracle(d, N, prec, sigma):
    L = 8.0
    kern, R = (ef.EF_KERNEL_MAXWELL, 16) if d == 2 else (ef.EF_KERNEL_HARD_SPHERE, 32)
    cells = [inputs.mixture_cell(d, N, L, 60 + i) for i in range(3)]
    g = ef.Galerkin(d, N, L, kern, R, prec, max_cells=4, sigma_enabled=sigma)
    dt = torch.float64 if prec == ef.EF_PREC_F64 else torch.float32
    F = torch.tensor(np.stack(cells), dtype=dt, device="cuda")
    Q = torch.empty_like(F)
    g.collide(F, Q, ncells=3)
    torch.cuda.synchronize()
    assert g.status() == ef.EF_OK
    p = oracle.Params(d=d, N=N, T=L, kernel=kern, R=R, J=6, filter=bool(sigma))
    for i in range(3):
        ref = oracle.collide_galerkin(p, F[i].double().cpu().numpy())
        got = Q[i].double().cpu().numpy()
        if prec == ef.EF_PREC_F64:
            assert _rel_l2(got, ref) <= 1e-12
        else:
            assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
        assert abs(got.sum()) <= (1e-12 if prec == ef.EF_PREC_F64 else 1e-5) * np.abs(got).sum()   # mass


def test_fig2_fgm_positivity_error_against_efm():
    """Example 1, N = 16, M = 32 (R = 64), R_tr = 6, T = (3 sqrt 2 + 1) R_tr / 4: ten SSP-RK3 steps
    (dt = 0.05) from BKW at t = 0.  EFM's positivity error stays exactly zero; FGM's grows above
    zero, and the GPU's FGM trajectory matches the oracle's to FP64 round-off."""
    N, M, dt, steps = 16, 32, 0.05, 10
    F0 = inputs.bkw(2, N, T_PAPER, 0.0)
    plan = ef.Plan(2, N, T_PAPER, ef.EF_KERNEL_MAXWELL, 2 * M, ef.EF_PREC_F64, R_tr=6.0, sigma_enabled=1)
    F = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
    mom = torch.zeros(1, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    eps_efm = []
    for _ in range(steps):
        plan.rk3(F, dt, nsteps=1, ncells=1)
        plan.moments(F, None, mom, ncells=1)
        eps_efm.append(mom[0, 8].item())
    g = ef.Galerkin(2, N, T_PAPER, ef.EF_KERNEL_MAXWELL, 2 * M, ef.EF_PREC_F64, max_cells=1, R_tr=6.0, sigma_enabled=0)
    G = torch.tensor(F0[None], dtype=torch.float64, device="cuda")
    Qg = torch.empty_like(G)

    def Qof(X):
        g.collide(X, Qg, ncells=1)
        return Qg.clone()

    eps_fgm = []
    for _ in range(steps):                        # SSP-RK3 (Sec. 4.1) around the Galerkin operator
        G1 = G + dt * Qof(G)
        G2 = 0.75 * G + 0.25 * (G1 + dt * Qof(G1))
        G = G / 3.0 + 2.0 / 3.0 * (G2 + dt * Qof(G2))
        plan.moments(G, None, mom, ncells=1)
        eps_fgm.append(mom[0, 8].item())
    torch.cuda.synchronize()
    assert g.status() == ef.EF_OK and plan.status() == ef.EF_OK
    assert all(e == 0.0 for e in eps_efm)
    assert max(eps_fgm) > 1e-6
    p = oracle.Params(d=2, N=N, T=T_PAPER, kernel=oracle.KERNEL_MAXWELL, R=2 * M, Rtr=6.0, filter=False)
    ref = oracle.ssp_rk3_with(lambda X: oracle.collide_galerkin(p, X), F0, dt, steps=steps)
    assert _rel_l2(G[0].cpu().numpy(), ref) <= 1e-12
    assert abs(eps_fgm[-1] - oracle.positivity_error(ref)) <= 1e-12
