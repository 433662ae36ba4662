"""GPU classical form (ef_classical_collide: the remark after eq. EFMk, kernel modes of
eq. classical_hatB, 3D Maxwell molecules, FP64 direct pair sum) against the oracle's classical
form, and Table 3 (Example 4) reproduced from the GPU path at N = 16, 32 and 64."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
T_CLASSICAL = (3.0 + np.sqrt(2.0)) * 6.0 / 4.0     # T = (3 + sqrt 2) R / 4 with R = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _within_print(ours, printed, sig):
    unit = 10.0 ** (np.floor(np.log10(abs(printed))) - (sig - 1))
    return abs(ours - printed) <= unit * 1.0001


@pytest.mark.parametrize("N,filt", [(8, 1), (12, 1), (8, 0)])
def test_classical_matches_oracle(N, filt):
    """Two cells in one call (random mixtures), with and without the filter."""
    cells = np.stack([inputs.mixture_cell(3, N, T_CLASSICAL, 800 + i) for i in range(2)])
    c = ef.Classical(N, T_CLASSICAL, 6.0, sigma_enabled=filt)
    F = torch.tensor(cells, dtype=torch.float64, device="cuda")
    Q = torch.full_like(F, float("nan"))
    c.collide(F, Q)
    torch.cuda.synchronize()
    p = oracle.Params(d=3, N=N, T=T_CLASSICAL, kernel=oracle.KERNEL_MAXWELL, R=32, Rtr=6.0, filter=bool(filt))
    for i in range(2):
        ref = oracle.collide_classical(p, cells[i])
        got = Q[i].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (N, filt, i)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_table3_from_gpu(N):
    """One SSP-RK3 step of dt = 0.01 from the 3D BKW solution at t = 0 (the stages combined here,
    each evaluation on the GPU): N = 32 and 64 to all printed figures; N = 16 l2 and l_inf to the
    printed figures and l1 within 0.35% (the oracle's reading of the classical form gives 4.0675e-3
    against the printed 4.08e-3)."""
    rows = {}
    with open(os.path.join(GOLD, "table3_bkw3d.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                v = [float(x) for x in line.split()]
                rows[int(v[0])] = v[1:]
    V = oracle.grid(3, N, T_CLASSICAL)
    c = ef.Classical(N, T_CLASSICAL, 6.0)
    dt = 0.01
    F0 = torch.tensor(oracle.bkw3d(0.0, V), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(F0)

    def q(X):
        c.collide(X, Q, ncells=1)
        return Q.clone()

    F1 = F0 + dt * q(F0)
    F2 = 0.75 * F0 + 0.25 * (F1 + dt * q(F1))
    F3 = F0 / 3.0 + 2.0 / 3.0 * (F2 + dt * q(F2))
    torch.cuda.synchronize()
    errs = oracle.rel_errors(F3.cpu().numpy(), oracle.bkw3d(dt, V))
    if N >= 32:
        for e, printed in zip(errs, rows[N]):
            assert _within_print(e, printed, 3), (e, printed)
    else:
        assert _within_print(errs[1], rows[16][1], 3) and _within_print(errs[2], rows[16][2], 3), errs
        assert abs(errs[0] - rows[16][0]) <= 0.0035 * rows[16][0], errs[0]


def test_classical_conserves_mass_and_dissipates_entropy():
    N = 12
    V = oracle.grid(3, N, T_CLASSICAL)
    F = torch.tensor(oracle.bkw3d(0.0, V), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(F)
    ef.Classical(N, T_CLASSICAL, 6.0).collide(F, Q, ncells=1)
    torch.cuda.synchronize()
    f, qv = F.cpu().numpy(), Q.cpu().numpy()
    assert abs(qv.sum()) <= 1e-13 * np.abs(qv).sum()
    assert (qv[f > 0] * np.log(f[f > 0])).sum() < 0
