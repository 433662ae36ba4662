"""GPU free transport between cells (ef_transport_step) and its Lie splitting with the collision
step, against the oracle's upwind transport: the spatially inhomogeneous setting that Sec. 5 leaves
to future work, with the cells of a uniform batch as the points of a periodic 1D spatial grid."""
import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _dtype(prec):
    return torch.float64 if prec == ef.EF_PREC_F64 else torch.float32


@pytest.mark.parametrize("d,N,M,prec", [(3, 16, 37, ef.EF_PREC_F64), (3, 16, 37, ef.EF_PREC_F32),
                                        (2, 32, 5, ef.EF_PREC_F32), (3, 8, 1, ef.EF_PREC_F64),
                                        (2, 12, 300, ef.EF_PREC_F64)])
def test_transport_matches_oracle(d, N, M, prec):
    """Every point of every cell, the periodic wrap at both ends included (and a single cell, its
    own neighbour), at Courant number 0.9."""
    L, dx = 8.0, 0.25
    h = 2.0 * L / N
    dt = 0.9 * dx / ((N // 2) * h)
    cells = np.stack([inputs.mixture_cell(d, N, L, 300 + i) for i in range(M)])
    plan = ef.Plan(d, N, L, ef.EF_KERNEL_HARD_SPHERE if d == 3 else ef.EF_KERNEL_MAXWELL, 32 if d == 3 else 16, prec)
    F = torch.tensor(cells, dtype=_dtype(prec), device="cuda")
    G = torch.full_like(F, float("nan"))
    plan.transport(F, G, dx, dt)
    torch.cuda.synchronize()
    assert plan.status(sync=1, reset=1) == ef.EF_OK
    ref = oracle.transport_upwind(F.double().cpu().numpy(), L, dx, dt)
    got = G.double().cpu().numpy()
    tol = 1e-15 if prec == ef.EF_PREC_F64 else 5e-7
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert got.min() >= 0.0
    assert np.allclose(got.sum(axis=0), ref.sum(axis=0), rtol=1e-12 if prec == ef.EF_PREC_F64 else 1e-5, atol=0)


def test_lie_splitting_matches_oracle_and_conserves_mass():
    """Two Lie steps (transport, then one Euler collision step per cell) on six 2D cells, FP64,
    against the oracle; then twelve SSP-RK3 steps on the GPU keep the total mass and F >= 0."""
    d, N, L, M = 2, 16, 8.0, 6
    dx, dt = 0.5, 0.01
    cells = np.stack([inputs.mixture_cell(d, N, L, 500 + i) for i in range(M)])
    plan = ef.Plan(d, N, L, ef.EF_KERNEL_MAXWELL, 16, ef.EF_PREC_F64)
    F = torch.tensor(cells, dtype=torch.float64, device="cuda")
    S = torch.empty_like(F)
    plan.inhomogeneous(F, S, dx, dt, nsteps=2)
    torch.cuda.synchronize()
    assert plan.status(sync=1, reset=1) == ef.EF_OK
    p = oracle.Params(d=d, N=N, T=L, kernel=oracle.KERNEL_MAXWELL, R=16)
    ref = oracle.inhomogeneous_lie(p, cells, dx, dt, steps=2)
    got = F.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    m0 = F.sum().item()
    diag = torch.zeros(12, M, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.inhomogeneous(F, S, dx, dt, nsteps=12, rk3=True, diag=diag)
    torch.cuda.synchronize()
    assert abs(F.sum().item() - m0) <= 1e-12 * m0
    assert F.min().item() >= 0.0
    assert (diag[:, :, 6] <= 0).all()          # H-theorem in every cell at every step


def test_transport_argument_checks():
    plan = ef.Plan(3, 8, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    F = torch.ones(4, 8, 8, 8, device="cuda")
    with pytest.raises(ef.EfError):
        plan.transport(F, F, 0.1, 0.01)                       # in place: overlapping
    with pytest.raises(ef.EfError):
        plan.transport(F, torch.empty_like(F), 0.0, 0.01)     # dx <= 0
    bplan = ef.Plan(3, None, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, batched_N=[8, 8])
    with pytest.raises(ef.EfError):
        bplan.transport(F[:2], torch.empty_like(F[:2]), 0.1, 0.01, ncells=2)   # batched plan
