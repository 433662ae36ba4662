"""ef_collide_noalloc: the allocation-free variant of ef_collide, for callers that cannot call
cudaMalloc when they evaluate the operator (its scratch lives in a static device array).

Collected last on purpose: a failure here leaves every other test already run.  Works alone in a
fresh process and after the other tests.  Two calls in a row with different inputs check that the
shared scratch (queue counter, accumulators) carries nothing from one call into the next; both
calls are compared with ef_collide and with the FP64 oracle.  The cases cover 2D (one row per
plane) and 3D plans, FP64 and both FP32 occupancy variants, shapes whose accumulators ef_collide
keeps in shared memory and in global memory.
"""
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


@pytest.mark.parametrize("d,prec,N", [(3, ef.EF_PREC_F64, 16), (3, ef.EF_PREC_F32, 24), (3, ef.EF_PREC_F32, 32),
                                      (3, ef.EF_PREC_F32, 48), (2, ef.EF_PREC_F64, 16)])
def test_noalloc_matches_collide_and_oracle_on_two_calls(d, prec, N):
    L = 8.0
    dt = torch.float64 if prec == ef.EF_PREC_F64 else torch.float32
    if d == 3:
        plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, prec)
        p = oracle.Params(d=3, N=N, T=L, kernel=oracle.KERNEL_HARD_SPHERE, R=32, J=6)
    else:
        plan = ef.Plan(2, N, L, ef.EF_KERNEL_MAXWELL, 16, prec)
        p = oracle.Params(d=2, N=N, T=L, kernel=oracle.KERNEL_MAXWELL, R=16)
    shape = plan.class_info()[0]
    assert shape["N"] == N and shape["cluster"] >= 1 and shape["sg_global"] in (0, 1)
    for call in range(2):
        if d == 3:
            cells = [inputs.mixture_cell(3, N, L, 900 + 10 * call + i) for i in range(5)]
        else:
            cells = [inputs.bigauss2d(N, L, shift=1.0 + 0.2 * i + 0.1 * call) for i in range(5)]
        F = torch.tensor(np.stack(cells), dtype=dt, device="cuda")
        Q_ref = torch.empty_like(F)
        Q_na = torch.full_like(F, float("nan"))
        plan.collide(F, Q_ref, ncells=5)
        ef.ef_collide_noalloc(plan.handle, F, Q_na, 5)
        torch.cuda.synchronize()
        assert plan.status() == ef.EF_OK
        a = Q_na.double().cpu().numpy()
        b = Q_ref.double().cpu().numpy()
        Fh = F.double().cpu().numpy()
        # the oracle on the first and last cell (the values the kernels read)
        refs = [(0, oracle.collide(p, Fh[0])), (4, oracle.collide(p, Fh[4]))] if N <= 24 or d == 2 else []
        if prec == ef.EF_PREC_F64:
            err = np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())
            assert err <= 1e-12, (call, err)
            for i, r in refs:
                assert np.sqrt(((a[i] - r) ** 2).sum() / (r ** 2).sum()) <= 1e-12, (call, i)
        else:
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err <= 2e-5, (call, err)
            for i, r in refs:
                assert np.abs(a[i] - r).max() <= 2e-5 * np.abs(r).max(), (call, i)
        if not refs:                              # larger 3D cells: sampled points against the oracle
            idx = np.unique(np.concatenate([np.argsort(np.abs(a[0]).ravel())[-8:],
                                            np.random.default_rng(call).integers(0, a[0].size, 120)]))
            r = oracle.collide_points_fft(p, Fh[0], idx)
            assert np.abs(a[0].ravel()[idx] - r).max() <= 2e-5 * np.abs(r).max(), call


def test_noalloc_rejects_batched_plans_and_bad_args():
    plan = ef.Plan(3, None, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, batched_N=[8, 12])
    F = torch.zeros(8 ** 3 + 12 ** 3, device="cuda")
    Q = torch.zeros_like(F)
    with pytest.raises(ef.EfError):
        ef.ef_collide_noalloc(plan.handle, F, Q, 2)
    uplan = ef.Plan(3, 8, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    with pytest.raises(ef.EfError):
        ef.ef_collide_noalloc(uplan.handle, F, F, 1)
