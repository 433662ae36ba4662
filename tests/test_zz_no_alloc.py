"""ef_collide_noalloc: the allocation-free variant of ef_collide, for callers that cannot call
cudaMalloc when they evaluate the operator (its scratch lives in a static device array).

Collected last on purpose: a failure here leaves every other test already run.  Works alone in a
fresh process and after the other tests.  Two calls in a row with different inputs check that the
shared scratch (queue counter, accumulators) carries nothing from one call into the next.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,N", [(ef.EF_PREC_F64, 16), (ef.EF_PREC_F32, 24), (ef.EF_PREC_F32, 48)])
def test_noalloc_matches_collide_on_two_calls(prec, N):
    L = 8.0
    dt = torch.float64 if prec == ef.EF_PREC_F64 else torch.float32
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, prec)
    for call in range(2):
        cells = [inputs.mixture_cell(3, N, L, 900 + 10 * call + i) for i in range(5)]
        F = torch.tensor(np.stack(cells), dtype=dt, device="cuda")
        Q_ref = torch.empty_like(F)
        Q_na = torch.full_like(F, float("nan"))
        plan.collide(F, Q_ref, ncells=5)
        ef.ef_collide_noalloc(plan.handle, F, Q_na, 5)
        torch.cuda.synchronize()
        assert plan.status() == ef.EF_OK
        a = Q_na.double().cpu().numpy()
        b = Q_ref.double().cpu().numpy()
        if prec == ef.EF_PREC_F64:
            err = np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())
            assert err <= 1e-12, (call, err)
        else:
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err <= 2e-5, (call, err)


def test_noalloc_rejects_batched_plans_and_bad_args():
    plan = ef.Plan(3, None, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, batched_N=[8, 12])
    F = torch.zeros(8 ** 3 + 12 ** 3, device="cuda")
    Q = torch.zeros_like(F)
    with pytest.raises(ef.EfError):
        ef.ef_collide_noalloc(plan.handle, F, Q, 2)
    uplan = ef.Plan(3, 8, 8.0, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    with pytest.raises(ef.EfError):
        ef.ef_collide_noalloc(uplan.handle, F, F, 1)
