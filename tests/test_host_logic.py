"""Host-side orchestration of the binding, on CPU with the library's entry points replaced by the
oracle: the Lie splitting of Plan.inhomogeneous (buffer alternation, the copy back after an odd
number of steps, per-step diagnostics slices)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402


class _OraclePlan(ef.Plan):
    """A Plan whose transport and collision steps are the oracle's, on CPU tensors."""

    def __init__(self, p, dx_expected):
        self.p, self.d, self.N, self.ncells = p, p.d, p.N, None
        self.dx_expected = dx_expected
        self.calls = []

    def transport(self, F_in, F_out, dx, dt, ncells=None, stream=None):
        assert dx == self.dx_expected and F_in.data_ptr() != F_out.data_ptr()
        self.calls.append(("transport", F_in.data_ptr(), F_out.data_ptr()))
        F_out.copy_(torch.from_numpy(oracle.transport_upwind(F_in.numpy(), self.p.T, dx, dt)))

    def euler(self, F, dt, nsteps=1, diag=None, ncells=None, stream=None):
        self.calls.append(("euler", F.data_ptr(), None if diag is None else tuple(diag.shape)))
        F.copy_(torch.from_numpy(np.stack([oracle.euler(self.p, c, dt) for c in F.numpy()])))

    def rk3(self, F, dt, nsteps=1, diag=None, ncells=None, stream=None):
        self.calls.append(("rk3", F.data_ptr(), None if diag is None else tuple(diag.shape)))
        F.copy_(torch.from_numpy(np.stack([oracle.ssp_rk3(self.p, c, dt) for c in F.numpy()])))

    def close(self):
        pass


@pytest.mark.parametrize("nsteps,rk3", [(1, False), (2, False), (3, True)])
def test_inhomogeneous_alternates_buffers_and_ends_in_F(nsteps, rk3):
    p = oracle.Params(d=2, N=8, T=4.0, kernel=oracle.KERNEL_MAXWELL, R=16)
    cells = np.random.default_rng(3).uniform(0.1, 1.0, size=(5, 8, 8))
    F = torch.tensor(cells)
    S = torch.full_like(F, float("nan"))
    diag = torch.zeros(nsteps, 5, 10, dtype=torch.float64)
    plan = _OraclePlan(p, 0.5)
    plan.inhomogeneous(F, S, 0.5, 0.02, nsteps=nsteps, rk3=rk3, diag=diag)
    ref = oracle.inhomogeneous_lie(p, cells, 0.5, 0.02, steps=nsteps, rk3=rk3)
    assert np.array_equal(F.numpy(), ref)
    bufs = [F.data_ptr(), S.data_ptr()]
    for k in range(nsteps):
        tr, col = plan.calls[2 * k], plan.calls[2 * k + 1]
        assert tr == ("transport", bufs[k % 2], bufs[(k + 1) % 2])
        assert col == ("rk3" if rk3 else "euler", bufs[(k + 1) % 2], (5, 10))
