"""GPU tests of the streamed host-resident batch (ef_stream_euler_step): the chunked, overlapped
upload / step / download gives what ef_euler_step gives on a device copy of the same batch."""
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


@pytest.mark.parametrize("nchunks", [1, 3, 8])
def test_streamed_batch_matches_device_path(nchunks):
    L, dt, nsteps = 8.0, 0.01, 2
    Ns = inputs.ragged_sizes(40, choices=(12, 16, 24), seed=11)
    host = torch.tensor(inputs.pack([inputs.mixture_cell(3, int(n), L, 500 + i) for i, n in enumerate(Ns)]),
                        dtype=torch.float32).pin_memory()
    ref = host.clone().cuda()
    plan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, batched_N=Ns)
    dref = torch.zeros(nsteps, len(Ns), ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.euler(ref, dt, nsteps=nsteps, diag=dref)
    sp = ef.StreamPlan(3, Ns, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, nchunks=nchunks)
    info = sp.info()
    assert info["cells"] == len(Ns) and info["chunks"] == min(nchunks, len(Ns)) and info["values"] == host.numel()
    dh = torch.zeros(nsteps, len(Ns), ef.EF_DIAG_STRIDE, dtype=torch.float64).pin_memory()
    sp.euler(host, dt, nsteps=nsteps, diag_host=dh)
    torch.cuda.synchronize()
    assert sp.status(sync=1, reset=1) == ef.EF_OK
    r = ref.cpu().numpy()
    assert np.abs(host.numpy() - r).max() <= 1e-6 * np.abs(r).max()
    d1, d2 = dh.numpy(), dref.cpu().numpy()
    for k in (0, 1, 2, 3, 4, 5, 7):       # moments, entropy, production, min F
        assert np.allclose(d1[..., k], d2[..., k], rtol=1e-6, atol=1e-12), k
    sp.close()


def test_streamed_batch_from_pageable_memory():
    """Pageable host memory: correct, the copies just do not overlap."""
    L = 8.0
    Ns = [16, 24, 16, 24]
    host = torch.tensor(inputs.pack([inputs.mixture_cell(3, n, L, 7 + i) for i, n in enumerate(Ns)]), dtype=torch.float32)
    ref = host.clone().cuda()
    ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, batched_N=Ns).euler(ref, 0.01)
    sp = ef.StreamPlan(3, Ns, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32, nchunks=2)
    sp.euler(host, 0.01)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.abs(host.numpy() - r).max() <= 1e-6 * np.abs(r).max()
    sp.close()
