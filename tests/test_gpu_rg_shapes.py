"""The FP32 3D register-accumulator collide kernel (gain accumulator in registers, forward spectrum
in shared memory, Nyquist column skipped) on every launch shape the autotuner can pick: cluster
sizes 1 to 16, one or two real rows per thread, and the two-lanes-per-line variants, pinned through
EF_SHAPE.  Each shape is checked
against the FP64 oracle (whole cells at N = 16, sampled points above) on a ragged two-cell batch,
with the dynamic cell queue and the Euler diagnostics (mass against the oracle's).

The shapes are those the kernel's layout admits: C | N, an even split of the N^2 / 2 pencils,
threads = N^2 / (C RPT) (twice that for the team variants) within the instantiation's launch bound, shared memory within the 227 KB
limit."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402

pytestmark = pytest.mark.gpu

def rg_bound(N, v):
    """Launch bound of instantiation v (1: one row per thread, 2: two rows, 3: one row, <= 200
    threads, 4: the gain accumulator in shared memory)."""
    if v == 1:
        return 320 if N == 40 else 256 if N in (32, 64) else 288
    if v == 2:
        return {16: 128, 24: 288, 32: 256, 40: 200, 48: 192, 64: 128}[N]
    if v == 3:
        return 200 if N in (40, 48) else 0
    if v in (5, 6):          # two lanes per line (collide_kernel_tm), one or two rows per team
        return {24: 288, 32: 256, 40: 400, 48: 384}.get(N, 0)
    return 320 if N == 40 else 288 if N in (24, 48) else 256


def _npp(N):
    swz = (N // 4) % 4 == 0
    rs = N // 2 if swz else N // 2 + 2
    s = N * rs
    r = 8 if swz else (N // 2) % 16
    return s + ((r - s % 16) % 16 + 16) % 16


def rg_shapes(N):
    out = []
    for C in (1, 2, 3, 4, 5, 6, 8, 10, 12, 16):
        if N % C or (N * N // 2) % C or (N * N // (2 * C)) % 2:
            continue
        P = N // C
        npc = N * N // (2 * C)
        for v in (1, 2, 3, 4, 5, 6):
            smem = 2 * P * _npp(N) * 8 + N * npc * 8 + (P * N * N * 4 if v == 4 else 0) + 33 * 10 * 8 + 16 + 128
            if smem > 232448:
                continue
            team = 2 if v >= 5 else 1
            for per in ((1, 2) if v == 4 else ((2,) if v in (2, 6) else (1,))):
                t = team * N * P // per
                if (N * P) % per == 0 and 32 <= t <= rg_bound(N, v):
                    out.append((C, t, 2 + v))
    return out


CASES = [(N, s) for N in (16, 24, 32, 40, 48, 64) for s in rg_shapes(N)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


@pytest.mark.parametrize("N,shape", CASES, ids=["N%d-C%d-t%d-v%d" % ((n,) + s) for n, s in CASES])
def test_rg_shape_against_oracle(N, shape, monkeypatch):
    C, tpb, occ = shape
    L = 8.0 if N < 64 else 10.0
    R = 32 if N < 64 else 64
    monkeypatch.setenv("EF_SHAPE", "%d:%d:%d:%d" % (N, C, tpb, occ))
    cells = [inputs.mixture_cell(3, N, L, 4000 + N + C), inputs.mixture_cell(3, N, L, 5000 + N + C)]
    plan = ef.Plan(3, None, L, ef.EF_KERNEL_HARD_SPHERE, R, ef.EF_PREC_F32, batched_N=[N, N])
    info = plan.class_info()[0]
    assert (info["cluster"], info["threads"]) == (C, tpb)
    F = torch.tensor(inputs.pack(cells), dtype=torch.float32, device="cuda")
    Q = torch.empty_like(F)
    plan.collide(F, Q)
    Fe = F.clone()
    diag = torch.zeros(1, 2, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    plan.euler(Fe, 0.0, 1, diag)
    torch.cuda.synchronize()
    assert plan.status() == ef.EF_OK
    q = Q.double().cpu().numpy().reshape(2, N, N, N)
    Fh = F.double().cpu().numpy().reshape(2, N, N, N)
    p = oracle.Params(d=3, N=N, T=L, kernel=oracle.KERNEL_HARD_SPHERE, R=R, J=6)
    for i in range(2):
        if N == 16:
            ref = oracle.collide(p, Fh[i])
            assert np.abs(q[i] - ref).max() <= 2e-5 * np.abs(ref).max()
        else:
            idx = np.unique(np.concatenate([np.argsort(np.abs(q[i]).ravel())[-8:],
                                            np.random.default_rng(i + N).integers(0, N ** 3, 56)]))
            ref = oracle.collide_points_fft(p, Fh[i], idx)
            assert np.abs(q[i].ravel()[idx] - ref).max() <= 2e-5 * np.abs(ref).max()
        # diagnostics of the fused output pass: mass of F (FP64 sum of FP32 row partials)
        m = Fh[i].sum() * (2 * L / N) ** 3
        assert abs(diag[0, i, 0].item() - m) <= 1e-6 * m
