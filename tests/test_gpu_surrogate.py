"""GPU tests of the surrogate path: low-mode features against the oracle's DFT, the tensor-core
MLP (forward and gradients) against the FP64 oracle MLP with the same bf16 roundings, training
that lowers the loss, and the gate / audit / fallback logic of ef_surrogate_infer."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1704_07369_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1704_07369_gb300 as ef  # noqa: E402
from paper_1704_07369_gb300 import surrogate as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ef.build()
    ef.lib()


def _modes(K=6):
    out = []
    for k0 in range(-K, K + 1):
        for k1 in range(-K, K + 1):
            for k2 in range(0, K + 1):
                if k0 * k0 + k1 * k1 + k2 * k2 > K * K:
                    continue
                if not (k2 > 0 or (k2 == 0 and (k1 > 0 or (k1 == 0 and k0 >= 0)))):
                    continue
                out.append((k0, k1, k2))
    return out


@pytest.mark.parametrize("d,N,prec", [(3, 16, ef.EF_PREC_F64), (3, 16, ef.EF_PREC_F32), (3, 24, ef.EF_PREC_F32), (3, 32, ef.EF_PREC_F32),
                                       (3, 40, ef.EF_PREC_F64), (3, 48, ef.EF_PREC_F32), (3, 64, ef.EF_PREC_F32),
                                       (2, 32, ef.EF_PREC_F64), (2, 64, ef.EF_PREC_F32)])
def test_features_match_oracle_dft(d, N, prec):
    """Band modes |k| <= 6 of F and of ln F (index-origin convention: the paper's Fh_k times
    (-1)^{sum k}) against the oracle's DFT: the direct sum for small grids, NumPy's FFT with the
    paper's phase for the large ones."""
    L = 8.0
    ncell = 3
    cells = [inputs.mixture_cell(d, N, L, 70 + i) for i in range(ncell)]
    dt = torch.float64 if prec == ef.EF_PREC_F64 else torch.float32
    plan = ef.Plan(d, N, L, ef.EF_KERNEL_HARD_SPHERE if d == 3 else ef.EF_KERNEL_MAXWELL, 32 if d == 3 else 16, prec)
    F = torch.tensor(np.stack(cells), dtype=dt, device="cuda")
    feat = torch.zeros(ncell, ef.EF_FEATURE_STRIDE, device="cuda")
    featL = torch.zeros_like(feat)
    ef.ef_features(plan.handle, F, feat, ncell)
    ef.ef_features(plan.handle, F, featL, ncell, log_input=1)
    torch.cuda.synchronize()
    modes = _modes() if d == 3 else [(k0, k1) for k0 in range(-6, 7) for k1 in range(0, 7)
                                     if k0 * k0 + k1 * k1 <= 36 and (k1 > 0 or k0 >= 0)]
    assert len(modes) == (463 if d == 3 else 57)
    for i, c in enumerate(cells):
        c = F[i].double().cpu().numpy()          # the values the kernel read
        for field, got in ((c, feat[i]), (np.log(np.maximum(c, 1e-30)), featL[i])):
            Fh = oracle.dft(field) if N <= 24 or d == 2 else oracle.dft_fft(field)
            ref = np.array([Fh[tuple(k % N for k in m)] * (-1) ** sum(m) for m in modes])
            g = got.cpu().numpy()[:2 * len(modes)].reshape(-1, 2)
            g = g[:, 0] + 1j * g[:, 1]
            assert np.abs(g - ref).max() <= 2e-6 * np.abs(ref).max(), (i, np.abs(g - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("N", [16, 24, 32])
def test_features_many_cells_per_cta(N):
    """FP32 3D batches several times larger than the resident CTAs, so each CTA walks many cells
    and stages the next cell's first planes while finishing the current one: sampled cells
    (first, middle, last) against the oracle's DFT, of F and of ln F."""
    L, n = 8.0, 1500
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    F = torch.empty(n, N, N, N, device="cuda")
    inputs.bkw_family_torch(N, L, n, 4242, device="cuda", out=F)
    feat = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    featL = torch.zeros_like(feat)
    ef.ef_features(plan.handle, F, feat, n)
    ef.ef_features(plan.handle, F, featL, n, log_input=1)
    torch.cuda.synchronize()
    assert plan.status(sync=1, reset=1) == ef.EF_OK
    modes = _modes()
    for i in (0, 1, 457, n // 2, n - 2, n - 1):
        c = F[i].double().cpu().numpy()
        for field, got in ((c, feat[i]), (np.log(np.maximum(c, 1e-30)), featL[i])):
            Fh = oracle.dft_fft(field)
            ref = np.array([Fh[tuple(k % N for k in m)] * (-1) ** sum(m) for m in modes])
            g = got.cpu().numpy()[:2 * len(modes)].reshape(-1, 2)
            g = g[:, 0] + 1j * g[:, 1]
            assert np.abs(g - ref).max() <= 2e-6 * np.abs(ref).max(), (i, np.abs(g - ref).max() / np.abs(ref).max())


def test_mlp_forward_and_gradients_match_oracle():
    rng = np.random.default_rng(5)
    nin, nh, nl, nout, B = 100, 64, 3, 70, 128
    net = ef.MLP(nin, nh, nl, nout, B, seed=11)
    layers = omlp.unpack(net.params(), net.layout())
    X = rng.normal(size=(B, nin)).astype(np.float32)
    T = rng.normal(size=(B, nout)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, nout).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    wd = torch.tensor(w, device="cuda")
    Y = torch.zeros(B, net.noutp, device="cuda")
    net.forward(Xd, Y, B)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(net.nparams, device="cuda")
    net.grad(Xd, Td, B, loss, grad, wmask=wd)
    torch.cuda.synchronize()
    Xp = np.zeros((B, net.ninp))
    Xp[:, :nin] = X
    y_ref, _ = omlp.forward(layers, Xp, bf=True)
    y = Y.cpu().numpy()
    assert np.sqrt(((y - y_ref) ** 2).sum() / (y_ref ** 2).sum()) <= 1e-4
    l_ref, g_ref = omlp.loss_and_grads(layers, Xp, T.astype(np.float64), nout, wmask=w, bf=True)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    gh = grad.cpu().numpy()
    for (woff, o, i, boff), (dW, db) in zip(net.layout(), g_ref):
        gW = gh[woff:woff + o * i].reshape(o, i)
        gb = gh[boff:boff + o]
        assert np.sqrt(((gW - dW) ** 2).sum() / (dW ** 2).sum()) <= 2e-3
        assert np.sqrt(((gb - db) ** 2).sum() / (db ** 2).sum()) <= 2e-3


def test_mlp_rowweight_gradients_and_exact_fp64_bound():
    """Per-sample loss weights (rowweight, as the surrogate's training uses them) against the oracle
    MLP with the same weights and the library's bf16 roundings; and the GPU against EXACT FP64
    backpropagation (no roundings) within a bound derived from the bf16 format.

    The bound is componentwise, first order in the bf16 unit roundoff u = 2^-8: every stored value
    (weight, split input, gradient signal) carries a relative error of at most u, and each dW_l is
    reached through at most 3 nl such roundings, so |dW_gpu - dW_exact| <= 3 nl u (g^_l^T a^_l), where
    a^ and g^ are the forward and backward passes with every weight and value replaced by its
    absolute value.  ReLU masks do not enter the bound because the hidden biases are set large
    enough that no pre-activation comes within its own rounding bound of zero (asserted)."""
    rng = np.random.default_rng(12)
    nin, nh, nl, nout, B = 96, 128, 3, 80, 256
    net = ef.MLP(nin, nh, nl, nout, B, seed=21)
    prm = net.params()
    for li, (woff, o, i, boff) in enumerate(net.layout()):
        if li + 1 < nl:                               # hidden pre-activations kept away from zero
            prm[woff:woff + o * i] *= 0.1
            prm[boff:boff + nh] = 4.0
    net.set_params(prm)
    layers = omlp.unpack(net.params(), net.layout())
    X = rng.normal(size=(B, nin)).astype(np.float32)
    T = rng.normal(size=(B, nout)).astype(np.float32)
    rw = rng.uniform(0.2, 3.0, B).astype(np.float32)
    Xd, Td, rwd = (torch.tensor(a, device="cuda") for a in (X, T, rw))
    Y = torch.zeros(B, net.noutp, device="cuda")
    net.forward(Xd, Y, B)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(net.nparams, device="cuda")
    net.grad(Xd, Td, B, loss, grad, rowweight=rwd)
    torch.cuda.synchronize()
    assert net.status() == ef.EF_OK
    Xp = np.zeros((B, net.ninp))
    Xp[:, :nin] = X
    gh = grad.cpu().numpy()

    def rel(a, b):
        return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())

    # same roundings: accumulation order only
    l_bf, g_bf = omlp.loss_and_grads(layers, Xp, T.astype(np.float64), nout, bf=True, rowweight=rw)
    assert abs(loss.item() - l_bf) <= 1e-4 * l_bf
    for (woff, o, i, boff), (dW, db) in zip(net.layout(), g_bf):
        assert rel(gh[woff:woff + o * i].reshape(o, i), dW) <= 2e-3
        assert rel(gh[boff:boff + o], db) <= 2e-3
    # exact FP64 against the bf16-derived componentwise bound
    u = 2.0 ** -8
    c = 3 * nl * u
    y_ex, (acts, pres) = omlp.forward(layers, Xp, bf=False)
    l_ex, g_ex = omlp.loss_and_grads(layers, Xp, T.astype(np.float64), nout, bf=False, rowweight=rw)
    ahat = [np.abs(Xp)]
    for li, (W, b) in enumerate(layers):
        pre_hat = ahat[-1] @ np.abs(W).T + np.abs(b)
        if li + 1 < nl:
            assert (pres[li] > c * pre_hat).all()    # no ReLU mask can flip
            ahat.append(pre_hat)
    gout = np.zeros_like(y_ex)
    gout[:, :nout] = np.abs(2.0 * rw[:, None] * (y_ex[:, :nout] - T) / (B * nout))
    ghat = [None] * nl
    ghat[nl - 1] = gout
    for li in range(nl - 1, 0, -1):
        ghat[li - 1] = ghat[li] @ np.abs(layers[li][0])
    for li, ((woff, o, i, boff), (dW, db)) in enumerate(zip(net.layout(), g_ex)):
        bW = c * (ghat[li].T @ ahat[li])
        bb = c * ghat[li].sum(axis=0)
        assert (np.abs(gh[woff:woff + o * i].reshape(o, i) - dW) <= bW + 1e-12).all(), li
        assert (np.abs(gh[boff:boff + o] - db) <= bb + 1e-12).all(), li
    yh = Y.cpu().numpy()
    assert (np.abs(yh - y_ex) <= c * (ahat[-1] @ np.abs(layers[-1][0]).T + np.abs(layers[-1][1])) + 1e-12).all()


def test_mlp_tcgen05_shapes_match_oracle():
    """A batch of 152 x 128 rows: the forward products and the input-gradient products then run on
    the tcgen05 kernel (N tiles of 256 and 192); outputs, loss and gradients against the FP64
    oracle MLP with the same bf16 roundings."""
    rng = np.random.default_rng(8)
    nin, nh, nl, nout, B = 900, 512, 3, 926, 152 * 128
    net = ef.MLP(nin, nh, nl, nout, B, seed=4)
    layers = omlp.unpack(net.params(), net.layout())
    X = rng.normal(size=(B, nin)).astype(np.float32)
    T = rng.normal(size=(B, nout)).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    Y = torch.zeros(B, net.noutp, device="cuda")
    net.forward(Xd, Y, B)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(net.nparams, device="cuda")
    net.grad(Xd, Td, B, loss, grad)
    torch.cuda.synchronize()
    Xp = np.zeros((B, net.ninp))
    Xp[:, :nin] = X
    y_ref, _ = omlp.forward(layers, Xp, bf=True)
    y = Y.cpu().numpy()
    assert np.sqrt(((y - y_ref) ** 2).sum() / (y_ref ** 2).sum()) <= 1e-4
    l_ref, g_ref = omlp.loss_and_grads(layers, Xp, T.astype(np.float64), nout, bf=True)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    gh = grad.cpu().numpy()
    for (woff, o, i, boff), (dW, db) in zip(net.layout(), g_ref):
        gW = gh[woff:woff + o * i].reshape(o, i)
        assert np.sqrt(((gW - dW) ** 2).sum() / (dW ** 2).sum()) <= 2e-3


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(6)
    nin, nh, nout, B = 64, 128, 32, 256
    net = ef.MLP(nin, nh, 3, nout, B, seed=3)
    A = rng.normal(size=(nin, nout)) / 8
    X = rng.normal(size=(B, nin)).astype(np.float32)
    T = np.tanh(X @ A).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    loss = torch.zeros(1, device="cuda")
    losses = []
    for _ in range(300):
        net.train_step(Xd, Td, B, 2e-3, loss)
        losses.append(loss.item())
    assert losses[-1] < 0.05 * losses[0]


def test_surrogate_gain_over_plain():
    """What the trained network buys over the method without it: on a batch of BKW-family cells
    (3D, N = 32, L = 8, hard spheres) the surrogate path, gates included, is several times faster
    than the plain operator, and after a short training its band of Q is already within a percent
    of the plain band for the typical cell (a no-op prediction Qh = 0 is off by 100%)."""
    plan = S.make_plan(ef.EF_KERNEL_HARD_SPHERE)
    fF, fQ, fM = S.features_of_family(plan, 30720, seed=1000)
    tr = S.Trainer(plan, batch=512, max_infer_batch=4096)
    hist = tr.fit(fF, fQ, fM, epochs=40, lr0=1e-3, warmup=0.05)
    assert hist[-1] < 0.01 * hist[0]
    n = 4096
    F = inputs.bkw_family_torch(32, 8.0, n, seed=9_000_000)
    Q = torch.empty_like(F)
    ref = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    plan.collide(F, Q, ncells=n)
    ef.ef_features(plan.handle, Q, ref, n)
    q = torch.zeros_like(ref)
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_plain = timed(lambda: plan.collide(F, Q, ncells=n))
    t_sur = timed(lambda: tr.sur.infer(F, q, flags, n, 0.0, 0, 1e-3))
    e = S.band_rel_l2(q, ref)
    assert t_plain / t_sur >= 3.0, (t_plain, t_sur)
    assert float(e.median()) <= 1e-2, float(e.median())
    assert int(((flags & 1) != 0).sum()) <= n // 20


def test_surrogate_audit_and_fallback_paths():
    """audit 1.0: every cell gets the plain band bit for bit; a tolerance no prediction can meet
    makes the audited cells fail and the whole batch fall back."""
    N, L, n = 16, 8.0, 128
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    net = ef.MLP(926, 64, 3, 926, n, seed=1)
    sur = ef.Surrogate(plan, net, n)
    F = inputs.bkw_family_torch(N, L, n, seed=77)
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=n)
    ref = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    ef.ef_features(plan.handle, Q, ref, n)
    fF = torch.zeros_like(ref)
    ef.ef_features(plan.handle, F, fF, n)
    mom = torch.zeros(n, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    ef.ef_moments_entropy(plan.handle, F, None, mom, n)
    Xt, Yt = torch.zeros_like(ref), torch.zeros_like(ref)
    sur.fit_stats(fF, ref, mom, Xt, Yt, n)
    q = torch.zeros_like(ref)
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    sur.infer(F, q, flags, n, audit_fraction=1.0, seed=5, tol=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(q[:, :926], ref[:, :926])
    assert bool(((flags & 8) != 0).all())
    sur.infer(F, q, flags, n, audit_fraction=0.25, seed=9, tol=1e-12)
    torch.cuda.synchronize()
    f = flags.cpu().numpy()
    assert ((f & 2) != 0).sum() > 0 and ((f & 4) != 0).sum() > 0
    assert ((f & 8) != 0).all()
    assert torch.equal(q[:, :926], ref[:, :926])
    # policy: tolerate every audited miss -> only the audited cells take the plain band
    sur.set_policy(max_miss_fraction=1.0)
    sur.infer(F, q, flags, n, audit_fraction=0.25, seed=9, tol=1e-12)
    torch.cuda.synchronize()
    f = flags.cpu().numpy()
    audited = (f & 2) != 0
    assert audited.sum() > 0 and ((f[audited] & 12) == 12).all()
    assert ((f & 16) == 0).all()
    keep = (f & 9) == 0                       # neither gated nor audited: the prediction stays
    assert keep.sum() > 0
    assert not torch.equal(q[torch.tensor(keep, device="cuda")][:, :926], ref[torch.tensor(keep, device="cuda")][:, :926])
    # an input envelope no cell meets gates every cell onto the plain operator
    sur.set_policy(max_miss_fraction=0.0, xmax=1e-6)
    sur.infer(F, q, flags, n, audit_fraction=0.0, seed=1, tol=1e-3)
    torch.cuda.synchronize()
    f = flags.cpu().numpy()
    assert ((f & 9) == 9).all()
    assert torch.equal(q[:, :926], ref[:, :926])
    with pytest.raises(ef.EfError):
        sur.set_policy(max_miss_fraction=1.5)


def test_entropy_gate_switch():
    """With the entropy-production gate off the inference skips the band of ln F: cells the gate
    did not flag keep the same prediction bit for bit, and no cell is flagged for a positive band
    production (an untrained network on a wide input envelope trips that gate on some cells)."""
    N, L, n = 16, 8.0, 256
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    net = ef.MLP(926, 64, 3, 926, n, seed=4)
    sur = ef.Surrogate(plan, net, n)
    F = inputs.bkw_family_torch(N, L, n, seed=79)
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=n)
    ref = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    ef.ef_features(plan.handle, Q, ref, n)
    fF = torch.zeros_like(ref)
    ef.ef_features(plan.handle, F, fF, n)
    mom = torch.zeros(n, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    ef.ef_moments_entropy(plan.handle, F, None, mom, n)
    Xt, Yt = torch.zeros_like(ref), torch.zeros_like(ref)
    sur.fit_stats(fF, ref, mom, Xt, Yt, n)
    sur.set_policy(max_miss_fraction=0.0, xmax=1e30)
    q1, q0 = torch.zeros_like(ref), torch.zeros_like(ref)
    f1 = torch.zeros(n, dtype=torch.int32, device="cuda")
    f0 = torch.zeros_like(f1)
    sur.infer(F, q1, f1, n, audit_fraction=0.0, seed=1, tol=1e-3)
    sur.set_entropy_gate(False)
    sur.infer(F, q0, f0, n, audit_fraction=0.0, seed=1, tol=1e-3)
    sur.set_entropy_gate(True)
    torch.cuda.synchronize()
    g1, g0 = f1.cpu().numpy(), f0.cpu().numpy()
    assert (g1 & 1).sum() > 0, "the untrained network should trip the entropy gate somewhere"
    assert (g0 == 0).all()
    keep = torch.tensor(g1 == 0, device="cuda")
    assert torch.equal(q0[keep], q1[keep])


@pytest.mark.parametrize("N", [16, 24, 32, 40, 48, 64])
def test_features_inverse_projects_on_the_band(N):
    """ef_features_inverse returns a band-limited field exactly (features -> grid -> features is the
    identity on the band) and maps a general cell to its truncation to |k| <= 6, against the
    oracle's DFT with the modes outside the band zeroed; every grid size of the band pass (its
    planes per chunk and row swizzle depend on N)."""
    L, n = 8.0, 3
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    cells = [inputs.mixture_cell(3, N, L, 90 + i) for i in range(n)]
    F = torch.tensor(np.stack(cells), dtype=torch.float32, device="cuda")
    feat = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    ef.ef_features(plan.handle, F, feat, n)
    P = torch.empty_like(F)
    ef.ef_features_inverse(plan.handle, feat, P, n)
    feat2 = torch.zeros_like(feat)
    ef.ef_features(plan.handle, P, feat2, n)
    torch.cuda.synchronize()
    a, b = feat2[:, :926].cpu().numpy(), feat[:, :926].cpu().numpy()
    assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max()
    k = np.fft.fftfreq(N, 1.0 / N)
    K0, K1, K2 = np.meshgrid(k, k, k, indexing="ij")
    band = K0 ** 2 + K1 ** 2 + K2 ** 2 <= 36
    for i in range(n):
        c = F[i].double().cpu().numpy()
        ref = np.real(np.fft.ifftn(np.fft.fftn(c) * band))   # index-origin DFT, truncated, inverted
        got = P[i].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_checker_gate_and_q_on_the_grid():
    """The checker gate: with the surrogate's own network as checker every score is at FP32
    round-off (the two forward passes need not agree bit for bit) and no cell is flagged at a
    threshold above it; with a different network and a threshold below every score, every cell goes
    to the plain operator (flags 32 and 8) and Q on the grid is the plain operator's Q bit for bit;
    cells that keep the prediction get its band mapped to the grid."""
    N, L, n = 16, 8.0, 128
    plan = ef.Plan(3, N, L, ef.EF_KERNEL_HARD_SPHERE, 32, ef.EF_PREC_F32)
    net = ef.MLP(926, 64, 3, 926, n, seed=1)
    other = ef.MLP(926, 64, 3, 926, n, seed=2)
    sur = ef.Surrogate(plan, net, n)
    F = inputs.bkw_family_torch(N, L, n, seed=78)
    Q = torch.empty_like(F)
    plan.collide(F, Q, ncells=n)
    ref = torch.zeros(n, ef.EF_FEATURE_STRIDE, device="cuda")
    ef.ef_features(plan.handle, Q, ref, n)
    fF = torch.zeros_like(ref)
    ef.ef_features(plan.handle, F, fF, n)
    mom = torch.zeros(n, ef.EF_DIAG_STRIDE, dtype=torch.float64, device="cuda")
    ef.ef_moments_entropy(plan.handle, F, None, mom, n)
    Xt, Yt = torch.zeros_like(ref), torch.zeros_like(ref)
    sur.fit_stats(fF, ref, mom, Xt, Yt, n)
    sur.set_policy(max_miss_fraction=0.0, xmax=1e30)        # no input-envelope gate here
    q = torch.zeros_like(ref)
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    score = torch.full((n,), -1.0, device="cuda")
    G = torch.empty_like(F)
    sur.set_checker(net, 1e-4)
    sur.infer_ex(F, q, flags, n, score=score, Q=G, audit_fraction=0.0, seed=3)
    torch.cuda.synchronize()
    assert 0.0 <= float(score.min()) and float(score.max()) <= 1e-6
    f = flags.cpu().numpy()
    assert ((f & 32) == 0).all()
    keep = torch.tensor((f & 8) == 0, device="cuda")
    if bool(keep.any()):                                    # delivered cells: Q on the grid = the band's inverse
        P = torch.empty_like(F)
        ef.ef_features_inverse(plan.handle, q, P, n)
        torch.cuda.synchronize()
        d = (G[keep] - P[keep]).abs().max() / P[keep].abs().max()
        assert float(d) <= 1e-6
    sur.set_checker(other, 1e-12)
    sur.infer_ex(F, q, flags, n, score=score, Q=G, audit_fraction=0.0, seed=3)
    torch.cuda.synchronize()
    f = flags.cpu().numpy()
    assert ((f & 40) == 40).all()
    assert float(score.min()) > 0.0
    assert torch.equal(G, Q)
    assert torch.equal(q[:, :926], ref[:, :926])
    sur.set_checker(None, 1.0)
    with pytest.raises(ef.EfError):
        sur.set_checker(other, 0.0)
