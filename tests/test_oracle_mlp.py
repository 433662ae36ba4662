"""Pin of the FP64 oracle MLP: its backpropagation (bf16 emulation off) equals central finite
differences of its own forward pass, and its bf16 rounding matches the bfloat16 format."""
import numpy as np
import pytest

from oracle import mlp


def _layers(rng, dims):
    return [(rng.normal(size=(o, i)) / np.sqrt(i), rng.normal(size=o) * 0.1) for i, o in zip(dims[:-1], dims[1:])]


@pytest.mark.parametrize("use_rowweight", [False, True])
def test_backprop_matches_finite_differences(use_rowweight):
    rng = np.random.default_rng(3)
    layers = _layers(rng, [7, 6, 5, 4])
    X = rng.normal(size=(5, 7))
    T = rng.normal(size=(5, 4))
    w = rng.uniform(0.5, 2.0, 3)
    rw = rng.uniform(0.1, 3.0, 5) if use_rowweight else None
    loss, grads = mlp.loss_and_grads(layers, X, T, 3, wmask=w, bf=False, rowweight=rw)
    eps = 1e-6
    for li, (W, b) in enumerate(layers):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + eps
                lp, _ = mlp.loss_and_grads(layers, X, T, 3, wmask=w, bf=False, rowweight=rw)
                arr[idx] = old - eps
                lm, _ = mlp.loss_and_grads(layers, X, T, 3, wmask=w, bf=False, rowweight=rw)
                arr[idx] = old
                assert abs((lp - lm) / (2 * eps) - g[idx]) <= 1e-7 * max(1.0, abs(g[idx]))


def test_bf16_rounding():
    # exactly representable values stay; halfway cases round to even; relative error <= 2^-9
    assert mlp.bf16(np.array([1.0, -2.5, 0.15625]))[0] == 1.0
    one_plus_half_ulp = 1.0 + 2.0 ** -8            # halfway between 1 and 1 + 2^-7 -> even (1.0)
    assert mlp.bf16(np.array([one_plus_half_ulp]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    x = np.random.default_rng(0).normal(size=10000)
    assert np.max(np.abs(mlp.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_split_precision_pair():
    x = np.random.default_rng(1).normal(size=10000).astype(np.float32).astype(np.float64)
    y = mlp.split(x)
    assert np.max(np.abs(y - x) / np.abs(x)) <= 2.0 ** -16
    hi = mlp.bf16(x)
    assert np.all(mlp.bf16(y - hi) == y - hi)      # the low half is itself a bf16 value


def test_rowweight_loss_is_the_weighted_mean_of_per_sample_losses():
    """The per-sample weights scale each sample's squared error: the loss with weights r equals
    sum_b r_b loss_b / B, where loss_b is the loss of the batch made of sample b alone (times 1)."""
    rng = np.random.default_rng(5)
    layers = _layers(rng, [4, 6, 3])
    X = rng.normal(size=(6, 4))
    T = rng.normal(size=(6, 3))
    r = rng.uniform(0.0, 2.0, 6)
    loss, _ = mlp.loss_and_grads(layers, X, T, 3, bf=False, rowweight=r)
    singles = [mlp.loss_and_grads(layers, X[b:b + 1], T[b:b + 1], 3, bf=False)[0] for b in range(6)]
    assert abs(loss - float(np.dot(r, singles)) / 6) <= 1e-14 * max(1.0, loss)
    # zero weight on a sample removes its gradient contribution exactly
    r0 = r.copy()
    r0[2] = 0.0
    _, g_all = mlp.loss_and_grads(layers, X, T, 3, bf=False, rowweight=r0)
    keep = [b for b in range(6) if b != 2]
    _, g_sub = mlp.loss_and_grads(layers, X[keep], T[keep], 3, bf=False, rowweight=r0[keep] * 5 / 6)
    for (a, b_), (c, d) in zip(g_all, g_sub):
        assert np.allclose(a, c, rtol=1e-12, atol=1e-15) and np.allclose(b_, d, rtol=1e-12, atol=1e-15)
