"""Pins of the oracle's surrogate network: gradients against central finite
differences, BF16 rounding against torch's conversion, Adam against
torch.optim.Adam, GELU against its closed-form derivative."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp


def _params(M=16, seed=3):
    r = W.rng(tag=300 + seed)
    return mlp.init_params(M, lambda n: r.uniform(size=n))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = W.rng(tag=301).standard_normal(10000) * np.exp(W.rng(tag=302).uniform(-20, 20, 10000))
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_gelu_derivative_is_the_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_backward_matches_central_differences():
    """Unrounded FP64 network: every layer's dW, db on sampled entries."""
    M, B = 16, 8
    params = _params(M)
    X = W.rng(tag=303).standard_normal((B, M))
    t = W.rng(tag=304).standard_normal(B)
    L0, grads = mlp.mse_loss_and_grad(params, X, t, rounding=False)
    r = W.rng(tag=305)
    h = 1e-6
    for l in range(mlp.LAYERS):
        Wl, bl = params[l]
        for _ in range(12):
            i, j = r.integers(Wl.shape[0]), r.integers(Wl.shape[1])
            Wp = Wl.copy(); Wp[i, j] += h
            Wm = Wl.copy(); Wm[i, j] -= h
            pp = list(params); pp[l] = (Wp, bl)
            pm = list(params); pm[l] = (Wm, bl)
            fd = (mlp.mse_loss_and_grad(pp, X, t, False)[0] - mlp.mse_loss_and_grad(pm, X, t, False)[0]) / (2 * h)
            assert abs(grads[l][0][i, j] - fd) < 1e-6 * max(1.0, abs(fd)), (l, i, j)
        i = r.integers(bl.shape[0])
        bp = bl.copy(); bp[i] += h
        bm = bl.copy(); bm[i] -= h
        pp = list(params); pp[l] = (Wl, bp)
        pm = list(params); pm[l] = (Wl, bm)
        fd = (mlp.mse_loss_and_grad(pp, X, t, False)[0] - mlp.mse_loss_and_grad(pm, X, t, False)[0]) / (2 * h)
        assert abs(grads[l][1][i] - fd) < 1e-6 * max(1.0, abs(fd))


def test_rounded_network_stays_close_to_the_exact_one():
    params = _params(16)
    X = W.rng(tag=306).standard_normal((64, 16))
    a, _ = mlp.forward(params, X, rounding=True)
    b, _ = mlp.forward(params, X, rounding=False)
    assert np.max(np.abs(a - b)) < 0.05 * np.max(np.abs(b)) + 1e-3


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    params = _params(8)
    X = W.rng(tag=307).standard_normal((32, 8))
    t = W.rng(tag=308).standard_normal(32)
    tp = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for Wb in params for p in Wb]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    adam = mlp.Adam(params, lr=1e-2)
    cur = params
    for _ in range(5):
        _, grads = mlp.mse_loss_and_grad(cur, X, t, rounding=False)
        for k, (gW, gb) in enumerate(grads):
            tp[2 * k].grad = torch.tensor(gW)
            tp[2 * k + 1].grad = torch.tensor(gb)
        opt.step()
        cur = adam.step(cur, grads)
    for k, (Wk, bk) in enumerate(cur):
        np.testing.assert_allclose(Wk, tp[2 * k].detach().numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(bk, tp[2 * k + 1].detach().numpy(), rtol=1e-12, atol=1e-14)


def test_training_reduces_the_loss_on_a_smooth_target():
    M = 8
    params = _params(M, seed=9)
    r = W.rng(tag=309)
    X = r.standard_normal((512, M))
    t = np.tanh(X @ np.linspace(-1, 1, M)) + 0.1 * X[:, 0] ** 2
    t = (t - t.mean()) / t.std()
    adam = mlp.Adam(params, lr=3e-3)
    L0 = mlp.mse_loss_and_grad(params, X, t)[0]
    for it in range(150):
        idx = r.integers(0, 512, 64)
        _, g = mlp.mse_loss_and_grad(params, X[idx], t[idx])
        params = adam.step(params, g)
    L1 = mlp.mse_loss_and_grad(params, X, t)[0]
    assert L1 < 0.2 * L0
