"""The MLP oracle against facts outside itself (no GPU)."""

import numpy as np
import pytest
import torch

from oracle import mlp as M

SIZES = [7, 6, 5, 4]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = M.init_params(SIZES, rng)
    X = rng.normal(size=(9, SIZES[0]))
    Y = rng.normal(size=(9, SIZES[-1]))
    loss, grads = M.loss_and_grads(params, X, Y)
    flat = M.flatten(params)
    g_flat = M.flatten(grads)
    h = 1e-6
    num = np.empty_like(flat)
    for i in range(flat.size):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = M.loss_and_grads(M.unflatten(fp, SIZES), X, Y)
        lm, _ = M.loss_and_grads(M.unflatten(fm, SIZES), X, Y)
        num[i] = (lp - lm) / (2 * h)
    rel = np.linalg.norm(num - g_flat) / np.linalg.norm(num)
    assert rel <= 1e-6, rel
    assert abs(loss - np.mean((M.forward(params, X)[0] - Y) ** 2)) == 0.0


def test_zero_weights_give_bias():
    rng = np.random.default_rng(1)
    params = [(np.zeros_like(W), b) for W, b in M.init_params(SIZES, rng)]
    X = rng.normal(size=(3, SIZES[0]))
    out, _ = M.forward(params, X)
    assert np.array_equal(out, np.broadcast_to(params[-1][1], out.shape))


def test_gelu_values():
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.8411919906082768) < 1e-15
    assert abs(M.gelu(np.array(-1.0)) + 0.15880800939172324) < 1e-15
    # the tanh form stays within 1e-3 of the exact erf form
    from scipy.special import erf

    z = np.linspace(-6, 6, 2001)
    exact = 0.5 * z * (1 + erf(z / np.sqrt(2)))
    assert np.abs(M.gelu(z) - exact).max() < 1e-3
    # derivative against central differences
    h = 1e-6
    assert np.abs(M.gelu_grad(z) - (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)).max() < 1e-8


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    params = M.init_params(SIZES, rng)
    grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in params]
    new, state = M.adam_step(params, grads, M.zero_state(params), lr=1e-3)
    for (W, b), (gW, gb), (W1, b1) in zip(params, grads, new):
        # t = 1: m^ = g, v^ = g^2, step = lr * g / (|g| + eps)
        assert np.allclose(W1, W - 1e-3 * gW / (np.abs(gW) + 1e-8), rtol=0, atol=1e-15)
        assert np.allclose(b1, b - 1e-3 * gb / (np.abs(gb) + 1e-8), rtol=0, atol=1e-15)
    assert state[0] == 1


@pytest.mark.parametrize("seed", [3, 4])
def test_bf16_rounding_matches_torch(seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -3.0 - 2 ** -7, 0.0, -0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.to_bf16(x), ref)
    assert M.to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0  # tie to even
