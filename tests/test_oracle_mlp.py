"""Pins of the warm-start network oracle: backpropagation against central
finite differences (FP64, roundings off), the BF16 rounding against the
bit-level definition, and Adam against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(5, 7, 4, seed=3)
    for p in params[1::2]:
        p[:] = rng.standard_normal(p.shape) * 0.1     # nonzero biases
    X = rng.standard_normal((6, 5))
    T = rng.standard_normal((6, 4))
    loss, grads = mlp.loss_and_grads(params, X, T, round_bf16=False)
    h = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, T, round_bf16=False)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, T, round_bf16=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx)


def test_bf16_rounding_definition():
    # exact bf16 values pass through; ties round to even; 8 significant bits
    assert mlp.bf16(np.array([1.0, -2.5, 0.0]))[1] == -2.5
    one_plus = 1.0 + 2.0 ** -8          # halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.array([one_plus]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)


def test_adam_first_step_is_signed_learning_rate():
    """With bias correction the first Adam step moves every parameter by
    -lr * sign(g) (up to eps), for any gradient scale."""
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([1e-3, -5.0, 2.0])]
    st = (0, [np.zeros(3)], [np.zeros(3)])
    mlp.adam_step(p, g, st, lr=0.1)
    np.testing.assert_allclose(p[0], [0.9, -1.9, 2.9], atol=1e-6)
