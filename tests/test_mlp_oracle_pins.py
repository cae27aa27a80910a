"""Pins of the CPU reference of the warm-start network: gradients against
central finite differences in float64, GELU against its definition, and
the bf16 rounding against known values."""
import numpy as np

from oracle import mlp_oracle as mo


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    dims = [(6, 10), (10, 10), (10, 8), (8, 5)]
    return [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o)) for i, o in dims], rng


def test_gradients_match_finite_differences():
    params, rng = _tiny(1)
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 4))          # 4 of the 5 outputs are trained
    loss, grads = mo.loss_and_grads(params, X, T, 4)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = mo.loss_and_grads(params, X, T, 4)
                arr[idx] = old - h
                lm, _ = mo.loss_and_grads(params, X, T, 4)
                arr[idx] = old
                num[idx] = (lp - lm) / (2 * h)
            assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_gelu_and_its_derivative():
    x = np.linspace(-4, 4, 101)
    want = 0.5 * x * (1 + np.tanh(np.sqrt(2 / np.pi) * (x + 0.044715 * x ** 3)))
    assert np.allclose(mo.gelu(x), want, atol=1e-15)
    h = 1e-6
    assert np.allclose(mo.gelu_grad(x), (mo.gelu(x + h) - mo.gelu(x - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    assert mo.bf16(1.0) == 1.0
    assert mo.bf16(1.0 + 2 ** -9) == 1.0                  # below half an ulp (2^-7)
    assert mo.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7   # above half an ulp
    assert mo.bf16(1.0 + 2 ** -8) == 1.0                  # tie -> even
    assert mo.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie -> even (upwards)
    assert mo.bf16(-3.0) == -3.0
