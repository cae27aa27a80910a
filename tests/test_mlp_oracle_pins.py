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


def test_one_layer_network_is_the_affine_map():
    """With no hidden layer the network is y = W x + b, written out here as
    explicit sums over a tiny input (brute force, no matrix routine)."""
    rng = np.random.default_rng(5)
    W, b = rng.standard_normal((3, 4)), rng.standard_normal(3)
    X = rng.standard_normal((2, 4))
    Y, _ = mo.forward([(W, b)], X)
    for i in range(2):
        for o in range(3):
            want = b[o]
            for k in range(4):
                want += X[i, k] * W[o, k]
            assert abs(Y[i, o] - want) < 1e-14


def test_activation_sits_on_hidden_layers_only():
    """Identity weights, zero hidden bias, output bias c: y = GELU(x) + c,
    GELU on the hidden layer and none on the output (a network with the
    activation on its output too would give GELU(GELU(x)) + c or GELU(x + c))."""
    rng = np.random.default_rng(6)
    d = 5
    c = rng.standard_normal(d)
    X = rng.standard_normal((4, d))
    Y, cache = mo.forward([(np.eye(d), np.zeros(d)), (np.eye(d), c)], X)
    want = 0.5 * X * (1 + np.tanh(np.sqrt(2 / np.pi) * (X + 0.044715 * X ** 3))) + c
    assert np.max(np.abs(Y - want)) < 1e-14
    # the cache holds each layer's input and pre-activation
    assert np.array_equal(cache[0][0], X) and np.max(np.abs(cache[1][1] - want)) < 1e-14


def test_loss_ignores_untrained_outputs():
    """The loss is the mean over the first n_out outputs only: the last
    layer's rows beyond n_out change neither the loss nor any gradient but
    their own, which is zero; with Y = T on the trained outputs the loss and
    every gradient vanish."""
    params, rng = _tiny(3)
    X = rng.standard_normal((6, 6))
    T = rng.standard_normal((6, 4))
    loss, grads = mo.loss_and_grads(params, X, T, 4)
    W4, b4 = params[-1]
    W4[4] += 1.7
    b4[4] -= 0.3
    loss2, grads2 = mo.loss_and_grads(params, X, T, 4)
    assert loss2 == loss
    assert np.all(grads2[-1][0][4] == 0) and grads2[-1][1][4] == 0
    for (gw, gb), (gw2, gb2) in zip(grads, grads2):
        assert np.array_equal(gw[:4] if gw.shape[0] == 5 else gw, gw2[:4] if gw2.shape[0] == 5 else gw2)
        assert np.array_equal(gb[:4] if gb.shape[0] == 5 else gb, gb2[:4] if gb2.shape[0] == 5 else gb2)
    Y, _ = mo.forward(params, X)
    loss0, grads0 = mo.loss_and_grads(params, X, Y[:, :4].copy(), 4)
    assert loss0 == 0.0
    assert all(np.all(gw == 0) and np.all(gb == 0) for gw, gb in grads0)
