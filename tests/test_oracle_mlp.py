"""Pins for the float64 selector-network oracle: finite differences and closed forms."""
import numpy as np
import pytest

from oracle import mlp


def rand_params(seed):
    rng = np.random.default_rng(seed)
    return mlp.he_uniform_init(rng.random(mlp.N_PARAMS)) + 0.05 * rng.standard_normal(mlp.N_PARAMS)


def test_param_count():
    assert mlp.N_PARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4 == 5252


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    w = rand_params(seed)
    X = rng.standard_normal((7, 12))
    T = rng.standard_normal((7, 4))
    _, g = mlp.loss_and_grad(w, X, T)
    idx = rng.choice(mlp.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num = (mlp.mse_loss(mlp.forward(wp, X)[0], T) - mlp.mse_loss(mlp.forward(wm, X)[0], T)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_zero_hidden_weights_give_bias_output():
    w = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(w)
    p["b3"][...] = [1.0, -2.0, 3.0, 0.5]
    p["b1"][...] = 1.0  # h1 = 1, but W2 = 0 so h2 = relu(b2) = 0
    Y, _ = mlp.forward(w, np.random.default_rng(0).standard_normal((5, 12)))
    assert np.allclose(Y, [[1.0, -2.0, 3.0, 0.5]] * 5)


def test_single_path_closed_form():
    # one active path: x0 -> h1[0] -> h2[0] -> y0, all weights 2, biases 0
    w = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(w)
    p["W1"][0, 0] = 2.0
    p["W2"][0, 0] = 2.0
    p["W3"][0, 0] = 2.0
    X = np.zeros((2, 12))
    X[0, 0], X[1, 0] = 1.5, -1.5
    Y, _ = mlp.forward(w, X)
    assert Y[0, 0] == 12.0 and Y[1, 0] == 0.0 and np.all(Y[:, 1:] == 0)
    # d loss / d W3[0,0] for target 0: 2*(12-0)/8 * h2 = 3 * 6 = 18 on sample 0
    _, g = mlp.loss_and_grad(w, X, np.zeros((2, 4)))
    assert mlp.unpack(g)["W3"][0, 0] == pytest.approx(18.0)


def test_he_uniform_bounds_and_zero_bias():
    w = mlp.he_uniform_init(np.linspace(0, 1, mlp.N_PARAMS, endpoint=False))
    p = mlp.unpack(w)
    for name, fan in (("W1", 12), ("W2", 64), ("W3", 64)):
        assert np.abs(p[name]).max() <= np.sqrt(6 / fan) + 1e-12
    assert all((p[b] == 0).all() for b in ("b1", "b2", "b3"))


def test_adam_first_step_closed_form():
    # at t = 1, bias correction gives mhat = g and vhat = g^2: step = lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w = np.ones(4)
    w1, m, v = mlp.adam_step(w, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    assert np.allclose(w1, 1 - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_scaling():
    f = mlp.features(n=1 << 20, nnz=1 << 24, k=3, f_count=100, f_edges=3000, unvisited=1 << 19,
                     unvisited_edges=1 << 23, bin_counts=(90, 9, 1))
    assert f.shape == (12,)
    assert f[0] == 20 / 32 and f[1] == 24 / 32 and f[2] == 2 / 10
    assert f[7] == 0.5 and f[8] == 0.5 and np.allclose(f[9:], [0.9, 0.09, 0.01])


@pytest.mark.parametrize("seed", [0, 1])
def test_grad_scale_bounds_the_gradient(seed):
    """The magnitude scale is never below |gradient| (triangle inequality), and
    equals it when every operand is non-negative and the targets are zero, so
    that no term of any sum (nor the output error Y - T) has a negative sign."""
    rng = np.random.default_rng(seed)
    w = rand_params(seed)
    X = rng.standard_normal((9, 12))
    T = rng.standard_normal((9, 4))
    _, g = mlp.loss_and_grad(w, X, T)
    assert np.all(mlp.grad_scale(w, X, T) >= np.abs(g) - 1e-15)
    wp = np.abs(w) + 0.01
    Xp = rng.random((9, 12))
    Y, _ = mlp.forward(wp, Xp)
    Tp = np.zeros_like(Y)
    assert np.all(Y > 0)
    _, gp = mlp.loss_and_grad(wp, Xp, Tp)
    np.testing.assert_allclose(mlp.grad_scale(wp, Xp, Tp), gp, rtol=1e-12, atol=0)


def test_grad_scale_catches_a_float32_error_that_rtol_alone_would_excuse():
    """A float32 evaluation of the gradient lies well within 1e-5 of the scale; a
    perturbation of one entry by 1e-4 of its scale is outside it."""
    rng = np.random.default_rng(5)
    w = rand_params(5).astype(np.float32).astype(np.float64)
    X = rng.random((64, 12)).astype(np.float32).astype(np.float64)
    T = (3 * rng.standard_normal((64, 4))).astype(np.float32).astype(np.float64)
    _, g = mlp.loss_and_grad(w, X, T)
    s = mlp.grad_scale(w, X, T)
    g32 = g.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(g32 - g) <= 1e-5 * s + 1e-12)
    i = int(np.argmax(s))
    bad = g.copy()
    bad[i] += 1e-4 * s[i]
    assert not np.all(np.abs(bad - g) <= 1e-5 * s + 1e-12)
