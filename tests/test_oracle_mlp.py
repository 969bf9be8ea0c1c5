"""Pin of the oracle MLP's backward pass by central finite differences."""
import numpy as np

from oracle import mlp


def _setup(seed=0, n=40):
    rng = np.random.default_rng(seed)
    w = np.concatenate([rng.normal(0, 0.3, sum(mlp.sizes()[:6])), rng.normal(0, 0.5, mlp.F),
                        rng.uniform(0.5, 2.0, mlp.F), [1.0]])
    X = rng.normal(0, 1, (n, mlp.F))
    T = rng.normal(0, 0.5, n)
    return w, X, T


def test_gradient_matches_finite_differences():
    w, X, T = _setup()
    loss, g = mlp.loss_grad(w, X, T)
    rng = np.random.default_rng(1)
    idx = rng.choice(sum(mlp.sizes()[:6]), 60, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_grad(wp, X, T)[0] - mlp.loss_grad(wm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(fd))
    assert np.all(g[sum(mlp.sizes()[:6]):] == 0)


def test_adam_decreases_loss():
    w, X, T = _setup(seed=2, n=200)
    T = np.sin(X[:, 0]) * 0.3 + 0.1 * X[:, 1]
    l0 = mlp.loss_grad(w, X, T)[0]
    w2 = mlp.adam(w, X, T, 200, 3e-3)
    assert mlp.loss_grad(w2, X, T)[0] < 0.2 * l0


def _single_path_weights(a, b, c, d, mean0=0.0, scale0=1.0, out_scale=1.0):
    """Every weight zero except one path x0 -> h1_0 -> h2_0 -> y:
    y = c tanh(b tanh(a (x0 - mean0) / scale0)) + d."""
    F, H = mlp.F, mlp.H
    W1 = np.zeros((H, F))
    W1[0, 0] = a
    W2 = np.zeros((H, H))
    W2[0, 0] = b
    W3 = np.zeros(H)
    W3[0] = c
    mean = np.zeros(F)
    mean[0] = mean0
    scale = np.ones(F)
    scale[0] = scale0
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [d], mean, scale, [out_scale]])


def test_forward_single_path_closed_form():
    w = _single_path_weights(0.7, -1.3, 2.0, 0.25, mean0=0.5, scale0=2.0)
    X = np.random.default_rng(3).normal(0, 2, (50, mlp.F))
    y, _ = mlp.forward(w, X)
    ref = 2.0 * np.tanh(-1.3 * np.tanh(0.7 * (X[:, 0] - 0.5) / 2.0)) + 0.25
    assert np.abs(y - ref).max() < 1e-15


def _const_output(beta, out_scale):
    """A network whose output is the constant beta (W3 = 0, b3 = beta)."""
    return _single_path_weights(0.0, 0.0, 0.0, beta, out_scale=out_scale)


def test_guess_rule_special_cases():
    x = np.zeros(mlp.F)
    g1, g2, g3 = 1.00010, 1.00004, 1.00001        # tau = 2 max(6e-5, 3e-5) = 1.2e-4
    tau = 2.0 * 6e-5
    # inside the trust region: gamma_{n-1} + out_scale * y
    assert abs(mlp.guess(_const_output(0.5, 1e-4), x, g1, g2, g3) - (g1 + 0.5e-4)) < 1e-15
    # clamped above and below
    assert abs(mlp.guess(_const_output(3.0, 1e-4), x, g1, g2, g3) - (g1 + tau)) < 1e-15
    assert abs(mlp.guess(_const_output(-3.0, 1e-4), x, g1, g2, g3) - (g1 - tau)) < 1e-15
    # no history (gamma = 1 so far): the method's own guess
    assert mlp.guess(_const_output(0.5, 1e-4), x, 1.0, 1.0, 1.0) == 1.0
    # a guess outside (0.5, 1.5) or a non-finite output falls back to gamma_{n-1}
    assert mlp.guess(_const_output(1.0, 1.0), x, 1.45, 1.2, 1.0) == 1.45
    assert mlp.guess(_const_output(np.nan, 1.0), x, g1, g2, g3) == g1
    assert mlp.guess(_const_output(np.inf, 1.0), x, g1, g2, g3) == g1


def test_guess_uses_normalised_features():
    """The guess evaluates the network on (x - mean) / scale."""
    w = _single_path_weights(1.0, 1.0, 1.0, 0.0, mean0=3.0, scale0=4.0, out_scale=1e-6)
    x = np.zeros(mlp.F)
    x[0] = 5.0
    y = np.tanh(np.tanh((5.0 - 3.0) / 4.0))
    g = mlp.guess(w, x, 1.0 + 1e-5, 1.0, 1.0)     # tau = 2e-5 > 1e-6 y
    assert abs(g - (1.0 + 1e-5 + 1e-6 * y)) < 1e-16
