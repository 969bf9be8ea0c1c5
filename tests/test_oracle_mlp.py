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
