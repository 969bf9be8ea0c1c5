"""GPU checks of the learned Newton guess: device gradient against the float64
oracle MLP, device training, and the guess in the relaxation loop (fewer
full-state passes than the gamma_{n-1} guess, same converged gamma)."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, 6))
    T = 0.3 * np.sin(X[:, 0]) + 0.1 * X[:, 1] * X[:, 2]
    return X, T


def test_device_gradient_matches_oracle():
    X, T = _data(1, 300)
    w = pk.mlp_init(3)
    w[omlp.H * 6 + omlp.H + omlp.H * omlp.H + omlp.H + omlp.H + 1:][:6] = 0.1      # non-trivial normalisation
    g_dev, loss_dev = pk.perrk_mlp_grad(X, T, w)
    Xf = X.astype(np.float32).astype(np.float64)
    Tf = T.astype(np.float32).astype(np.float64)
    loss, g = omlp.loss_grad(w.astype(np.float64), Xf, Tf)
    assert abs(loss_dev - loss) <= 1e-5 * loss
    ntr = sum(omlp.sizes()[:6])
    assert np.linalg.norm(g_dev[:ntr] - g[:ntr]) <= 1e-4 * np.linalg.norm(g[:ntr])


def test_device_training_tracks_oracle_adam():
    X, T = _data(2, 400)
    w0 = pk.mlp_init(4)
    w_dev, loss_dev = pk.perrk_mlp_train(X, T, w0, 150, 3e-3)
    w_ref = omlp.adam(w0.astype(np.float64), X.astype(np.float32).astype(np.float64),
                      T.astype(np.float32).astype(np.float64), 150, 3e-3)
    loss_ref = omlp.loss_grad(w_ref, X, T)[0]
    loss0 = omlp.loss_grad(w0.astype(np.float64), X, T)[0]
    assert loss_dev < 0.3 * loss0 and loss_ref < 0.3 * loss0
    assert abs(loss_dev - loss_ref) <= 0.1 * loss_ref


def _run(wl, steps, guess, weights=None, precision=pk.FP64):
    s = pk.Solver(wl, pk.options(precision=precision, guess=guess, max_it=8, tol_r=1e-14, tol_g=1e-14))
    if weights is not None:
        s.set_mlp(weights)
    recs = [r[0] for r in s.step(steps)]
    s.close()
    return recs


def test_learned_guess_cuts_newton_passes_same_gamma():
    """Train on gamma traces of the plain method (guess gamma_{n-1}), then run
    the same problem with the learned guess: fewer full-state passes on
    average, and the converged gamma is the same root (Newton still decides)."""
    wl = workloads.small_box_2d(n=8, seed=61, R=2, E=[6, 3], order=3, ic="khi")
    wl.dt *= 4
    train = _run(wl, 120, pk.GUESS_PREV)
    X, T = pk.mlp_dataset([[r] for r in train])
    W, loss = pk.mlp_fit(X, T, epochs=600, lr=3e-3)
    prev = _run(wl, 120, pk.GUESS_PREV)
    one = _run(wl, 120, pk.GUESS_ONE)
    learned = _run(wl, 120, pk.GUESS_MLP, W)
    it = lambda rs: float(np.mean([r["iters"] for r in rs[3:]]))
    err = lambda rs: float(np.mean([abs(r["gamma_guess"] - r["gamma"]) for r in rs[3:]]))
    print("passes one/prev/mlp", it(one), it(prev), it(learned), "guess error", err(one), err(prev), err(learned))
    assert err(learned) < err(prev) < err(one)
    assert it(learned) <= it(prev) <= it(one)
    for a, b in zip(prev, learned):
        assert abs(a["gamma"] - b["gamma"]) < 1e-9
