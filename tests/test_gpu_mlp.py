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


def _per_sample_abs(w, X, T):
    """sum over samples of |each sample's contribution| to the full-batch
    gradient, per parameter: the scale of that component's float32 rounding."""
    n = len(T)
    acc = 0.0
    for i in range(n):
        acc = acc + np.abs(omlp.loss_grad(w, X[i:i + 1], T[i:i + 1])[1]) / n
    return acc


def test_device_gradient_matches_oracle_elementwise():
    """Every gradient entry of the device backward pass against the float64
    oracle, to float32 accuracy of that entry's own sum: |g_dev - g| <= 1e-5
    times the sum of the absolute per-sample contributions (plus 1e-7 of the
    largest entry, for the entries that cancel to ~0)."""
    X, T = _data(1, 300)
    w = pk.mlp_init(3)
    w[omlp.H * 6 + omlp.H + omlp.H * omlp.H + omlp.H + omlp.H + 1:][:6] = 0.1      # non-trivial normalisation
    g_dev, loss_dev = pk.perrk_mlp_grad(X, T, w)
    Xf = X.astype(np.float32).astype(np.float64)
    Tf = T.astype(np.float32).astype(np.float64)
    w64 = w.astype(np.float64)
    loss, g = omlp.loss_grad(w64, Xf, Tf)
    assert abs(loss_dev - loss) <= 1e-5 * loss
    ntr = sum(omlp.sizes()[:6])
    scale = _per_sample_abs(w64, Xf, Tf)[:ntr]
    err = np.abs(g_dev[:ntr].astype(np.float64) - g[:ntr])
    bound = 1e-5 * scale + 1e-7 * np.abs(g[:ntr]).max()
    assert np.all(err <= bound), (int(np.argmax(err / bound)), float(np.max(err / bound)))
    assert np.all(g_dev[ntr:] == 0.0)


@pytest.mark.parametrize("epochs", [1, 5])
def test_device_adam_weights_track_oracle(epochs):
    """The weights after k epochs of device Adam against oracle Adam on the
    same float32-rounded data.  Adam's step lr m^/(sqrt(v^) + eps) is a smooth
    function of the gradient history where every gradient entry is well away
    from zero, so there the float32 and float64 weights agree to ~1e-6 of the
    distance moved; entries whose gradient came near zero in some epoch can
    flip a step's sign and only keep the bound |w_dev - w_0| <= k lr."""
    X, T = _data(2, 400)
    w0 = pk.mlp_init(4)
    lr = 3e-3
    w_dev, _ = pk.perrk_mlp_train(X, T, w0, epochs, lr)
    Xf = X.astype(np.float32).astype(np.float64)
    Tf = T.astype(np.float32).astype(np.float64)
    grads = []
    w_ref = omlp.adam(w0.astype(np.float64), Xf, Tf, epochs, lr, grads=grads)
    ntr = sum(omlp.sizes()[:6])
    G = np.abs(np.array(grads))                              # [epochs, ntr]
    well = np.all(G >= 1e-3 * G.max(axis=1, keepdims=True), axis=0)
    assert well.mean() > 0.5
    d = np.abs(w_dev[:ntr].astype(np.float64) - w_ref[:ntr])
    assert np.all(d[well] <= 1e-4 * epochs * lr + 2e-7 * np.abs(w_ref[:ntr][well])), float(d[well].max())
    moved = np.abs(w_dev[:ntr].astype(np.float64) - w0[:ntr].astype(np.float64))
    assert np.all(moved <= epochs * lr * (1 + 1e-3) + 2e-7 * np.abs(w0[:ntr]))
    assert np.all(w_dev[ntr:] == w0[ntr:])


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


def _history_from_records(recs):
    """(gamma_{n-1}, gamma_{n-2}, gamma_{n-3}) before each step, rebuilt from
    the step records: a step's gamma enters the history only if its solve
    converged (no fallback flag); 1 before the first steps."""
    hist = [1.0, 1.0, 1.0]
    out = []
    for r in recs:
        out.append(tuple(hist))
        if not r["flags"] & pk.FLAG_NEWTON_FALLBACK:
            hist = [r["gamma"], hist[0], hist[1]]
    return out


@pytest.mark.parametrize("n_inst", [1, 3])
def test_learned_guess_matches_oracle_rule(n_inst):
    """The device's learned initial guess gamma_0 per step and instance
    against the oracle's guess rule (network, output scale, gamma_{n-1}
    increment, trust-region clamp, fallback) evaluated on the step's recorded
    features and the gamma history of the records.  The network runs in
    float32 on the device: the increments agree to 2e-5 of out_scale (1 + |y|)."""
    base = workloads.small_box_2d(n=8, seed=61, R=2, E=[6, 3], order=3, ic="khi")
    base.dt *= 4
    train = _run(base, 60, pk.GUESS_PREV)
    X, T = pk.mlp_dataset([[r] for r in train])
    W, _ = pk.mlp_fit(X, T, epochs=300, lr=3e-3)
    wls = [workloads.small_box_2d(n=8, seed=61 + k, R=2, E=[6, 3], order=3, ic="khi") for k in range(n_inst)]
    for wl in wls:
        wl.dt = base.dt
    s = pk.Solver(wls, pk.options(guess=pk.GUESS_MLP, max_it=8, tol_r=1e-14, tol_g=1e-14))
    s.set_mlp(W)
    recs = s.step(40)
    s.close()
    out_scale = float(W[-1])
    n_clamped = n_free = 0
    for k in range(n_inst):
        rk = [row[k] for row in recs]
        for r, (g1, g2, g3) in zip(rk, _history_from_records(rk)):
            assert r["gamma_prev"] == g1
            x = np.asarray(r["features"], dtype=np.float64)
            g0 = omlp.guess(W.astype(np.float64), x, g1, g2, g3)
            y = float(omlp.forward(W.astype(np.float64), x[None, :])[0][0])
            tau = 2.0 * max(abs(g1 - g2), abs(g2 - g3))
            tol = 2e-5 * abs(out_scale) * (1.0 + abs(y)) + 1e-15
            assert abs(r["gamma_guess"] - g0) <= tol, (k, r["gamma_guess"], g0, tol)
            if tau > 0 and abs(out_scale * y) > tau * (1 + 1e-3):
                n_clamped += 1
            elif tau > 0:
                n_free += 1
    assert n_free > 0
