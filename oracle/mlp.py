"""2 x 64 tanh multilayer perceptron in float64 (oracle of the learned
Newton-guess kernels).  Weight layout (that of the C ABI): W1[64][F], b1[64],
W2[64][64], b2[64], W3[64], b3, then F input means, F input scales and an
output scale (the last three groups only normalise; they are not trained).

forward:  x^ = (x - mean) / scale, h1 = tanh(W1 x^ + b1), h2 = tanh(W2 h1 + b2),
          y = W3 . h2 + b3
loss:     mean over samples of (y - t)^2
gradient: chain rule (d tanh(z)/dz = 1 - tanh(z)^2)
Adam:     Kingma & Ba (2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.

guess:    the learned Newton initial guess for the relaxation equation
          (Sec. 3.1 starts Newton from gamma_{n-1}; the network predicts the
          step-to-step change instead):
          inc = clamp(out_scale * y(x), -tau, tau),
          tau = 2 max(|g1 - g2|, |g2 - g3|) with g1, g2, g3 = gamma_{n-1},
          gamma_{n-2}, gamma_{n-3} (the last converged values, 1 before the
          first steps), and gamma_0 = g1 + inc; a guess that is not finite or
          lies outside (0.5, 1.5) falls back to the method's own g1.  The clamp
          is a trust region: the learned increment moves the guess no further
          than the recent history of gamma itself moved.
"""
import numpy as np

F, H = 6, 64


def sizes():
    return [H * F, H, H * H, H, H, 1, F, F, 1]


def unpack(w):
    out, o = [], 0
    for n in sizes():
        out.append(w[o:o + n])
        o += n
    W1, b1, W2, b2, W3, b3, mean, scale, oscale = out
    return W1.reshape(H, F), b1, W2.reshape(H, H), b2, W3, b3, mean, scale, oscale


def forward(w, X):
    W1, b1, W2, b2, W3, b3, mean, scale, _ = unpack(np.asarray(w, dtype=np.float64))
    Xn = (X - mean) / scale
    h1 = np.tanh(Xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3 + b3[0], (Xn, h1, h2)


def loss_grad(w, X, T):
    w = np.asarray(w, dtype=np.float64)
    W1, b1, W2, b2, W3, b3, mean, scale, _ = unpack(w)
    y, (Xn, h1, h2) = forward(w, X)
    n = len(T)
    err = y - T
    loss = float(np.mean(err * err))
    dy = 2.0 * err / n
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = np.outer(dy, W3) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ Xn
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3, np.zeros(2 * F + 1)])
    return loss, g


def adam(w, X, T, epochs, lr, b1=0.9, b2=0.999, eps=1e-8, grads=None):
    """Full-batch Adam; when grads is a list, each epoch's gradient is appended."""
    w = np.asarray(w, dtype=np.float64).copy()
    ntrain = sum(sizes()[:6])
    m = np.zeros(ntrain)
    v = np.zeros(ntrain)
    for t in range(1, epochs + 1):
        _, g = loss_grad(w, X, T)
        g = g[:ntrain]
        if grads is not None:
            grads.append(g.copy())
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        w[:ntrain] -= lr * mh / (np.sqrt(vh) + eps)
    return w


def guess(w, x, g1, g2, g3):
    """Learned initial guess gamma_0 for one step (see the module docstring).
    x: the step's F features; g1, g2, g3: gamma_{n-1}, gamma_{n-2}, gamma_{n-3}."""
    w = np.asarray(w, dtype=np.float64)
    y, _ = forward(w, np.asarray(x, dtype=np.float64)[None, :])
    out_scale = unpack(w)[8][0]
    raw = out_scale * float(y[0])
    if not np.isfinite(raw):
        return g1
    tau = 2.0 * max(abs(g1 - g2), abs(g2 - g3))
    inc = min(max(raw, -tau), tau)
    g0 = g1 + inc
    if not np.isfinite(g0) or not abs(g0 - 1.0) < 0.5:
        return g1
    return g0
