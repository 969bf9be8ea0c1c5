"""Legendre-Gauss-Lobatto quadrature and the nodal differentiation matrix.

The DGSEM collocates solution and quadrature on the N+1 LGL nodes (the paper
uses DGSEM with k = 3, Sec. 2.1 and Sec. 4.1).  Nodes: the end points and the
roots of P_N' (float64 roots refined by Newton's method on P_N' in extended
precision, so that D is that of the exact nodes: D multiplies large
free-stream fluxes whose differences are small); weights
2 / (N (N+1) P_N(x_i)^2); D_ij = l_j'(x_i) from the barycentric form of the
Lagrange basis, evaluated in extended precision.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def _legendre(N, x):
    """P_N(x), P_N'(x), P_N''(x) by the three-term recurrence (x in extended precision)."""
    p0, p1 = np.ones_like(x), x.copy()
    if N == 0:
        return p0, 0 * x, 0 * x
    for k in range(1, N):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    with np.errstate(divide="ignore", invalid="ignore"):      # endpoints: only P_N is used there
        dp = N * (x * p1 - p0) / (x * x - 1)
        d2p = (2 * x * dp - N * (N + 1) * p1) / (1 - x * x)
    return p1, dp, d2p


def lgl_nodes_weights(N, extended=False):
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    interior = np.sort(npleg.legroots(npleg.legder(cN)).real).astype(np.longdouble)
    for _ in range(6):
        _, dp, d2p = _legendre(N, interior)
        interior = interior - dp / d2p
    x = np.concatenate([[np.longdouble(-1)], interior, [np.longdouble(1)]])
    PN, _, _ = _legendre(N, x)
    w = 2 / (N * (N + 1) * PN * PN)
    if extended:
        return x, w
    return x.astype(np.float64), w.astype(np.float64)


def diff_matrix(x):
    """D_ij = l_j'(x_i) via barycentric weights lambda_j = 1 / prod_{k!=j}(x_j - x_k)."""
    xl = np.asarray(x, dtype=np.longdouble)
    n = len(xl)
    lam = np.ones(n, dtype=np.longdouble)
    for j in range(n):
        for k in range(n):
            if k != j:
                lam[j] /= (xl[j] - xl[k])
    D = np.zeros((n, n), dtype=np.longdouble)
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (xl[i] - xl[j])
        D[i, i] = -np.sum(D[i, :])
    return D.astype(np.float64)


def lgl(N=3):
    xl, wl = lgl_nodes_weights(N, extended=True)
    return xl.astype(np.float64), wl.astype(np.float64), diff_matrix(xl)
