"""Legendre-Gauss-Lobatto quadrature and the nodal differentiation matrix.

The DGSEM collocates solution and quadrature on the N+1 LGL nodes (the paper
uses DGSEM with k = 3, Sec. 2.1 and Sec. 4.1).  Nodes: the end points and the
roots of P_N'; weights 2 / (N (N+1) P_N(x_i)^2); D_ij = l_j'(x_i) from the
barycentric form of the Lagrange basis, evaluated in extended precision.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def lgl_nodes_weights(N):
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    interior = npleg.legroots(npleg.legder(cN))
    x = np.concatenate([[-1.0], np.sort(interior.real), [1.0]])
    PN = npleg.legval(x, cN)
    w = 2.0 / (N * (N + 1) * PN * PN)
    return x, w


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
    x, w = lgl_nodes_weights(N)
    return x, w, diff_matrix(x)
