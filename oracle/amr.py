"""Adaptive mesh refinement on quadtree meshes of 2D boxes (oracle, float64):
the refinement indicator and the solution transfer between meshes.

The paper's adaptive runs (Sec. 3.2.2, Sec. 5.3) refine where the
shock-capturing indicator of Hennemann et al. (2021) computed from the
density is large; the mesh changes every few steps and the partitions are
re-derived from the new element sizes (Sec. 2.2).

Indicator of one element (N = 3): the indicator variable (here the density)
in the orthonormal Legendre basis, m = (V^-1 (x) V^-1) rho with
V_ik = sqrt((2k+1)/2) P_k(x_i) on the LGL nodes; the energies
E_N = sum_{a,b <= N} m_ab^2, E_{N-1} and E_{N-2} of the modes up to degree
N-1 and N-2 in each direction; the relative energy of the highest modes
    e = max((E_N - E_{N-1}) / E_N, (E_{N-1} - E_{N-2}) / E_{N-1}),
the threshold T = 0.5 10^(-1.8 (N+1)^(1/4)), the sharpness s = log((1 - 1e-4) / 1e-4),
and the indicator alpha = 1 / (1 + exp(-(s / T) (e - T))).

Transfer (N = 3, child (a, b) of a parent covers the parent's reference
quarter a in xi and b in eta, a, b in {0, 1}, child index a + 2 b):
  refine:  the child's nodal values are the parent polynomial at the child's
           nodes, u_c = (P_b (x) P_a) u_parent, P_0, P_1 the half-interval
           interpolation matrices of the mortars;
  coarsen: the L2 projection of the four children onto the parent,
           u_parent = 1/4 sum_{a,b} (R_b (x) R_a) u_(a,b), R_m = M^-1 P_m^T M.
Both keep every element integral sum omega J u exactly (up to rounding).
"""
import math

import numpy as np

from . import dgsem, lgl as _lgl


def legendre_vandermonde(N=3):
    """V_ik = sqrt((2k+1)/2) P_k(x_i) on the LGL nodes (orthonormal Legendre basis)."""
    x, _, _ = _lgl.lgl(N)
    V = np.zeros((N + 1, N + 1))
    for k in range(N + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        V[:, k] = math.sqrt((2 * k + 1) / 2.0) * np.polynomial.legendre.legval(x, c)
    return V


def indicator(rho, N=3):
    """Hennemann et al.'s indicator per element; rho[n_elem, (N+1)^2] nodal
    density (index i + (N+1) j)."""
    Vinv = np.linalg.inv(legendre_vandermonde(N))
    n = N + 1
    r = rho.reshape(-1, n, n)                         # [e, j, i]
    m = np.einsum("ai,bj,eji->eba", Vinv, Vinv, r)    # m[e, b (eta degree), a (xi degree)]
    m2 = m * m
    E_N = m2.sum(axis=(1, 2))
    E_1 = m2[:, :N, :N].sum(axis=(1, 2))
    E_2 = m2[:, :N - 1, :N - 1].sum(axis=(1, 2))
    e = np.maximum((E_N - E_1) / E_N, (E_1 - E_2) / E_1)
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    s = math.log((1.0 - 1e-4) / 1e-4)
    return 1.0 / (1.0 + np.exp(-(s / T) * (e - T)))


def _ops(N=3):
    P, R = dgsem.mortar_operators(N)
    return P, R


def refine_child(u_parent, child, N=3):
    """u_parent[V, (N+1)^2] -> the child's nodal values [V, (N+1)^2]."""
    P, _ = _ops(N)
    a, b = child & 1, child >> 1
    n = N + 1
    up = u_parent.reshape(-1, n, n)                   # [V, j, i]
    return np.einsum("jl,ik,vlk->vji", P[b], P[a], up).reshape(u_parent.shape)


def coarsen_parent(u_children, N=3):
    """u_children[4][V, (N+1)^2] (child index a + 2 b) -> the parent's nodal values."""
    _, R = _ops(N)
    n = N + 1
    out = 0.0
    for c, uc in enumerate(u_children):
        a, b = c & 1, c >> 1
        out = out + 0.25 * np.einsum("jl,ik,vlk->vji", R[b], R[a], uc.reshape(-1, n, n))
    return out.reshape(u_children[0].shape)


def transfer(U_old, amap, N=3):
    """U_old[V, n_old, NP] -> U_new[V, n_new, NP] by a map of rows
    (kind, a0, a1, a2, a3): kind 0 copy of old element a0; 1 child a1 of old
    element a0; 2 parent of the old children a0..a3 (child order a + 2 b)."""
    amap = np.asarray(amap)
    V, _, NP = U_old.shape
    U = np.empty((V, len(amap), NP))
    for e, (kind, a0, a1, a2, a3) in enumerate(amap):
        if kind == 0:
            U[:, e] = U_old[:, a0]
        elif kind == 1:
            U[:, e] = refine_child(U_old[:, a0], int(a1), N)
        else:
            U[:, e] = coarsen_parent([U_old[:, k] for k in (a0, a1, a2, a3)], N)
    return U
