"""Pins of the oracle's AMR parts (oracle/amr.py): the indicator of Hennemann
et al. (2021) on known modal content, and the solution transfer between
quadtree meshes (refinement by interpolation, coarsening by L2 projection)
against polynomial exactness and conservation; a planted mistake fails."""
import math

import numpy as np
import pytest

from oracle import amr, dgsem, lgl
import workloads

X = lgl.lgl(3)[0]


def _orthonormal(k, x):
    c = np.zeros(k + 1)
    c[k] = 1.0
    return math.sqrt((2 * k + 1) / 2.0) * np.polynomial.legendre.legval(x, c)


def test_indicator_recovers_modal_energy():
    """rho = c0 L0(x) + c3 L3(x) (orthonormal Legendre, constant in y): the
    highest-mode energy is c3^2 / (c0^2 + c3^2); alpha follows from it."""
    T = 0.5 * 10.0 ** (-1.8 * 4 ** 0.25)
    s = math.log((1 - 1e-4) / 1e-4)
    for c0, c3 in ((2.0, 0.0), (2.0, 0.01), (1.5, 0.3), (1.0, 1.0)):
        rx = c0 * _orthonormal(0, X) + c3 * _orthonormal(3, X)
        # y-constant field: a 2D orthonormal mode factor L0(y) = 1/sqrt(2)
        rho = np.tile(rx, 4)[None, :]
        e = c3 ** 2 / (c0 ** 2 + c3 ** 2)
        alpha = amr.indicator(rho)[0]
        assert abs(alpha - 1.0 / (1.0 + math.exp(-(s / T) * (e - T)))) < 1e-12


def test_indicator_second_mode_branch():
    """Energy in degree N-1 only: e = (E_{N-1} - E_{N-2}) / E_{N-1}."""
    c0, c2 = 1.0, 0.2
    rx = c0 * _orthonormal(0, X) + c2 * _orthonormal(2, X)
    rho = np.tile(rx, 4)[None, :]
    e = c2 ** 2 / (c0 ** 2 + c2 ** 2)
    T = 0.5 * 10.0 ** (-1.8 * 4 ** 0.25)
    s = math.log((1 - 1e-4) / 1e-4)
    assert abs(amr.indicator(rho)[0] - 1.0 / (1.0 + math.exp(-(s / T) * (e - T)))) < 1e-12


def _poly(x, y):
    return 1.0 + 0.3 * x - 0.2 * y + 0.1 * x ** 3 * y ** 2 - 0.05 * x * y ** 3


def test_refinement_is_exact_for_polynomials():
    XX, YY = np.meshgrid(X, X)                        # [j, i]
    up = _poly(XX, YY).ravel()[None]
    for child in range(4):
        a, b = child & 1, child >> 1
        xc, yc = 0.5 * (X + (2 * a - 1)), 0.5 * (X + (2 * b - 1))
        XC, YC = np.meshgrid(xc, yc)
        assert np.abs(amr.refine_child(up, child) - _poly(XC, YC).ravel()[None]).max() < 1e-14


def test_coarsening_projects_back_and_conserves():
    rng = np.random.default_rng(4)
    up = rng.standard_normal((4, 16))
    kids = [amr.refine_child(up, c) for c in range(4)]
    assert np.abs(amr.coarsen_parent(kids) - up).max() < 1e-13          # projection of an interpolant
    w2 = np.outer(lgl.lgl(3)[1], lgl.lgl(3)[1]).ravel()
    kids = [rng.standard_normal((4, 16)) for _ in range(4)]
    par = amr.coarsen_parent(kids)
    # J of a child is a quarter of the parent's
    assert np.abs(par @ w2 - 0.25 * sum(k @ w2 for k in kids)).max() < 1e-14


def test_planted_interpolation_instead_of_projection_fails(monkeypatch):
    P, R = dgsem.mortar_operators(3)
    monkeypatch.setattr(amr, "_ops", lambda N=3: (P, [2.0 * p.T for p in P]))
    rng = np.random.default_rng(5)
    kids = [rng.standard_normal((1, 16)) for _ in range(4)]
    w2 = np.outer(lgl.lgl(3)[1], lgl.lgl(3)[1]).ravel()
    par = amr.coarsen_parent(kids)
    assert abs(par @ w2 - 0.25 * sum(k @ w2 for k in kids)).max() > 1e-6


def test_adapt_map_and_mass_through_cycles():
    """Refine where a KHI-like density is steep, then coarsen back: the map
    rows describe the new leaves, and the total mass is kept exactly."""
    tree = workloads.Quadtree.uniform(8, 1.0)
    wl = workloads.quadtree_workload(tree, "t", (3,), 3, ic="khi")
    U = wl.u0
    geo = dgsem.Geometry(wl.coords, wl.faces, mortars=wl.mortars)
    m0 = geo.integrate(U[0])
    for cycle in range(3):
        alpha = amr.indicator(U[0])
        ref, coa = workloads.amr_marks(tree, alpha, thresholds=(0.3, 0.9), levels=(0, 1, 2))
        if cycle == 2:
            ref, coa = [], [c for c in tree.leaves if c[0] > 0]
        new, amap = tree.adapt(ref, coa)
        U = amr.transfer(U, amap)
        tree = new
        coords, faces, mortars, levels = tree.mesh()
        geo = dgsem.Geometry(coords, faces, mortars=mortars)
        assert abs(geo.integrate(U[0]) - m0) < 1e-13 * abs(m0)
    assert len(tree.leaves) >= 64
