"""Pins of the oracle's 2:1 non-conforming interfaces (L2 projection mortars,
the interface treatment of the paper's adaptive runs; Sec. 4.2 notes that
they are not entropy-conservative).

* The operators against their definitions evaluated independently:
  interpolation reproduces polynomials, and the projection equals the L2
  projection integral computed by brute-force Gauss quadrature on each half.
* The right-hand side on quadtree meshes: conservation of every conserved
  variable, free-stream preservation, and convergence of the semidiscrete
  residual of the translating isentropic vortex (an exact Euler solution,
  Sec. 4.1.2) at the order of the conforming scheme.
* The paper's remark itself: with EC volume and surface fluxes the entropy
  rate vanishes to round-off on a conforming mesh, not with mortars.
* Planted mistakes (swapped halves, projection by the transpose) fail.
"""
import numpy as np
import pytest

from oracle import dgsem, physics, perrk as operrk
from oracle import lgl
import workloads


def test_interpolation_reproduces_polynomials():
    P, _ = dgsem.mortar_operators(3)
    x, _, _ = lgl.lgl(3)
    for k in range(4):
        assert np.abs(P[0] @ x ** k - (0.5 * (x - 1)) ** k).max() < 1e-14
        assert np.abs(P[1] @ x ** k - (0.5 * (x + 1)) ** k).max() < 1e-14


def test_projection_is_the_l2_projection_integral():
    """G_i = sum_j (M^-1)_ij int_{-1}^{1} l_j(s) G(s) ds with G(s) = 2 g_m(s'(s))
    on half m, integrated by 20-point Gauss on each half: equals R_0 g_0 + R_1 g_1."""
    _, R = dgsem.mortar_operators(3)
    x, _, _ = lgl.lgl(3)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((2, 4))
    gx, gw = np.polynomial.legendre.leggauss(20)
    Lx = dgsem.lagrange_matrix(x, gx)                   # l_j at Gauss points of [-1, 1]
    M = Lx.T @ (gw[:, None] * Lx)
    rhs = np.zeros(4)
    for m, shift in ((0, -1.0), (1, 1.0)):
        s = 0.5 * (gx + shift)                          # Gauss points of half m in coarse coordinates
        Gm = 2.0 * (dgsem.lagrange_matrix(x, gx) @ g[m])  # G at those points (g_m is a polynomial in s')
        rhs += dgsem.lagrange_matrix(x, s).T @ (0.5 * gw * Gm)
    ref = np.linalg.solve(M, rhs)
    assert np.abs(R[0] @ g[0] + R[1] @ g[1] - ref).max() < 1e-13


def _geo_phys(wl, surface=None):
    geo = dgsem.Geometry(wl.coords, wl.faces, mortars=wl.mortars)
    ph = physics.Physics(wl.equation, surface or wl.surface_flux)
    return geo, ph


@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("surface", ["ec", "es_rusanov"])
def test_conservation_on_quadtree(depth, surface):
    E = (6, 3) if depth == 1 else (12, 6, 3)
    wl = workloads.quadtree_patch_2d(n=8, depth=depth, E=E, surface=surface)
    assert len(wl.mortars) > 0
    geo, ph = _geo_phys(wl)
    rng = np.random.default_rng(5)
    U = wl.u0 * (1 + 0.05 * rng.standard_normal(wl.u0.shape))
    K = dgsem.rhs(geo, ph, U)
    tot = np.array([geo.integrate(K[v]) for v in range(4)])
    scale = np.array([geo.integrate(np.abs(K[v])) for v in range(4)])
    assert np.all(np.abs(tot) <= 1e-13 * scale), tot / scale


def test_free_stream_on_quadtree():
    wl = workloads.quadtree_patch_2d(n=8, depth=2, E=(12, 6, 3))
    geo, ph = _geo_phys(wl)
    U = np.broadcast_to(workloads.prim_to_cons(np.array(1.3), np.array([0.4, -0.7]), np.array(2.1))[:, None, None],
                        wl.u0.shape).copy()
    K = dgsem.rhs(geo, ph, U)
    # round-off scale of the cancelling terms: |f| (2 / h_min) / omega_end
    h_min = 2 * 5.0 / (8 * 4)
    T = max(np.abs(ph.flux(U[:, :1, :1], np.array([1.0, 0.0])[:, None, None])).max(),
            np.abs(ph.flux(U[:, :1, :1], np.array([0.0, 1.0])[:, None, None])).max()) * (2 / h_min) * 6.0
    assert np.abs(K).max() < 1e-13 * T, (np.abs(K).max(), T)


def _vortex_residual(n, depth, mortars_override=None):
    """max |F(u_exact) - du_exact/dt| for the translating vortex (v_inf = (1, 1)),
    du/dt by a centred difference in t of the exact solution."""
    tree = workloads.Quadtree.uniform(n, 5.0)
    for _ in range(depth):
        tree = tree.refine([c for c in tree.leaves if max(abs(v) for v in tree.centre(c)) < 0.35 * 5.0])
    coords, faces, mortars, _ = tree.mesh()
    if mortars_override is not None:
        mortars = mortars_override(mortars)
    x, y = coords[:, :, 0], coords[:, :, 1]
    c = (0.3, -0.2)
    U = workloads.to_soa(workloads.isentropic_vortex(x, y, 0.0, c, 4.0, L=5.0, R=1.0))
    eps = 1e-5
    Up = workloads.to_soa(workloads.isentropic_vortex(x, y, eps, c, 4.0, L=5.0, R=1.0))
    Um = workloads.to_soa(workloads.isentropic_vortex(x, y, -eps, c, 4.0, L=5.0, R=1.0))
    dUdt = (Up - Um) / (2 * eps)
    geo = dgsem.Geometry(coords, faces, mortars=mortars)
    K = dgsem.rhs(geo, physics.Physics("euler2d", "es_rusanov"), U)
    return float(np.abs(K - dUdt).max())


def test_vortex_residual_converges_through_mortars():
    e1 = _vortex_residual(8, 1)
    e2 = _vortex_residual(16, 1)
    order = np.log2(e1 / e2)
    print("residual", e1, e2, "order", order)
    assert order > 2.5


def test_planted_swapped_halves_fail_convergence():
    swap = lambda m: m[:, [0, 1, 3, 2]]
    e1 = _vortex_residual(8, 1, swap)
    e2 = _vortex_residual(16, 1, swap)
    assert np.log2(e1 / e2) < 1.5


def test_planted_transpose_projection_fails_conservation(monkeypatch):
    P, R = dgsem.mortar_operators(3)
    monkeypatch.setattr(dgsem, "mortar_operators", lambda N=3: (P, [0.5 * Pm.T for Pm in P]))
    wl = workloads.quadtree_patch_2d(n=8, depth=1)
    geo, ph = _geo_phys(wl)
    K = dgsem.rhs(geo, ph, wl.u0)
    tot = abs(geo.integrate(K[0]))
    assert tot > 1e-8 * geo.integrate(np.abs(K[0]))


def test_entropy_conserved_only_without_mortars():
    """EC volume and surface fluxes: sum omega J w.F(U) = 0 to round-off on
    the conforming mesh; the L2 mortars break it (the paper's remark)."""
    rng = np.random.default_rng(9)
    rates = {}
    for depth in (0, 1):
        wl = workloads.quadtree_patch_2d(n=8, depth=depth, E=(6, 3) if depth else (3,), surface="ec")
        geo, ph = _geo_phys(wl)
        U = wl.u0 * (1 + 0.05 * rng.standard_normal(wl.u0.shape))
        K = dgsem.rhs(geo, ph, U)
        W = ph.entropy_vars(U)
        rates[depth] = abs(geo.integrate(np.sum(W * K, axis=0))) / geo.integrate(np.sum(np.abs(W * K), axis=0))
    assert rates[0] < 1e-13
    assert rates[1] > 1e-9


def test_relaxed_stage_loop_conserves_on_quadtree():
    """Ten relaxed P-ERRK steps with partitions by refinement level: mass,
    momentum and energy kept to round-off, the relaxation target met."""
    wl = workloads.quadtree_patch_2d(n=8, depth=2, E=(12, 6, 3))
    s = operrk.Solver(wl)
    geo = s.geo
    m0 = [geo.integrate(wl.u0[v]) for v in range(4)]
    for _ in range(10):
        r = s.step(wl.dt)
        assert r.converged and abs(r.H_next - (r.H_n + r.gamma * r.dH)) <= 1e-12 * s.abs_entropy(s.U)
    for v in range(4):
        assert abs(geo.integrate(s.U[v]) - m0[v]) <= 1e-13 * geo.integrate(np.abs(s.U[v]))
