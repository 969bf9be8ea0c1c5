"""Optimised stability polynomials on the GPU path: the Jacobian the
optimiser reads (through perrk_rhs) against the oracle's, stepping parity of a
family built from stability polynomials, and the optimised member staying
stable, in the linear regime, at a step where the default member grows."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
from paper_2507_04991_gb300 import stability as st
import workloads
from oracle import dgsem, perrk as operrk, physics, tableau as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    __graft_entry__.build()
    torch.zeros(1, device="cuda")


def _free_stream(wl, amp, seed):
    rng = np.random.default_rng(seed)
    u = np.empty_like(wl.u0)
    u[0] = 1.0
    u[1] = 0.5
    u[2] = 0.3
    u[3] = 1.0 / 0.4 + 0.5 * (0.25 + 0.09)
    return u * (1.0 + amp * rng.standard_normal(u.shape))


def _one_partition(S, p, n=4):
    return workloads.small_box_2d(n=n, seed=51, R=1, E=[S], order=p)


def test_jacobian_matches_oracle():
    wl = _one_partition(6, 3)
    u = _free_stream(wl, 1e-3, 1)
    s = pk.Solver(wl, pk.options())
    J = st.jacobian(s, u)
    s.close()
    geo = dgsem.Geometry(wl.coords, wl.faces)
    ph = physics.Physics(wl.equation, wl.surface_flux, wl.gamma_gas)
    f0 = dgsem.rhs(geo, ph, u).ravel()
    step = 1e-7 * max(1.0, float(np.abs(u).max()))
    cols = []
    for k in range(0, u.size, 37):                 # sampled columns
        du = u.copy().ravel()
        du[k] += step
        cols.append((k, (dgsem.rhs(geo, ph, du.reshape(u.shape)).ravel() - f0) / step))
    scale = np.abs(J).max()
    for k, col in cols:
        assert np.abs(J[:, k] - col).max() < 1e-6 * scale, k


def _chain_alphas(p, E_list, seed):
    rng = np.random.default_rng(seed)
    S = max(E_list)
    c, b = T.abscissae(p, S), T.weights(p, S)
    out = []
    for E in E_list:
        A = T.member(p, S, E)
        first = S - E + 2
        for m in range(first + 1, S):
            if A[m - 1, m - 2] != 0.0:
                a = A[m - 1, m - 2] * (1.0 + 0.2 * rng.uniform(-1, 1))
                A[m - 1, m - 2] = a
                A[m - 1, 0] = c[m - 1] - a
        if p == 3 and E > 3:
            A[S - 1, S - 2] = (1.0 - A[S - 2, S - 3]) / 4.0
            A[S - 1, 0] = c[S - 1] - A[S - 1, S - 2]
        elif p == 2:
            m = S
            a = A[m - 1, m - 2] * (1.0 + 0.2 * rng.uniform(-1, 1))
            A[m - 1, m - 2] = a
            A[m - 1, 0] = c[m - 1] - a
        out.append(T.stability_coeffs(b, A)[:E + 1])
    return out


@pytest.mark.parametrize("p,E", [(2, [6, 4, 2]), (3, [7, 5, 3])])
def test_polynomial_family_step_parity(p, E):
    wl = workloads.small_box_2d(n=6, seed=52, R=3, E=E, order=p, random_parts=True)
    alphas = _chain_alphas(p, E, 53)
    ref = operrk.Solver(wl, operrk.NewtonOptions(tol_r=1e-14, tol_g=1e-14), alphas=alphas)
    for _ in range(6):
        ref.step(wl.dt)
    tab = st.optimised_tableau(p, E, alphas)
    s = pk.Solver(wl, pk.options(max_it=10, tol_r=1e-14, tol_g=1e-14), tableaux=[tab])
    s.step(6)
    u = s.state()
    s.close()
    assert np.abs(u - ref.U).max() / np.abs(ref.U).max() < 1e-10


@pytest.mark.parametrize("p", [3, 4])
def test_optimised_member_stable_where_default_grows(p):
    """One partition, S = E = 8, around a free stream (perturbation 1e-6, so
    the linearisation governs).  At the optimised step h_opt the optimised
    member's amplification max |P(h lambda)| is <= 1 on the spectrum the
    library's right-hand side gives, the default member's is above 1;
    stepping for as many steps as that rate needs to grow 1e3-fold shows the
    same on the GPU.  p = 3 from the optimised polynomial, p = 4 from its
    directly optimised chain."""
    import math
    S = 8
    wl = _one_partition(S, p)
    base = _free_stream(wl, 0.0, 0)
    s = pk.Solver(wl, pk.options(relaxation=False))
    lam = st.jacobian_spectrum(s, base)
    s.close()
    if p == 3:
        h_opt, alpha = st.optimal_polynomial(lam, p, S, n_dir=32, rel_tol=1e-3)
        tab = st.optimised_tableau(p, [S], [alpha])
    else:
        c, b, a1, asub, steps = st.optimised_family_p4(lam, [S], max_eval=200)
        tab, h_opt = (c, b, a1, asub), steps[0]
    A = np.zeros((S, S))
    for i in range(1, S):
        A[i, 0] += tab[2][0, i]
        A[i, i - 1] += tab[3][0, i]
    alpha = T.stability_coeffs(tab[1], A)[:S + 1]
    a_def = T.stability_coeffs(T.weights(p, S), T.member(p, S, S))[:S + 1]
    h_def = st.stable_step(a_def, lam, 2.0 * h_opt)
    assert h_opt > 1.5 * h_def, (h_opt, h_def)
    dt = h_opt
    rho_opt = np.abs(np.polyval(alpha[::-1], dt * lam)).max()
    rho_def = np.abs(np.polyval(a_def[::-1], dt * lam)).max()
    assert rho_opt <= 1.0 + 1e-7 and rho_def > 1.0 + 1e-3, (rho_opt, rho_def)
    nsteps = min(5000, int(math.ceil(math.log(1e3) / math.log(rho_def))))
    u0 = _free_stream(wl, 1e-6, 2)

    def growth(t):
        s = pk.Solver(wl, pk.options(relaxation=False), tableaux=[t])
        s.set_state(u0)
        s.set_dt(dt)
        s.step(nsteps, info=False)
        u = s.state()
        s.close()
        return np.abs(u - base).max() / np.abs(u0 - base).max()

    g_opt = growth(tab)
    g_def = growth(pk.perrk_build_tableau(p, [S]))
    assert g_opt < 20.0, (g_opt, nsteps)
    assert g_def > 100.0 or not np.isfinite(g_def), (g_def, nsteps, rho_def)
