"""Pins of the oracle's P-ERRK stepping against closed forms and invariants."""
import math

import numpy as np
import pytest

import workloads
from oracle import perrk, tableau


def test_closed_form_gamma_quadratic_entropy():
    """Burgers, s = u^2/2: r(g) = g dt <u,d> + g^2 dt^2 <d,d>/2 - g dH has the
    nonzero root g = 2 (dH - dt <u,d>) / (dt^2 <d,d>) (inner products with omega J)."""
    wl = workloads.burgers_1d()
    s = perrk.Solver(wl, perrk.NewtonOptions(tol_r=1e-15, tol_g=1e-16))
    for _ in range(3):
        U = s.U.copy()
        dt = wl.dt * 2
        d, dH, _ = s.stages(U, dt)
        ud = s.geo.integrate(U[0] * d[0])
        dd = s.geo.integrate(d[0] * d[0])
        g_cf = 2.0 * (dH - dt * ud) / (dt * dt * dd)
        rec = s.step(dt)
        assert rec.converged
        # attainable agreement: rounding of H (~1e-16 |H|) divided by r'(gamma)
        rp = dt * ud + rec.gamma * dt * dt * dd - dH
        tol = 20 * 2.2e-16 * abs(rec.H_n) / abs(rp)
        assert abs(rec.gamma - g_cf) < tol
        assert abs(rec.gamma - 1.0) > 100 * tol  # relaxation is active


@pytest.mark.parametrize("assign", ["random", "round_robin"])
@pytest.mark.parametrize("p,E", [(2, [6, 4, 2]), (3, [6, 4, 3]), (4, [8, 6, 5])])
def test_linear_invariants_random_partitions(p, E, assign):
    """Mass, momentum and energy to round-off whatever the partition ids:
    random, or round-robin (neighbouring elements always in different
    partitions), the paper's conservation experiments (Sec. 4.2)."""
    wl = workloads.small_box_2d(n=6, seed=3, R=3, E=E, order=p, random_parts=True)
    if assign == "round_robin":
        wl.part = (np.arange(wl.n_elem) % 3).astype(np.int32)
    s = perrk.Solver(wl)
    m0 = [s.geo.integrate(s.U[v]) for v in range(4)]
    for _ in range(6):
        s.step(wl.dt)
    m1 = [s.geo.integrate(s.U[v]) for v in range(4)]
    for a, b in zip(m0, m1):
        assert abs(a - b) < 1e-13 * (abs(a) + 1.0)


@pytest.mark.parametrize("target", [perrk.TARGET_DELTA_H, perrk.TARGET_PREV, perrk.TARGET_INITIAL])
def test_entropy_conservation_ec(target):
    wl = workloads.small_box_2d(n=6, seed=4, R=2, E=[6, 3], order=3, surface="ec")
    s = perrk.Solver(wl, perrk.NewtonOptions(target=target))
    A = s.abs_entropy(s.U)
    H0 = s.H0
    for _ in range(5):
        rec = s.step(wl.dt * 4)
        assert rec.converged
        assert abs(rec.H_next - rec.H_n) <= 1e-13 * A
    assert abs(s.entropy(s.U) - H0) <= 1e-13 * A
    # without relaxation the same run changes entropy by much more than round-off
    s2 = perrk.Solver(wl, perrk.NewtonOptions(relax=False))
    for _ in range(5):
        rec = s2.step(wl.dt * 4)
    assert abs(s2.entropy(s2.U) - H0) > 1e-11 * A


def test_entropy_stable_es():
    wl = workloads.small_box_2d(n=6, seed=5, R=2, E=[6, 3], order=3, ic="khi")
    s = perrk.Solver(wl)
    for _ in range(4):
        rec = s.step(wl.dt)
        assert rec.dH < 0
        assert rec.H_next - rec.H_n == pytest.approx(rec.gamma * rec.dH, abs=1e-12 * abs(rec.H_n))


@pytest.mark.parametrize("p,E", [(2, [8, 4]), (3, [8, 4]), (4, [8, 5])])
def test_gamma_minus_one_rate(p, E):
    """gamma_n = 1 + O(dt^(p-1)) (Sec. 2.4)."""
    wl = workloads.burgers_1d(E=E)
    dev = []
    for k in range(3):
        s = perrk.Solver(wl, perrk.NewtonOptions(tol_r=0.0, tol_g=1e-10, max_it=30), p=p, E=E)
        rec = s.step((4 if p < 4 else 8) * wl.dt / 2 ** k)
        dev.append(abs(rec.gamma - 1.0))
    rates = [math.log2(dev[i] / dev[i + 1]) for i in range(2)]
    assert min(rates) > (p - 1) - 0.35, (dev, rates)


def _run_to(wl, p, E, dt, n, relax):
    s = perrk.Solver(wl, perrk.NewtonOptions(relax=relax, tol_r=1e-16, tol_g=1e-16), p=p, E=E)
    for _ in range(n):
        s.step(dt)
    return s


@pytest.mark.parametrize("p,E", [(2, [8, 4]), (3, [8, 4]), (4, [8, 5])])
def test_temporal_order(p, E):
    """Observed temporal order p: the relaxed solution at its own final time
    t = sum gamma_n dt against a fine non-relaxed fourth-order reference run
    to that same time on the same mesh."""
    wl = workloads.burgers_1d(E=E)
    T = 0.02
    errs = []
    for k in range(3):
        n = 16 * 2 ** k
        s = _run_to(wl, p, E, T / n, n, relax=True)
        ref = _run_to(wl, 4, [8, 5], s.t / 256, 256, relax=False)
        errs.append(np.abs(s.U - ref.U).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > p - 0.4, (errs, rates)


def test_ssprk3_special_case():
    wl = workloads.small_box_2d(n=4, seed=6, R=1, E=[3], order=3)
    s = perrk.Solver(wl, perrk.NewtonOptions(relax=False))
    U = s.U.copy()
    dt = wl.dt
    F = s.rhs
    u1 = U + dt * F(U)
    u2 = 0.75 * U + 0.25 * (u1 + dt * F(u1))
    u3 = U / 3.0 + 2.0 / 3.0 * (u2 + dt * F(u2))
    s.step(dt)
    assert np.abs(s.U - u3).max() < 1e-13 * np.abs(U).max()


def test_newton_fallback():
    wl = workloads.burgers_1d()
    s = perrk.Solver(wl, perrk.NewtonOptions(max_it=0))
    rec = s.step(wl.dt)
    assert rec.gamma == 1.0 and not rec.converged
    s = perrk.Solver(wl, perrk.NewtonOptions(max_it=1, tol_r=0.0, tol_g=0.0))
    rec = s.step(wl.dt)
    assert rec.gamma == 1.0 and not rec.converged and rec.iters == 1


def _burgers_root_case():
    wl = workloads.burgers_1d()
    s = perrk.Solver(wl)
    U = s.U.copy()
    dt = wl.dt * 2
    d, dH, _ = s.stages(U, dt)
    ud = s.geo.integrate(U[0] * d[0])
    dd = s.geo.integrate(d[0] * d[0])
    g_cf = 2.0 * (dH - dt * ud) / (dt * dt * dd)
    return wl, dt, g_cf


def test_bisection_pass_count_and_bracket():
    """Bisection (Sec. 3.1) on [0.8, 1.2] with only the bracket-length stop:
    2 end evaluations, then k halvings with 0.4 / 2^k <= tol_g, and the root
    within tol_g of the accepted midpoint (closed-form root of the quadratic
    entropy)."""
    wl, dt, g_cf = _burgers_root_case()
    tol_g = 1e-6
    k = math.ceil(math.log2(0.4 / tol_g))
    s = perrk.Solver(wl, perrk.NewtonOptions(solver=perrk.SOLVER_BISECTION, tol_r=0.0, tol_g=tol_g, max_it=60))
    rec = s.step(dt)
    assert rec.converged and rec.iters == 2 + k
    assert abs(rec.gamma - g_cf) <= tol_g
    # bracket without a sign change: no root to bisect, fallback gamma = 1
    s = perrk.Solver(wl, perrk.NewtonOptions(solver=perrk.SOLVER_BISECTION, lo=g_cf + 0.1, hi=g_cf + 0.2))
    rec = s.step(dt)
    assert not rec.converged and rec.gamma == 1.0 and rec.iters == 2


def test_secant_and_newton_reach_the_closed_form_root():
    """Secant from the two guesses 0.8, 1.2 and Newton from 1 converge to the
    closed-form root of the quadratic entropy; the secant takes a handful of
    passes (superlinear), bisection to the same tolerance dozens."""
    wl, dt, g_cf = _burgers_root_case()
    res = {}
    for solver in (perrk.SOLVER_NEWTON, perrk.SOLVER_SECANT, perrk.SOLVER_BISECTION):
        s = perrk.Solver(wl, perrk.NewtonOptions(solver=solver, guess=perrk.GUESS_ONE, tol_r=1e-15, tol_g=1e-13,
                                                 max_it=80))
        rec = s.step(dt)
        assert rec.converged, solver
        res[solver] = rec
    for solver, rec in res.items():
        assert abs(rec.gamma - g_cf) < 1e-9, (solver, rec.gamma, g_cf)
    assert res[perrk.SOLVER_SECANT].iters <= 8
    assert res[perrk.SOLVER_BISECTION].iters > 3 * res[perrk.SOLVER_SECANT].iters


def test_root_finders_agree_euler():
    """Euler (KHI, ES fluxes): the three root finders give the same gamma
    within their tolerances over several steps."""
    wl = workloads.small_box_2d(n=6, seed=7, R=2, E=[6, 3], order=3, ic="khi")
    wl.dt *= 3
    gammas = {}
    for solver in (perrk.SOLVER_NEWTON, perrk.SOLVER_SECANT, perrk.SOLVER_BISECTION):
        s = perrk.Solver(wl, perrk.NewtonOptions(solver=solver, tol_r=1e-15, tol_g=1e-12, max_it=80))
        gammas[solver] = [s.step(wl.dt).gamma for _ in range(3)]
    g0 = np.array(gammas[perrk.SOLVER_NEWTON])
    assert np.all(np.abs(g0 - 1.0) > 1e-9)
    for solver in (perrk.SOLVER_SECANT, perrk.SOLVER_BISECTION):
        assert np.max(np.abs(np.array(gammas[solver]) - g0)) < 1e-8, solver


def test_update_matrix_row_sums_and_conservation():
    """The fully discrete multirate update U_{n+1} = D U_n of a linear problem
    (Sec. 3.2.1): rows of D sum to one and the omega J weighted sum is
    conserved, for the unrelaxed step and for any gamma.  The linear operator
    is the exact Jacobian (complex step) of the two-level Burgers DGSEM at
    u = 1, i.e. linear advection; D comes from the oracle's partitioned stage
    loop applied column by column."""
    wl = workloads.burgers_1d()
    s = perrk.Solver(wl)
    n = wl.u0.size
    one = np.ones_like(wl.u0)
    L = np.empty((n, n))
    h = 1e-30
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1j * h
        L[:, k] = s.rhs(one + e.reshape(one.shape)).ravel().imag / h
    s.rhs = lambda U: (L @ U.ravel()).reshape(U.shape)
    D1 = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        d, _, _ = s.stages(e.reshape(one.shape), wl.dt)
        D1[:, k] = e + wl.dt * d.ravel()
    wJ = s.geo.wJ.ravel()
    for gamma in (1.0, 0.97):
        D = np.eye(n) + gamma * (D1 - np.eye(n))
        assert np.abs(D.sum(axis=1) - 1.0).max() < 1e-12
        assert np.abs(wJ @ D - wJ).max() < 1e-12 * np.abs(wJ).max()
    # the multirate step is not the identity: the fine partition's stages act
    assert np.abs(D1 - np.eye(n)).max() > 1e-3
