"""Optimised stability polynomials (Sec. 2.2) and the tableaux they fix.

Optimiser pins: the shifted Chebyshev polynomial's real stability interval
2 s^2 (first order, textbook), the unique second-order two-stage and
third-order three-stage polynomials (real intervals 2 and 2.5127...), and
|P(h lambda)| <= 1 on the spectrum at the returned step.  Map pins: the
library's tableau (from a polynomial) reproduces that polynomial when its
full Butcher matrix is expanded by the oracle, keeps the order conditions of
every member pair, and equals the oracle's independently built member."""
import math

import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
from paper_2507_04991_gb300 import stability as st
from oracle import tableau as T


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return pk.load()


REAL = -np.linspace(0.0, 1.0, 401)[1:]


@pytest.mark.parametrize("s", [4, 8])
def test_chebyshev_real_interval(s):
    h, alpha = st.optimal_polynomial(REAL, 1, s)
    assert abs(h / (2 * s * s) - 1.0) < 2e-3
    # the optimum is T_s(1 + z / s^2): its leading coefficient is 2^{s-1} / s^{2s}
    assert abs(alpha[s] * s ** (2 * s) / 2 ** (s - 1) - 1.0) < 2e-2


def test_fixed_polynomials():
    h2, a2 = st.optimal_polynomial(REAL, 2, 2)
    assert abs(h2 - 2.0) < 1e-3 and np.allclose(a2, [1, 1, 0.5])
    h3, _ = st.optimal_polynomial(REAL, 3, 3)
    # real root of |1 + z + z^2/2 + z^3/6| = 1 left of 0: z^3 + 3 z^2 + 6 z + 12 = 0
    r = np.roots([1, 3, 6, 12])
    zr = float(r[np.abs(r.imag) < 1e-12].real[0])
    assert abs(h3 + zr) < 1e-3 * abs(zr)


SPEC = np.concatenate([-0.2 * np.linspace(0, 1, 150)[1:] + 1j * np.linspace(0, 1, 150)[1:],
                       -0.1 + 1j * np.linspace(0, 1, 40), -np.linspace(0, 1, 40)[1:]])


@pytest.mark.parametrize("p,E", [(2, 6), (3, 8)])
def test_optimised_step_is_stable_and_beats_default(p, E):
    h, alpha = st.optimal_polynomial(SPEC, p, E)
    assert np.abs(np.polyval(alpha[::-1], h * SPEC)).max() <= 1.0 + 1e-8
    assert all(abs(alpha[k] - 1.0 / math.factorial(k)) < 1e-15 for k in range(p + 1))
    # the default member of the same E on the same spectrum
    S = E
    A = T.member(p, S, E)
    a_def = T.stability_coeffs(T.weights(p, S), A)[:E + 1]
    h_def = st.stable_step(a_def, SPEC, 2.0 * h)
    assert h > 1.05 * h_def, (h, h_def)


def _chain_alphas(p, E_list, seed):
    """Stability polynomials of members with seeded random chains near the
    defaults, expanded by the oracle (an input for both builders)."""
    rng = np.random.default_rng(seed)
    S = max(E_list)
    c, b = T.abscissae(p, S), T.weights(p, S)
    out = []
    for E in E_list:
        A = T.member(p, S, E)
        first = S - E + 2
        for m in range(first + 1, S + 1):
            if A[m - 1, m - 2] != 0.0 and not (p == 3 and m == S):
                a = A[m - 1, m - 2] * (1.0 + 0.2 * rng.uniform(-1, 1))
                A[m - 1, m - 2] = a
                A[m - 1, 0] = c[m - 1] - a
        if p == 3 and E > 3:
            t = A[S - 2, S - 3]
            A[S - 1, S - 2] = (1.0 - t) / 4.0
            A[S - 1, 0] = c[S - 1] - A[S - 1, S - 2]
        out.append(T.stability_coeffs(b, A)[:E + 1])
    return out


def _full(c, a1, asub, r):
    S = len(c)
    A = np.zeros((S, S))
    for i in range(1, S):
        A[i, 0] += a1[r, i]
        A[i, i - 1] += asub[r, i]
    return A


@pytest.mark.parametrize("p,E_list", [(2, [8, 4]), (2, [6, 4, 3]), (3, [8, 5, 3]), (3, [10, 6, 4])])
def test_tableau_from_polynomial(lib, p, E_list):
    alphas = _chain_alphas(p, E_list, 7 + len(E_list))
    c, b, a1, asub = st.optimised_tableau(p, E_list, alphas)
    As = [_full(c, a1, asub, r) for r in range(len(E_list))]
    for r, E in enumerate(E_list):
        al = T.stability_coeffs(b, As[r])
        # the chain solve divides by products of chain entries: the top
        # coefficients carry ~1e-9 relative rounding
        assert np.allclose(al[:E + 1], alphas[r], rtol=1e-7, atol=0.0), r
        assert np.all(al[E + 1:] == 0.0)
    worst, cons = T.order_residuals(c, b, As, p)
    assert worst < 1e-13 and cons < 1e-15
    oc, ob, oAs = T.family_from_poly(p, E_list, alphas)
    assert np.abs(oc - c).max() < 1e-15 and np.abs(ob - b).max() == 0.0
    for r in range(len(E_list)):
        assert np.abs(oAs[r] - As[r]).max() < 1e-8, r


def test_optimised_family_is_valid(lib):
    """A whole family optimised on one spectrum: every member stable at its
    own step, the steps grow with E, order conditions hold."""
    E_list = [8, 5, 3]
    hs, alphas = zip(*[st.optimal_polynomial(SPEC, 3, E) for E in E_list])
    assert hs[0] > hs[1] > hs[2]
    c, b, a1, asub = st.optimised_tableau(3, E_list, alphas)
    As = [_full(c, a1, asub, r) for r in range(3)]
    assert T.order_residuals(c, b, As, 3)[0] < 1e-13
    for r, E in enumerate(E_list):
        al = T.stability_coeffs(b, As[r])[:E + 1]
        assert np.abs(np.polyval(al[::-1], hs[r] * SPEC)).max() <= 1.0 + 1e-7


def test_gain_on_a_dg_spectrum():
    """The spectrum of the oracle's DGSEM Jacobian (free stream, Ranocha EC
    volume and Rusanov ES surface fluxes, 4 x 4 periodic boxes): the
    optimised p = 3, E = 8 polynomial is stable there at a step well above the
    default member's."""
    import workloads
    from oracle import dgsem, physics
    wl = workloads.small_box_2d(n=4, seed=51, R=1, E=[8], order=3)
    u = np.empty_like(wl.u0)
    u[0], u[1], u[2] = 1.0, 0.5, 0.3
    u[3] = 1.0 / 0.4 + 0.5 * (0.25 + 0.09)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    ph = physics.Physics(wl.equation, wl.surface_flux, wl.gamma_gas)
    f0 = dgsem.rhs(geo, ph, u).ravel()
    step = 1e-7 * np.abs(u).max()
    J = np.empty((u.size, u.size))
    for k in range(u.size):
        du = u.copy().ravel()
        du[k] += step
        J[:, k] = (dgsem.rhs(geo, ph, du.reshape(u.shape)).ravel() - f0) / step
    lam = np.linalg.eigvals(J)
    h, alpha = st.optimal_polynomial(lam, 3, 8, n_dir=32, rel_tol=1e-3)
    a_def = T.stability_coeffs(T.weights(3, 8), T.member(3, 8, 8))[:9]
    h_def = st.stable_step(a_def, lam, 2.0 * h)
    assert h > 2.0 * h_def, (h, h_def)
    assert st.stable_step(alpha, lam, h) == h


def test_p4_family_optimised_on_its_chain():
    """p = 4: the chain entries are optimised directly.  The family keeps the
    fourth-order conditions of every member pair (checked by the oracle on
    the full Butcher matrices), each member is stable at its reported step,
    and the member with free entries gains over the default chain."""
    E_list = [7, 5]
    c, b, a1, asub, steps = st.optimised_family_p4(SPEC, E_list, max_eval=150)
    As = [_full(c, a1, asub, r) for r in range(len(E_list))]
    worst, cons = T.order_residuals(c, b, As, 4)
    assert worst < 1e-13 and cons < 1e-15
    for r, E in enumerate(E_list):
        al = T.stability_coeffs(b, As[r])[:E + 1]
        assert np.abs(np.polyval(al[::-1], steps[r] * SPEC)).max() <= 1.0 + 1e-8
        a_def = T.stability_coeffs(T.weights(4, max(E_list)), T.member(4, max(E_list), E))[:E + 1]
        h_def = st.stable_step(a_def, SPEC, 3.0 * steps[r])
        assert steps[r] >= h_def * (1.0 - 1e-12)
    assert steps[0] > 1.1 * st.stable_step(T.stability_coeffs(T.weights(4, 7), T.member(4, 7, 7))[:8], SPEC, 10.0)


def test_p4_chain_is_refused():
    """p = 4's base stages fix one coefficient: no chain reproduces an
    arbitrary polynomial (its chain is optimised directly instead)."""
    c = T.abscissae(4, 8)
    with pytest.raises(NotImplementedError):
        st.member_chain(4, c, 8, 8, np.ones(9))
    with pytest.raises(NotImplementedError):
        T.member_from_poly(4, 8, 8, np.ones(9))


def test_state_copy_modes(lib):
    assert (pk.STATE_HOST, pk.STATE_DEVICE, pk.STATE_HOST_ASYNC) == (0, 1, 2)
    for bad in (3, -1):
        with pytest.raises(ValueError):
            pk._state_mode(bad)
