"""Pins of the oracle's LGL tables and fluxes against closed forms and identities."""
import math

import numpy as np

from oracle import lgl, physics
import workloads


def test_lgl_closed_form_n3():
    x, w, D = lgl.lgl(3)
    s5 = 1.0 / math.sqrt(5.0)
    assert np.allclose(x, [-1, -s5, s5, 1], atol=1e-15, rtol=0)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15, rtol=0)
    assert np.allclose(workloads.REF_NODES, x, atol=1e-15, rtol=0)


def test_sbp_property_and_exactness():
    for N in (2, 3, 4, 5):
        x, w, D = lgl.lgl(N)
        Q = np.diag(w) @ D
        B = np.zeros((N + 1, N + 1))
        B[0, 0], B[-1, -1] = -1.0, 1.0
        assert np.abs(Q + Q.T - B).max() < 1e-13
        for k in range(N + 1):
            assert np.abs(D @ x ** k - (k * x ** (k - 1) if k else 0 * x)).max() < 1e-12
        # quadrature exact up to degree 2N - 1
        for k in range(2 * N):
            exact = (1 - (-1) ** (k + 1)) / (k + 1)
            assert abs(w @ x ** k - exact) < 1e-13
        # and not beyond the polynomial degree for D
        assert np.abs(D @ x ** (N + 1) - (N + 1) * x ** N).max() > 1e-6


def _random_euler_states(rng, n, dim):
    rho = rng.uniform(0.3, 3.0, n)
    v = rng.uniform(-2.0, 2.0, (dim, n))
    p = rng.uniform(0.2, 5.0, n)
    return workloads.prim_to_cons(rho, v, p)


def test_ln_mean_accuracy():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 10.0, 2000)
    for rel in (1e-14, 1e-10, 1e-6, 1e-3, 1e-1, 0.9):
        y = x * (1.0 + rel * rng.uniform(-1, 1, x.size))
        xl, yl = x.astype(np.longdouble), y.astype(np.longdouble)
        # independent reference: ln_mean = (x + y) f / (2 atanh f), f = (y - x)/(y + x);
        # atanh(f)/f = sum_k f^(2k)/(2k+1) for |f| < 0.2, the log form otherwise
        f = (yl - xl) / (yl + xl)
        ser = np.zeros_like(f)
        term = np.ones_like(f)
        for k in range(60):
            ser += term / (2 * k + 1)
            term = term * f * f
        with np.errstate(all="ignore"):
            ref = np.where(np.abs(f) < 0.2, (xl + yl) / (2 * ser), (yl - xl) / np.log(yl / xl))
        got = physics.ln_mean(x, y)
        if np.finfo(np.longdouble).eps < 1e-17:
            assert np.max(np.abs(got - ref) / ref) < 5e-15
        assert np.all(np.abs(got - np.sqrt(x * y)) <= np.abs(0.5 * (x + y) - np.sqrt(x * y)) + 1e-15 * x)
    assert physics.ln_mean(2.0, 2.0) == 2.0


def test_entropy_variables_complex_step():
    rng = np.random.default_rng(2)
    for dim in (1, 2, 3):
        u = _random_euler_states(rng, 50, dim)
        w = physics.euler_entropy_vars(u, 1.4)
        h = 1e-30
        for k in range(dim + 2):
            uc = u.astype(complex)
            uc[k] += 1j * h
            rho = uc[0]
            v = uc[1:1 + dim] / rho
            p = 0.4 * (uc[-1] - 0.5 * rho * np.sum(v * v, axis=0))
            s = -rho * (np.log(p) - 1.4 * np.log(rho))
            assert np.max(np.abs(s.imag / h - w[k]) / (1 + np.abs(w[k]))) < 1e-13


def test_euler_flux_consistency_symmetry_tadmor():
    rng = np.random.default_rng(3)
    g = 1.4
    for dim in (1, 2, 3):
        n_pairs = 10000
        ul = _random_euler_states(rng, n_pairs, dim)
        ur = _random_euler_states(rng, n_pairs, dim)
        n = rng.standard_normal((dim, n_pairs))
        f = physics.euler_ranocha(ul, ur, n, g)
        assert np.abs(physics.euler_ranocha(ul, ul, n, g) - physics.euler_flux(ul, n, g)).max() < 1e-12 * (1 + np.abs(f).max())
        assert np.abs(physics.euler_ranocha(ur, ul, n, g) - f).max() == 0.0 or \
            np.abs(physics.euler_ranocha(ur, ul, n, g) - f).max() < 1e-13 * np.abs(f).max()
        assert np.abs(physics.euler_ranocha(ur, ul, -n, g) + f).max() < 1e-13 * np.abs(f).max()
        wl = physics.euler_entropy_vars(ul, g)
        wr = physics.euler_entropy_vars(ur, g)
        lhs = np.sum((wr - wl) * f, axis=0)
        rhs = physics.euler_entropy_potential(ur, n, g) - physics.euler_entropy_potential(ul, n, g)
        scale = np.sum(np.abs(wr - wl) * np.abs(f), axis=0) + 1.0
        assert np.max(np.abs(lhs - rhs) / scale) < 1e-13
        # the potential really is w.f - s v.n for this entropy
        psi = np.sum(wl * physics.euler_flux(ul, n, g), axis=0) - physics.euler_entropy(ul, g) * np.sum(
            ul[1:1 + dim] / ul[0] * n, axis=0)
        assert np.max(np.abs(psi - physics.euler_entropy_potential(ul, n, g)) / (1 + np.abs(psi))) < 1e-12
        # ES flux dissipates entropy: (w_R - w_L).(f_es - f_ec) <= 0
        fes = physics.euler_es(ul, ur, n, g)
        assert np.all(np.sum((wr - wl) * (fes - f), axis=0) <= 1e-12 * scale)
        # KEP structure: momentum flux = f_rho * avg(v) + avg(p) n
        vl, vr = ul[1:1 + dim] / ul[0], ur[1:1 + dim] / ur[0]
        pl = physics.euler_prims(ul, g)[2]
        pr = physics.euler_prims(ur, g)[2]
        assert np.abs(f[1:1 + dim] - f[0] * 0.5 * (vl + vr) - 0.5 * (pl + pr) * n).max() < 1e-12 * np.abs(f).max()


def test_burgers_flux_tadmor():
    rng = np.random.default_rng(4)
    a = rng.uniform(-3, 3, 10000)[None]
    b = rng.uniform(-3, 3, 10000)[None]
    n = np.ones((1, 10000))
    f = physics.burgers_ec(a, b, n)
    assert np.abs((b - a) * f - (b ** 3 - a ** 3) / 6.0).max() < 1e-13
    assert np.abs(physics.burgers_ec(a, a, n) - physics.burgers_flux(a, n)).max() < 1e-14
    fes = physics.burgers_es(a, b, n)
    assert np.all((b - a) * (fes - f) <= 1e-14)
