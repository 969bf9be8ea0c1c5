"""Pins of the oracle's wave-speed bound in the entropy-stable surface flux.

The ES interface flux is the EC flux minus local Lax-Friedrichs (Rusanov)
dissipation 1/2 lambda_max (u+ - u-) (Sec. 2.1), with lambda_max the largest
characteristic speed of the two traces in the direction of the scaled normal
(Sec. 2.2, eq. CharSpeed_DG).  The characteristic speeds in direction n are
the eigenvalues of the flux Jacobian d(f(u).n)/du, so lambda_max must equal
the spectral radius of that Jacobian, maximised over both traces.  Here the
Jacobian is formed by complex-step differentiation of the physical flux,
written out in this file from the conservation law, and its eigenvalues come
from numpy's general eigensolver; nothing of the oracle's speed formula is
reused.  Normals are random and NOT of unit length, so a bound that drops
|n| on the sound speed, or takes it on the wrong term, fails.  Three planted
mistakes check that the pin catches what it must.
"""
import numpy as np
import pytest

from oracle import physics
import workloads

GAMMA = 1.4


def _flux_dot_n(u, n, gamma):
    """f(u).n of the Euler equations for one state u[V] and direction n[dim]:
    (rho v.n, rho v v.n + p n, (rho E + p) v.n), p = (gamma-1)(rho E - rho|v|^2/2)."""
    dim = len(n)
    rho, m, E = u[0], u[1:1 + dim], u[-1]
    v = m / rho
    p = (gamma - 1.0) * (E - 0.5 * np.dot(m, v))
    vn = np.dot(v, n)
    return np.concatenate([[rho * vn], m * vn + p * n, [(E + p) * vn]])


def _spectral_radius(u, n, gamma):
    V = len(u)
    J = np.empty((V, V))
    h = 1e-30
    for k in range(V):
        uc = u.astype(complex)
        uc[k] += 1j * h
        J[:, k] = _flux_dot_n(uc, n.astype(complex), gamma).imag / h
    return float(np.max(np.abs(np.linalg.eigvals(J))))


def _random_pairs(rng, n_pairs, dim):
    def states():
        rho = rng.uniform(0.2, 4.0, n_pairs)
        v = rng.uniform(-3.0, 3.0, (dim, n_pairs))
        p = rng.uniform(0.1, 6.0, n_pairs)
        return workloads.prim_to_cons(rho, v, p)
    nrm = rng.standard_normal((dim, n_pairs)) * rng.uniform(0.05, 20.0, n_pairs)   # non-unit normals
    return states(), states(), nrm


def _max_speed_error(max_speed, dim, seed=11, n_pairs=300):
    rng = np.random.default_rng(seed + dim)
    ul, ur, nrm = _random_pairs(rng, n_pairs, dim)
    got = max_speed(ul, ur, nrm, GAMMA)
    worst = 0.0
    for i in range(n_pairs):
        ref = max(_spectral_radius(ul[:, i], nrm[:, i], GAMMA), _spectral_radius(ur[:, i], nrm[:, i], GAMMA))
        worst = max(worst, abs(got[i] - ref) / ref)
    return worst


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_max_speed_is_the_jacobian_spectral_radius(dim):
    assert _max_speed_error(physics.euler_max_speed, dim) < 1e-10


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_es_dissipation_uses_that_speed(dim):
    """f_es - f_ec = -1/2 lambda_max (u_R - u_L), lambda_max from the spectrum."""
    rng = np.random.default_rng(20 + dim)
    ul, ur, nrm = _random_pairs(rng, 200, dim)
    diss = physics.euler_es(ul, ur, nrm, GAMMA) - physics.euler_ranocha(ul, ur, nrm, GAMMA)
    for i in range(200):
        lam = max(_spectral_radius(ul[:, i], nrm[:, i], GAMMA), _spectral_radius(ur[:, i], nrm[:, i], GAMMA))
        ref = -0.5 * lam * (ur[:, i] - ul[:, i])
        assert np.abs(diss[:, i] - ref).max() <= 1e-10 * (np.abs(ref).max() + 1e-300)


def test_burgers_es_dissipation_uses_the_characteristic_speed():
    """Burgers: d(u^2/2 n)/du = u n, so lambda_max = max(|u_L|, |u_R|) |n|."""
    rng = np.random.default_rng(31)
    a = rng.uniform(-3, 3, 5000)[None]
    b = rng.uniform(-3, 3, 5000)[None]
    for scale in (0.1, 1.0, 7.5, -2.0):
        n = np.full((1, 5000), scale)
        h = 1e-30
        speed = lambda u: np.abs((0.5 * (u + 1j * h) ** 2 * n[0]).imag / h)   # |f'(u) n|
        lam = np.maximum(speed(a[0]), speed(b[0]))
        diss = physics.burgers_es(a, b, n) - physics.burgers_ec(a, b, n)
        assert np.abs(diss[0] + 0.5 * lam * (b[0] - a[0])).max() < 1e-13


# --------------------------------------------------------- planted mistakes

def _speed_without_norm_on_c(ul, ur, n, gamma):
    """Mistake: the sound speed is not scaled by |n|."""
    rl, vl, pl = physics.euler_prims(ul, gamma)
    rr, vr, pr = physics.euler_prims(ur, gamma)
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    return np.maximum(np.abs(np.sum(vl * n, axis=0)) + cl, np.abs(np.sum(vr * n, axis=0)) + cr)


def _speed_min_over_sides(ul, ur, n, gamma):
    """Mistake: the smaller of the two sides' speeds."""
    rl, vl, pl = physics.euler_prims(ul, gamma)
    rr, vr, pr = physics.euler_prims(ur, gamma)
    nn = np.sqrt(np.sum(n * n, axis=0))
    return np.minimum(np.abs(np.sum(vl * n, axis=0)) + np.sqrt(gamma * pl / rl) * nn,
                      np.abs(np.sum(vr * n, axis=0)) + np.sqrt(gamma * pr / rr) * nn)


def _speed_signed_vn(ul, ur, n, gamma):
    """Mistake: v.n without its absolute value."""
    rl, vl, pl = physics.euler_prims(ul, gamma)
    rr, vr, pr = physics.euler_prims(ur, gamma)
    nn = np.sqrt(np.sum(n * n, axis=0))
    return np.maximum(np.sum(vl * n, axis=0) + np.sqrt(gamma * pl / rl) * nn,
                      np.sum(vr * n, axis=0) + np.sqrt(gamma * pr / rr) * nn)


@pytest.mark.parametrize("mutant", [_speed_without_norm_on_c, _speed_min_over_sides, _speed_signed_vn])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_planted_wave_speed_mistakes_fail_the_pin(mutant, dim):
    assert _max_speed_error(mutant, dim) > 1e-3
