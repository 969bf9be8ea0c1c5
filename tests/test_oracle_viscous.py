"""Pins of the oracle's Navier-Stokes-Fourier part (BR1 on entropy-variable
gradients): the paper's traveling viscous shock (Sec. 4.3.2, eq.
ViscousShockSolution) as an exact solution of the full semidiscrete
right-hand side, frame indifference and Stokes' hypothesis of the stress,
polynomial exactness of the BR1 gradient and divergence, conservation, the
discrete entropy identity of BR1 and the temporal order of the relaxed
stage loop with viscosity."""
import math

import numpy as np
import pytest

import workloads
from oracle import dgsem, perrk, physics


def _rhs_error(n, angle):
    wl = workloads.viscous_shock_2d(n=n, angle=angle)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    ph = physics.Physics("euler2d", "es_rusanov", wl.gamma_gas, wl.mu, wl.prandtl)
    K = dgsem.rhs(geo, ph, wl.u0)
    nrm = wl.info["normal"]
    s = wl.coords[:, :, 0] * nrm[0] + wl.coords[:, :, 1] * nrm[1]
    h = 1e-30
    rho, un, p = workloads.viscous_shock_prims(s + 1j * h, wl.gamma_gas, wl.mu)
    U = workloads.prim_to_cons(rho, un[None] * nrm[:, None, None], p, wl.gamma_gas)
    dUds = U.imag / h
    exact = -1.0 * dUds                     # U(x, t) = U0(x.n - v t), v = 1
    inner = np.abs(wl.coords).max(axis=(1, 2)) <= 1.0 + 1e-12   # two element rings away from the seams
    return np.abs(K - exact)[:, inner].max(), np.abs(exact).max()


@pytest.mark.parametrize("angle", [0.0, 0.6])
def test_viscous_shock_is_a_discrete_solution(angle):
    """dU/dt of the traveling profile is -v dU/ds: the semidiscrete RHS on
    the exact profile converges to it at the DGSEM's order.  Rotating the
    shock normal exercises every stress component."""
    errs = [_rhs_error(n, angle) for n in (16, 32, 64)]
    rates = [math.log2(errs[i][0] / errs[i + 1][0]) for i in range(2)]
    assert min(rates) > 2.6, (errs, rates)
    assert errs[-1][0] < 1e-3 * errs[-1][1]


def _gw_complex_step(prims, x, gamma, dim):
    """Exact gradients d w / d x_l of the entropy variables of a state given
    as a function of position, by complex steps."""
    h = 1e-30
    out = []
    for l in range(dim):
        xc = x.astype(complex)
        xc[l] = xc[l] + 1j * h
        rho, v, p = prims(xc)
        u = workloads.prim_to_cons(rho, v, p, gamma)
        out.append(physics.euler_entropy_vars(u, gamma).imag / h)
    rho, v, p = prims(x)
    return workloads.prim_to_cons(rho, v, p, gamma), np.array(out)


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_flux_frame_indifference(dim):
    """Rigid rotation plus translation at uniform temperature: no viscous
    stress, no heat flux (the stress depends on the symmetric part of the
    velocity gradient only)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (dim, 50))
    W = rng.standard_normal((dim, dim))
    Om = W - W.T
    b = rng.standard_normal(dim)
    T0 = 1.7

    def prims(y):
        rho = 1.0 + 0.3 * np.sin(y[0] + 2 * y[1])
        v = Om @ y + b[:, None]
        return rho, v, rho * T0

    u, gw = _gw_complex_step(prims, x, 1.4, dim)
    fv = physics.nsf_viscous_flux(u, gw, 1.4, 0.3, 0.72)
    assert np.abs(fv).max() < 1e-12


def test_viscous_stress_traceless_3d():
    """Stokes' hypothesis (zero bulk viscosity): a uniform isotropic
    dilatation at uniform temperature carries no viscous stress in 3D."""
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (3, 40))
    x0 = rng.standard_normal(3)

    def prims(y):
        rho = 1.0 + 0.2 * np.cos(y[2] - y[0])
        return rho, 0.8 * (y - x0[:, None]), rho * 2.0

    u, gw = _gw_complex_step(prims, x, 1.4, 3)
    fv = physics.nsf_viscous_flux(u, gw, 1.4, 0.5, 0.72)
    assert np.abs(fv).max() < 1e-12


def _interior(wl):
    """Elements none of whose faces is a periodic seam (where the two sides'
    face nodes are at different positions)."""
    dim = wl.coords.shape[2]
    q = np.arange(4 ** dim)
    idx = [q % 4, (q // 4) % 4, q // 16]
    ok = np.ones(wl.coords.shape[0], bool)
    for eL, fL, eR, fR in wl.faces:
        k = fL // 2
        xL = wl.coords[eL][idx[k] == 3].mean(axis=0)
        xR = wl.coords[eR][idx[k] == 0].mean(axis=0)
        if np.abs(xL - xR).max() > 1e-9:
            ok[eL] = ok[eR] = False
    return ok


@pytest.mark.parametrize("case", ["box2d", "curved2d", "box3d"])
def test_br1_gradient_polynomial_exactness(case):
    """Away from the periodic seams (where the field jumps) a field that is
    continuous and of degree <= N in the reference coordinates has an exact
    BR1 gradient: cubics on affine elements, linear fields on the curved
    (degree-3 mapped) elements."""
    if case == "box2d":
        wl = workloads.small_box_2d(n=6)
    elif case == "curved2d":
        wl = workloads.vortex_2d(n=8)
    else:
        wl = workloads.tgv_3d(n=4, n_fine=2)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    X = np.moveaxis(wl.coords, 2, 0)
    d = geo.dim
    if case == "curved2d":
        W = np.array([0.3 * X[0] - 1.1 * X[1] + 2.0, 0.7 * X[1]])
        grad = [np.array([0.3 + 0 * X[0], 0 * X[0]]), np.array([-1.1 + 0 * X[0], 0.7 + 0 * X[0]])]
    else:
        W = np.array([X[0] ** 3 - 2 * X[0] * X[1] ** 2 + X[d - 1], X[1] ** 2 * X[0]])
        gx = [3 * X[0] ** 2 - 2 * X[1] ** 2 + (1.0 if d == 1 else 0.0), X[1] ** 2]
        gy = [-4 * X[0] * X[1] + (1.0 if d == 2 else 0.0), 2 * X[1] * X[0]]
        grad = [np.array(gx), np.array(gy)]
        if d == 3:
            grad.append(np.array([1.0 + 0 * X[0], 0 * X[0]]))
    Q = dgsem.br1_gradient(geo, W)
    inner = _interior(wl)
    assert inner.sum() > 0
    scale = np.abs(W).max() + 1.0
    for l in range(d):
        assert np.abs(Q[l][:, inner] - grad[l][:, inner]).max() < 1e-11 * scale, l


def test_br1_divergence_polynomial_exactness():
    wl = workloads.small_box_2d(n=6)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    x, y = wl.coords[:, :, 0], wl.coords[:, :, 1]
    Fv = np.array([[x ** 3 * y, x * y], [y ** 2 - x ** 2 * y ** 3, x + y ** 3]])   # Fv[l][component]
    exact = np.array([3 * x ** 2 * y + 2 * y - 3 * x ** 2 * y ** 2, y + 3 * y ** 2])
    div = dgsem.br1_divergence(geo, Fv)
    inner = _interior(wl)
    assert np.abs(div[:, inner] - exact[:, inner]).max() < 1e-10 * np.abs(exact).max()


VISC_CASES = [
    ("box2d", lambda: workloads.small_box_2d(n=6, seed=2, mu=0.05)),
    ("curved2d", lambda: workloads.vortex_2d(n=10)),
    ("box3d", lambda: workloads.tgv_3d(n=4, n_fine=2, mu=0.02)),
]


@pytest.mark.parametrize("name,make", VISC_CASES)
def test_viscous_conservation_and_entropy_identity(name, make):
    """Periodic meshes: sum omega J F_v = 0 for every variable, and the BR1
    summation-by-parts identity sum omega J w . F_v = - sum omega J q . f_v
    (central traces make the interface terms cancel), which is <= 0 because
    q . f_v(u, q) is a positive semidefinite quadratic form in q."""
    wl = make()
    rng = np.random.default_rng(9)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    ph = physics.Physics(wl.equation, "ec", wl.gamma_gas, 0.05, 0.72)
    u = wl.u0 * (1.0 + 0.03 * rng.standard_normal(wl.u0.shape))
    Fv = dgsem.viscous_rhs(geo, ph, u)
    w = ph.entropy_vars(u)
    Q = dgsem.br1_gradient(geo, w)
    fv = ph.viscous_flux(u, Q)
    scale = geo.integrate(np.sum(np.abs(Fv), axis=0)) + 1e-300
    for v in range(Fv.shape[0]):
        assert abs(geo.integrate(Fv[v])) < 1e-12 * scale, v
    lhs = geo.integrate(np.sum(w * Fv, axis=0))
    dissip = geo.integrate(np.sum(Q * fv, axis=(0, 1)))
    assert abs(lhs + dissip) < 1e-11 * abs(dissip)
    assert lhs < 0.0
    # a constant state carries no viscous flux
    assert np.abs(dgsem.viscous_rhs(geo, ph, np.ones_like(u) * u[:, :1, :1])).max() < 1e-12


def _run(wl, p, E, dt, n, relax):
    s = perrk.Solver(wl, perrk.NewtonOptions(relax=relax, tol_r=1e-16, tol_g=1e-16), p=p, E=E)
    for _ in range(n):
        s.step(dt)
    return s


@pytest.mark.parametrize("p,E", [(2, [6, 3]), (3, [6, 3]), (4, [6, 5])])
def test_temporal_order_with_viscosity(p, E):
    """The relaxed multirate scheme keeps its order p on the Navier-Stokes-
    Fourier semidiscretisation (the paper's claim for entropy-diffusive
    problems, Sec. 4.3.2), by self-convergence against a fine non-relaxed
    fourth-order run to the relaxed run's own final time."""
    wl = workloads.small_box_2d(n=4, seed=8, R=2, E=E, order=p, mu=0.2)
    T = 0.4
    errs = []
    for k in range(3):
        n = 8 * 2 ** k
        s = _run(wl, p, E, T / n, n, relax=True)
        ref = _run(wl, 4, [6, 5], s.t / 128, 128, relax=False)
        errs.append(np.abs(s.U - ref.U).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > p - 0.4, (errs, rates)
