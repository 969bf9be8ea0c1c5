"""Fluxes, two-point fluxes and entropy functions (oracle, float64).

States are arrays u[V, ...]; directions n[dim, ...] are NOT normalised: a
flux "in direction n" is f(u) . n, and the numerical fluxes are linear (EC
part) or positively homogeneous (dissipation) in n, so that an interface flux
times the face length is f*(u-, u+; nu) with nu the scaled normal.

Burgers (1D, V = 1): f = u^2/2, entropy s = u^2/2, entropy variable w = u,
EC two-point flux (a^2 + a b + b^2)/6.

Euler (d = 1, 2, 3; V = d + 2; ideal gas): the paper's entropy
s(u) = -rho log(p rho^-gamma) (eq. EntropyMathematical) and w = ds/du
(eq. EntropyVariables); EC and kinetic-energy preserving two-point flux of
Ranocha (2018/2020) built from logarithmic means; Rusanov / local
Lax-Friedrichs dissipation -1/2 lambda_max (u+ - u-) with
lambda_max = max(|v.n| + c |n|) over both states (Sec. 2.2, ref. for LLF).
"""
import numpy as np


# ---------------------------------------------------------------- Burgers ---

def burgers_flux(u, n):
    return 0.5 * u * u * n[0]


def burgers_ec(ul, ur, n):
    return (ul * ul + ul * ur + ur * ur) / 6.0 * n[0]


def burgers_es(ul, ur, n):
    lam = np.maximum(np.abs(ul), np.abs(ur)) * np.abs(n[0])
    return burgers_ec(ul, ur, n) - 0.5 * lam * (ur - ul)


def burgers_entropy(u):
    return 0.5 * u[0] * u[0]


def burgers_entropy_vars(u):
    return u.copy()


# ------------------------------------------------------------------ Euler ---

def ln_mean(x, y):
    """Logarithmic mean (y - x) / (log y - log x), = x when x == y.  Evaluated
    as (y - x) / log1p((y - x) / x), which keeps full relative accuracy when
    x and y are close (y - x is then exact)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = y - x
    same = d == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        out = d / np.log1p(d / x)
    return np.where(same, x, out)


def euler_prims(u, gamma):
    rho = u[0]
    dim = u.shape[0] - 2
    v = u[1:1 + dim] / rho
    p = (gamma - 1.0) * (u[-1] - 0.5 * rho * np.sum(v * v, axis=0))
    return rho, v, p


def euler_flux(u, n, gamma):
    rho, v, p = euler_prims(u, gamma)
    vn = np.sum(v * n, axis=0)
    out = np.empty_like(u)
    out[0] = rho * vn
    out[1:-1] = u[1:-1] * vn + p * n
    out[-1] = (u[-1] + p) * vn
    return out


def euler_ranocha(ul, ur, n, gamma):
    """Ranocha's EC/KEP flux in direction n:
    f_rho = ln(rho) * avg(v.n); f_m = f_rho avg(v) + avg(p) n;
    f_E = f_rho (v_L.v_R / 2 + 1 / ((gamma-1) ln(rho/p))) + (p_L v_R.n + p_R v_L.n) / 2."""
    rl, vl, pl = euler_prims(ul, gamma)
    rr, vr, pr = euler_prims(ur, gamma)
    vnl = np.sum(vl * n, axis=0)
    vnr = np.sum(vr * n, axis=0)
    rho_ln = ln_mean(rl, rr)
    beta_ln = ln_mean(rl / pl, rr / pr)
    f = np.empty(np.broadcast(ul, ur).shape)
    f[0] = rho_ln * 0.5 * (vnl + vnr)
    f[1:-1] = f[0] * 0.5 * (vl + vr) + 0.5 * (pl + pr) * n
    f[-1] = f[0] * (0.5 * np.sum(vl * vr, axis=0) + 1.0 / ((gamma - 1.0) * beta_ln)) \
        + 0.5 * (pl * vnr + pr * vnl)
    return f


def euler_max_speed(ul, ur, n, gamma):
    rl, vl, pl = euler_prims(ul, gamma)
    rr, vr, pr = euler_prims(ur, gamma)
    nn = np.sqrt(np.sum(n * n, axis=0))
    cl = np.sqrt(gamma * pl / rl)
    cr = np.sqrt(gamma * pr / rr)
    return np.maximum(np.abs(np.sum(vl * n, axis=0)) + cl * nn, np.abs(np.sum(vr * n, axis=0)) + cr * nn)


def euler_es(ul, ur, n, gamma):
    lam = euler_max_speed(ul, ur, n, gamma)
    return euler_ranocha(ul, ur, n, gamma) - 0.5 * lam * (ur - ul)


def euler_entropy(u, gamma):
    """s(u) = -rho (log p - gamma log rho)   (eq. EntropyMathematical)."""
    rho, v, p = euler_prims(u, gamma)
    return -rho * (np.log(p) - gamma * np.log(rho))


def euler_entropy_vars(u, gamma):
    """w = ds/du = (gamma - S - (gamma-1) rho|v|^2/(2p), (gamma-1) rho v / p, -(gamma-1) rho / p),
    S = log p - gamma log rho."""
    rho, v, p = euler_prims(u, gamma)
    S = np.log(p) - gamma * np.log(rho)
    w = np.empty_like(u)
    w[0] = gamma - S - (gamma - 1.0) * rho * np.sum(v * v, axis=0) / (2.0 * p)
    w[1:-1] = (gamma - 1.0) * rho * v / p
    w[-1] = -(gamma - 1.0) * rho / p
    return w


def euler_entropy_potential(u, n, gamma):
    """psi = w . f(u).n - F(u).n with entropy flux F = s v; for this entropy
    psi = (gamma - 1) rho v.n (used by the Tadmor-condition pin)."""
    rho, v, p = euler_prims(u, gamma)
    return (gamma - 1.0) * rho * np.sum(v * n, axis=0)


# ------------------------------------------------- Navier-Stokes-Fourier ---

def nsf_viscous_flux(u, gw, gamma, mu, prandtl):
    """Viscous flux of the compressible Navier-Stokes-Fourier equations (the
    parabolic part of the paper's viscous test, Sec. 4.3.2: constant dynamic
    viscosity mu, Stokes' hypothesis, Fourier heat conduction with Prandtl
    number Pr = c_p mu / kappa, c_p = gamma / (gamma - 1), gas constant 1 so
    T = p / rho).

    The gradients come as gw[l] = d w / d x_l of the entropy variables of the
    paper's entropy (eq. EntropyVariables).  With w_m = (gamma-1) v / T and
    w_E = -(gamma-1) / T the primitive gradients follow by the chain rule:
        d T = (gamma-1) d w_E / w_E^2,      d v = -(d w_m + v d w_E) / w_E.
    Stress tau = mu (grad v + grad v^T) - 2/3 mu (div v) I, heat flux
    -kappa grad T.  Returns fv[l] = (0, tau[l, :], tau[l, :] . v + kappa d_l T)."""
    dim = u.shape[0] - 2
    rho, v, p = euler_prims(u, gamma)
    T = p / rho
    wE = -(gamma - 1.0) / T
    dT = np.array([(gamma - 1.0) * gw[l][-1] / (wE * wE) for l in range(dim)])
    dv = np.array([[-(gw[l][1 + a] + v[a] * gw[l][-1]) / wE for a in range(dim)] for l in range(dim)])  # dv[l][a] = d v_a / d x_l
    div = sum(dv[a][a] for a in range(dim))
    kappa = mu * gamma / ((gamma - 1.0) * prandtl)
    fv = np.zeros((dim,) + u.shape)
    for l in range(dim):
        for a in range(dim):
            tau = mu * (dv[l][a] + dv[a][l]) - (2.0 / 3.0) * mu * div * (1.0 if a == l else 0.0)
            fv[l][1 + a] = tau
            fv[l][-1] += tau * v[a]
        fv[l][-1] += kappa * dT[l]
    return fv


# ------------------------------------------------------------- dispatch ---

class Physics:
    """Bundle of the functions one equation needs."""

    def __init__(self, equation, surface="ec", gamma=1.4, mu=0.0, prandtl=0.75):
        self.equation = equation
        self.gamma = gamma
        self.surface = surface
        self.mu = mu
        self.prandtl = prandtl
        if equation == "burgers1d":
            self.dim, self.nvar = 1, 1
        else:
            self.dim = {"euler1d": 1, "euler2d": 2, "euler3d": 3}[equation]
            self.nvar = self.dim + 2

    def flux(self, u, n):
        if self.equation == "burgers1d":
            return burgers_flux(u, n)
        return euler_flux(u, n, self.gamma)

    def volume_flux(self, ul, ur, n):
        if self.equation == "burgers1d":
            return burgers_ec(ul, ur, n)
        return euler_ranocha(ul, ur, n, self.gamma)

    def surface_flux(self, ul, ur, n):
        if self.equation == "burgers1d":
            return burgers_ec(ul, ur, n) if self.surface == "ec" else burgers_es(ul, ur, n)
        if self.surface == "ec":
            return euler_ranocha(ul, ur, n, self.gamma)
        return euler_es(ul, ur, n, self.gamma)

    def entropy(self, u):
        if self.equation == "burgers1d":
            return burgers_entropy(u)
        return euler_entropy(u, self.gamma)

    def entropy_vars(self, u):
        if self.equation == "burgers1d":
            return burgers_entropy_vars(u)
        return euler_entropy_vars(u, self.gamma)

    @property
    def viscous(self):
        return self.mu > 0.0 and self.equation != "burgers1d"

    def viscous_flux(self, u, gw):
        return nsf_viscous_flux(u, gw, self.gamma, self.mu, self.prandtl)
