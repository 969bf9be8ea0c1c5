"""Flux-differencing DGSEM on conforming quad/hex meshes (oracle, float64).

The paper evaluates its semidiscretisation U' = F(U) (eq. SemidiscretizationODE)
with the DGSEM on LGL nodes, an entropy-conservative two-point volume flux
via flux differencing with SBP operators, and an EC or ES (LLF-dissipative)
surface flux (Sec. 2.1, Sec. 4.1).  Written out for one element with
reference coordinates xi^k, nodal metric terms Ja^k and Jacobian J:

  J_q dU_q/dt = - sum_k sum_m 2 D_{q m} f#(U_q, U_m; (Ja^k_q + Ja^k_m)/2)   (m along the xi^k line of q)
                - sum_{faces at q} (1/omega_face) ( f*(U^-, U^+; nu) - f(U_q).nu )

where nu is the element's outward scaled normal (+-Ja^k at the face node) and
omega_face the LGL weight of the face node's index across the face.  Metric
terms: 1D Ja = 1, J = x_xi; 2D Ja^1 = (y_eta, -x_eta), Ja^2 = (-y_xi, x_xi),
J = x_xi y_eta - x_eta y_xi, derivatives by D (this satisfies the discrete
metric identities); 3D cross-product form Ja^1 = x_eta x x_zeta etc. (exact
for affine elements, the only 3D elements used here).

An interface's flux is evaluated once, with the normal of its '+' side (the
row's left element), and enters both elements with opposite signs.
"""
import math

import numpy as np

from . import lgl as _lgl


class Geometry:
    def __init__(self, coords, faces, N=3):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.n_elem, self.NP, self.dim = self.coords.shape
        self.N = N
        self.x, self.w, self.D = _lgl.lgl(N)
        self.faces = np.asarray(faces)
        self.shape_nodes = (N + 1,) * self.dim          # (k, j, i) order reversed below
        self._metrics()

    def tens(self, a):
        """[..., n_elem, NP] -> [..., n_elem, (k), (j), i]  (i fastest)."""
        return a.reshape(a.shape[:-1] + (self.N + 1,) * self.dim)

    def flat(self, a):
        return a.reshape(a.shape[:-self.dim] + (self.NP,))

    def dxi(self, a, k):
        """Derivative along reference direction k (0 = xi, 1 = eta, 2 = zeta) of a
        nodal field a[..., n_elem, NP]."""
        t = self.tens(a)
        ax = t.ndim - 1 - k
        t = np.moveaxis(t, ax, -1)
        t = np.einsum("qm,...m->...q", self.D, t)
        t = np.moveaxis(t, -1, ax)
        return self.flat(t)

    def _metrics(self):
        X = np.moveaxis(self.coords, 2, 0)             # [dim, n_elem, NP]
        d = self.dim
        dX = [self.dxi(X, k) for k in range(d)]         # dX[k][comp] = d x_comp / d xi^k
        if d == 1:
            self.J = dX[0][0]
            self.Ja = np.ones((1, 1) + self.J.shape)
        elif d == 2:
            xx, xy = dX[0][0], dX[1][0]
            yx, yy = dX[0][1], dX[1][1]
            self.J = xx * yy - xy * yx
            self.Ja = np.array([[yy, -xy], [-yx, xx]])  # Ja[k][comp]
        else:
            a, b, c = dX[0], dX[1], dX[2]
            self.Ja = np.array([np.cross(b, c, axis=0), np.cross(c, a, axis=0), np.cross(a, b, axis=0)])
            self.J = np.sum(a * self.Ja[0], axis=0)
        wn = self.w
        if d == 1:
            wq = wn
        elif d == 2:
            wq = np.outer(wn, wn).ravel()               # index j*4 + i -> w_j w_i
        else:
            wq = np.einsum("k,j,i->kji", wn, wn, wn).ravel()
        self.wq = wq                                    # quadrature weight per node
        self.wJ = wq[None, :] * self.J                  # [n_elem, NP]

    def integrate(self, f):
        """sum_e sum_q omega_q J_q f_q  for a nodal scalar f[n_elem, NP],
        summed exactly rounded (math.fsum): the relaxation root gamma is
        conditioned by 1/r'(gamma) = O(dt^-2), so the entropy sums must carry
        no summation-order error."""
        return math.fsum((self.wJ * f).ravel().tolist())


def rhs(geo, phys, U):
    """dU/dt = F(U) on all elements; U[V, n_elem, NP] -> K[V, n_elem, NP]."""
    d, N = geo.dim, geo.N
    V = U.shape[0]
    Ut = geo.tens(U)                                   # [V, E, (k),(j), i]
    acc = np.zeros_like(Ut)
    # ---- volume: flux differencing along each reference direction
    for k in range(d):
        ax = Ut.ndim - 1 - k
        Uk = np.moveaxis(Ut, ax, -1)                   # [V, E, ..., 4]
        Jak = np.moveaxis(geo.tens(geo.Ja[k]), ax, -1)  # [dim, E, ..., 4]
        nav = 0.5 * (Jak[..., :, None] + Jak[..., None, :])
        F = phys.volume_flux(Uk[..., :, None], Uk[..., None, :], nav)   # [V, E, ..., q, m]
        vol = 2.0 * np.einsum("qm,...qm->...q", geo.D, F)
        acc += np.moveaxis(vol, -1, ax)
    # ---- surface: each listed interface once, normal of the '+' side
    eL, fL, eR, fR = (geo.faces[:, c] for c in range(4))
    for k in range(d):
        sel = fL == 2 * k + 1
        if not np.any(sel):
            continue
        el, er = eL[sel], eR[sel]
        ax = Ut.ndim - 1 - k
        Uk = np.moveaxis(Ut, ax, -1)
        Jak = np.moveaxis(geo.tens(geo.Ja[k]), ax, -1)
        uL = Uk[..., N][:, el]                         # [V, nf, face nodes...]
        uR = Uk[..., 0][:, er]
        nu = Jak[..., N][:, el]                        # outward normal of the '+' side
        fs = phys.surface_flux(uL, uR, nu)
        # acc holds -J dU/dt, so the surface term enters with a + sign
        cL = (fs - phys.flux(uL, nu)) / geo.w[N]
        cR = (-fs + phys.flux(uR, nu)) / geo.w[0]
        accm = np.moveaxis(acc, ax, -1)                # view
        np.add.at(accm[..., N], (slice(None), el), cL)
        np.add.at(accm[..., 0], (slice(None), er), cR)
    K = -geo.flat(acc) / geo.J[None]
    if getattr(phys, "viscous", False):
        K = K + viscous_rhs(geo, phys, U)
    return K


# ----------------------------------------------------------------------------
# Parabolic part: BR1 (Bassi & Rebay 1997; Gassner, Winters, Hindenlang &
# Kopriva 2018), the viscous discretisation of the paper's viscous test
# (Sec. 4.3.2), with the gradients taken of the entropy variables.
#
# Gradient (one element, strong form, central trace W* = (W^- + W^+)/2):
#   J_q q_l(q) = sum_k Ja^k_l(q) sum_m D_{qm} W(m along xi^k)
#                + sum_{faces at q} (1/omega_face) (W* - W_q) nu_l
# Divergence of the viscous flux (central flux f_v* = (f_v^- + f_v^+)/2):
#   J_q (div f_v)_q = sum_k sum_m D_{qm} (sum_l Ja^k_l f_v,l)(m along xi^k)
#                + sum_{faces at q} (1/omega_face) (f_v* - f_v(q)) . nu
# with nu the element's outward scaled normal; the viscous contribution to
# the right-hand side is + div f_v.  Both face terms use the '+' side's
# normal for the two elements of an interface, like the inviscid part.
# ----------------------------------------------------------------------------

def _interfaces(geo, k):
    eL, fL, eR = geo.faces[:, 0], geo.faces[:, 1], geo.faces[:, 2]
    sel = fL == 2 * k + 1
    return eL[sel], eR[sel]


def br1_gradient(geo, W):
    """q[l, V, n_elem, NP] ~ d W / d x_l for a nodal field W[V, n_elem, NP]."""
    d, N = geo.dim, geo.N
    Wt = geo.tens(W)
    JQ = np.zeros((d,) + Wt.shape)
    for k in range(d):
        dW = geo.tens(geo.dxi(W, k))
        Jak = geo.tens(geo.Ja[k])
        for l in range(d):
            JQ[l] += Jak[l][None] * dW
    for k in range(d):
        el, er = _interfaces(geo, k)
        if el.size == 0:
            continue
        ax = Wt.ndim - 1 - k
        Wk = np.moveaxis(Wt, ax, -1)
        wL, wR = Wk[..., N][:, el], Wk[..., 0][:, er]
        nu = np.moveaxis(geo.tens(geo.Ja[k]), ax, -1)[..., N][:, el]
        half = 0.5 * (wR - wL)          # W* - W_L;  W* - W_R = -half
        for l in range(d):
            Ql = np.moveaxis(JQ[l], ax, -1)
            # left element, outward normal +nu;  right element, outward -nu
            np.add.at(Ql[..., N], (slice(None), el), half * nu[l][None] / geo.w[N])
            np.add.at(Ql[..., 0], (slice(None), er), (-half) * (-nu[l][None]) / geo.w[0])
    return geo.flat(JQ) / geo.J[None, None]


def br1_divergence(geo, Fv):
    """(div f_v)[V, n_elem, NP] for a nodal flux Fv[l, V, n_elem, NP]."""
    d, N = geo.dim, geo.N
    acc = np.zeros(geo.tens(Fv[0]).shape)
    for k in range(d):
        Fk = sum(geo.Ja[k][l][None] * Fv[l] for l in range(d))    # contravariant component k
        acc += geo.tens(geo.dxi(Fk, k))
    for k in range(d):
        el, er = _interfaces(geo, k)
        if el.size == 0:
            continue
        ax = acc.ndim - 1 - k
        nu = np.moveaxis(geo.tens(geo.Ja[k]), ax, -1)[..., N][:, el]
        fnL = 0.0
        fnR = 0.0
        for l in range(d):
            Fl = np.moveaxis(geo.tens(Fv[l]), ax, -1)
            fnL = fnL + Fl[..., N][:, el] * nu[l][None]
            fnR = fnR + Fl[..., 0][:, er] * nu[l][None]
        half = 0.5 * (fnR - fnL)
        accm = np.moveaxis(acc, ax, -1)
        # left: (f* - f_L) . nu = half;  right: (f* - f_R) . (-nu) = half
        np.add.at(accm[..., N], (slice(None), el), half / geo.w[N])
        np.add.at(accm[..., 0], (slice(None), er), half / geo.w[0])
    return geo.flat(acc) / geo.J[None]


def viscous_rhs(geo, phys, U):
    """+ div f_v(U, grad w) with the BR1 gradient of the entropy variables."""
    Q = br1_gradient(geo, phys.entropy_vars(U))
    return br1_divergence(geo, phys.viscous_flux(U, Q))
