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


def lagrange_matrix(xn, s):
    """L[i, j] = l_j(s_i): the Lagrange basis of the nodes xn evaluated at the
    points s (barycentric form, extended precision)."""
    xn = np.asarray(xn, dtype=np.longdouble)
    s = np.asarray(s, dtype=np.longdouble)
    n = len(xn)
    lam = np.array([1 / np.prod([xn[j] - xn[k] for k in range(n) if k != j]) for j in range(n)])
    L = np.zeros((len(s), n), dtype=np.longdouble)
    for i, si in enumerate(s):
        hit = np.nonzero(si == xn)[0]
        if len(hit):
            L[i, hit[0]] = 1
            continue
        t = lam / (si - xn)
        L[i] = t / t.sum()
    return L.astype(np.float64)


def mortar_operators(N=3):
    """Operators of the L2 projection mortar method (Kopriva 1996), the
    non-conforming interface treatment the paper runs with its adaptive
    meshes (Sec. 4.2 notes that it is not entropy-conservative).  A coarse
    face s in [-1, 1] is split at s = 0 into two mortars m = 0 (lower half)
    and m = 1 (upper half), each matching one fine face s' in [-1, 1] with
    s = (s' - 1)/2 or (s' + 1)/2:
      P[m][i, j] = l_j(s_m(x_i))      coarse face polynomial at the mortar's LGL nodes
      R[m] = M^-1 P[m]^T M            L2 projection of a mortar polynomial back to the
                                      coarse face, M_ij = int l_i l_j exact (Gauss-Legendre)
    A flux g_m on each mortar (with the fine face's scaled normal) gives the
    coarse face's flux G = R[0] g_0 + R[1] g_1 (with the coarse face's
    normal: the factor 1/2 of ds = ds'/2 cancels the halved face length)."""
    x, w, _ = _lgl.lgl(N)
    gx, gw = np.polynomial.legendre.leggauss(N + 1)          # exact for degree 2N + 1
    Lg = lagrange_matrix(x, gx)
    M = Lg.T @ (gw[:, None] * Lg)
    P = [lagrange_matrix(x, 0.5 * (x - 1.0)), lagrange_matrix(x, 0.5 * (x + 1.0))]
    R = [np.linalg.solve(M, Pm.T @ M) for Pm in P]
    return P, R


class Geometry:
    def __init__(self, coords, faces, N=3, mortars=None):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.n_elem, self.NP, self.dim = self.coords.shape
        self.N = N
        self.x, self.w, self.D = _lgl.lgl(N)
        self.faces = np.asarray(faces)
        # 2:1 non-conforming interfaces, rows (coarse element, its face, fine
        # element on the lower half, fine element on the upper half)
        self.mortars = np.zeros((0, 4), dtype=np.int64) if mortars is None else np.asarray(mortars, dtype=np.int64)
        if len(self.mortars):
            self.P_mortar, self.R_mortar = mortar_operators(N)
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
    if len(geo.mortars):
        _mortar_terms(geo, phys, Ut, acc)
    K = -geo.flat(acc) / geo.J[None]
    if getattr(phys, "viscous", False):
        if len(geo.mortars):
            raise NotImplementedError("viscous terms on non-conforming meshes")
        K = K + viscous_rhs(geo, phys, U)
    return K


def _mortar_terms(geo, phys, Ut, acc):
    """Surface terms of the 2:1 mortars (see mortar_operators).  For each
    mortar m the coarse face state is interpolated to the mortar nodes,
    the numerical flux g_m = f*(U_plus, U_minus; nu_m) is evaluated with the
    '+' side first and the fine face's scaled normal nu_m, the fine element
    takes g_m like a conforming face, and the coarse element takes the L2
    projection G = sum_m R[m] g_m (with its own normal in f(U_q).nu)."""
    N = geo.N
    P, R = geo.P_mortar, geo.R_mortar
    ec, fc, elo, ehi = (geo.mortars[:, c] for c in range(4))
    for f in range(2 * geo.dim):
        sel = fc == f
        if not np.any(sel):
            continue
        k, cplus = f >> 1, f & 1
        ic, jf = (N, 0) if cplus else (0, N)           # coarse face index, fine face index along xi^k
        ax = Ut.ndim - 1 - k
        Uk = np.moveaxis(Ut, ax, -1)                   # [V, E, t, n]: face nodes t in tangential order
        Jak = np.moveaxis(geo.tens(geo.Ja[k]), ax, -1)
        accm = np.moveaxis(acc, ax, -1)
        e_c = ec[sel]
        uC = Uk[..., ic][:, e_c]                       # [V, nm, N+1]
        nu_c = Jak[..., ic][:, e_c]
        G = 0.0
        for m, e_f in enumerate((elo[sel], ehi[sel])):
            uF = Uk[..., jf][:, e_f]
            nu_m = Jak[..., jf][:, e_f]
            uCm = np.einsum("ij,vmj->vmi", P[m], uC)
            g = phys.surface_flux(uCm, uF, nu_m) if cplus else phys.surface_flux(uF, uCm, nu_m)
            G = G + np.einsum("ij,vmj->vmi", R[m], g)
            if cplus:                                  # fine element on the '-' side
                np.add.at(accm[..., jf], (slice(None), e_f), (-g + phys.flux(uF, nu_m)) / geo.w[0])
            else:
                np.add.at(accm[..., jf], (slice(None), e_f), (g - phys.flux(uF, nu_m)) / geo.w[N])
        if cplus:
            np.add.at(accm[..., ic], (slice(None), e_c), (G - phys.flux(uC, nu_c)) / geo.w[N])
        else:
            np.add.at(accm[..., ic], (slice(None), e_c), (-G + phys.flux(uC, nu_c)) / geo.w[0])


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
