"""Optimised stability polynomials for P-ERK families (Sec. 2.2).

A P-ERK member with E stage evaluations and order p has the stability
polynomial P(z) = sum_{k=0}^{E} alpha_k z^k with alpha_k = 1/k! for k <= p;
its E - p remaining coefficients are free (Sec. 2.2).  Given the spectrum of
the semidiscretisation's Jacobian, they are chosen to maximise the step h
with |P(h lambda)| <= 1 on the spectrum (the approach the paper cites:
Ketcheson & Ahmadia 2013):

* for fixed h the coefficients enter P linearly, so feasibility is a convex
  problem; it is solved here by linear programs (scipy's HiGHS): |w| <= 1
  is replaced by the polygon Re(e^{-i theta_k} w) <= 1 over K directions,
  then refined by cutting planes (the tangent Re(e^{-i arg w} w) <= 1 at
  every point where |w| > 1) until |P(h lambda)| <= 1 + 1e-9 at every
  eigenvalue;
* P is written in the Chebyshev basis T_j(1 + 2 z / (h rho)), rho the
  spectral radius, which keeps the program well scaled up to E ~ 16;
* bisection on h.

The polynomial then fixes the member's free tableau entries.  p = 2 (b = e_S):
alpha_j = c_{S-j+2} prod_{m=S-j+3}^{S} a_m, solved from the last row upwards.
p = 3 (b_1 = b_{S-1} = 1/6, b_S = 2/3, a_{S,S-1} = (1 - a_{S-1,S-2}) / 4):
for a trial t = a_{S-1,S-2} the coefficients alpha_4 .. alpha_{E-1} fix the
chain a_{S-2,S-3} .. a_{first+1,first} one at a time, and the last
coefficient alpha_E is a scalar equation in t, solved by bracketing and
bisection.  p = 4: the base stages (the constants of the fourth-order
archetype) fix one coefficient, so the polynomials a chain can reach are not
a linear family; the chain entries a_{i,i-1} (rows first+1 .. S-3) are then
optimised directly (optimised_family_p4): a least-squares fit to the
linear-program optimum, refined by Nelder-Mead on the stable step, kept only
where it beats the default chain.

The spectrum of a context is taken from its own right-hand side through the
C ABI (perrk_rhs), by finite differences column by column.
"""
import math

import numpy as np

__all__ = ["optimal_polynomial", "stable_step", "member_chain", "optimised_tableau", "optimised_family_p4",
           "jacobian", "jacobian_spectrum"]


def _cheb_values(x, deg):
    """T_0..T_deg at complex points x: [len(x), deg + 1]."""
    T = np.empty((len(x), deg + 1), dtype=complex)
    T[:, 0] = 1.0
    if deg >= 1:
        T[:, 1] = x
    for j in range(2, deg + 1):
        T[:, j] = 2.0 * x * T[:, j - 1] - T[:, j - 2]
    return T


def _cheb_derivs_at_one(deg, k):
    """d^k T_j / dx^k at x = 1 for j = 0..deg:  prod_{m<k} (j^2 - m^2) / (2m + 1)."""
    out = np.ones(deg + 1)
    for j in range(deg + 1):
        for m in range(k):
            out[j] *= (j * j - m * m) / (2.0 * m + 1.0)
    return out


def _feasible(z, R, p, E, n_dir, max_rounds=60):
    """Is there a P with the order conditions and |P(z_i)| <= 1 + 1e-9 at the
    scaled spectrum z = h lambda (radius R = h rho)?  Returns the Chebyshev
    coefficients of one, or None."""
    from scipy.optimize import linprog
    x = 1.0 + 2.0 * z / R                          # [-R, 0] -> [-1, 1]
    T = _cheb_values(x, E)
    th = 2.0 * math.pi * np.arange(n_dir) / n_dir
    rows = [(np.exp(-1j * th[k]) * T).real for k in range(n_dir)]
    # P^{(k)}(0) = sum_j gamma_j (2/R)^k T_j^{(k)}(1) = 1 for k <= p, rows times (R/2)^k
    A_eq = np.array([np.append(_cheb_derivs_at_one(E, k), 0.0) for k in range(p + 1)])
    b_eq = np.array([(R / 2.0) ** k for k in range(p + 1)])
    cost = np.zeros(E + 2)
    cost[-1] = 1.0
    for _ in range(max_rounds):
        A_ub = np.concatenate(rows, axis=0)
        A_ub = np.concatenate([A_ub, -np.ones((A_ub.shape[0], 1))], axis=1)
        res = linprog(cost, A_ub=A_ub, b_ub=np.zeros(A_ub.shape[0]), A_eq=A_eq, b_eq=b_eq,
                      bounds=[(None, None)] * (E + 2), method="highs")
        if res.status != 0 or res.x[-1] > 1.0 + 1e-9:
            return None
        gam = res.x[:-1]
        w = T @ gam
        bad = np.abs(w) > 1.0 + 1e-9
        if not bad.any():
            return gam
        rows.append((np.exp(-1j * np.angle(w[bad]))[:, None] * T[bad]).real)
    return None


def _to_monomial(gamma, R):
    """Coefficients alpha_k of P(z) = sum_j gamma_j T_j(1 + 2 z / R)."""
    from numpy.polynomial import Chebyshev, Polynomial
    px = Chebyshev(gamma).convert(kind=Polynomial)
    return (px(Polynomial([1.0, 2.0 / R]))).coef


def stable_step(alpha, lam, h_hi, tol=1e-9, n_grid=4000):
    """Largest h in (0, h_hi] with |P(h lambda)| <= 1 + tol for every lambda of
    the spectrum: a descending scan (stability in h need not be monotone on a
    discrete spectrum), then bisection between the first stable grid point
    and the unstable one above it."""
    lam = _clean_spectrum(lam)
    coef = np.asarray(alpha)[::-1]

    def ok(h):
        return np.abs(np.polyval(coef, h * lam)).max() <= 1.0 + tol

    if ok(h_hi):
        return h_hi
    grid = h_hi * np.arange(n_grid, 0, -1) / n_grid
    for k in range(1, n_grid):
        if ok(grid[k]):
            lo, hi = grid[k], grid[k - 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if ok(mid):
                    lo = mid
                else:
                    hi = mid
            return lo
    return 0.0


def _clean_spectrum(spectrum):
    """Upper half of a conjugate-symmetric spectrum.  Eigenvalues within
    1e-8 rho of the origin are the conserved modes (P(0) = 1 for every P) and
    are dropped; real parts in (0, 1e-8 rho] are rounding of a
    finite-difference Jacobian and are set to 0."""
    lam = np.asarray(spectrum, dtype=complex)
    lam = lam[lam.imag >= 0.0]
    rho = float(np.abs(lam).max()) if lam.size else 0.0
    lam = lam[np.abs(lam) > 1e-8 * rho]
    small = (lam.real > 0.0) & (lam.real <= 1e-8 * rho)
    lam[small] = 1j * lam[small].imag
    return lam


def optimal_polynomial(spectrum, p, E, n_dir=64, rel_tol=1e-4, h_hi=None):
    """(h, alpha): the largest step with |P(h lambda)| <= 1 on the spectrum
    and P's monomial coefficients alpha[0..E] (alpha_k = 1/k! for k <= p)."""
    lam = _clean_spectrum(spectrum)
    if E < p or lam.size == 0:
        raise ValueError("need E >= p and a non-zero spectrum")
    rho = float(np.abs(lam).max())
    hi = h_hi if h_hi else 2.5 * E * E / rho
    lo = 0.0
    best = None
    while hi - lo > rel_tol * hi:
        h = 0.5 * (lo + hi)
        gam = _feasible(lam * h, h * rho, p, E, n_dir)
        if gam is not None:
            lo, best = h, (h, gam)
        else:
            hi = h
    if best is None:
        raise RuntimeError("no stable step found")
    h, gam = best
    alpha = _to_monomial(gam, h * rho)
    alpha = np.concatenate([alpha, np.zeros(E + 1 - len(alpha))])[:E + 1]
    for k in range(p + 1):
        alpha[k] = 1.0 / math.factorial(k)
    return h, alpha


# ------------------------------------------------------------ tableau chain ---

def _chain_p3(c, S, E, alpha, t):
    """a_m (1-based rows) for p = 3 given t = a_{S-1,S-2}: the triangular
    solve of alpha_4 .. alpha_{E-1}; returns (a, residual of alpha_E)."""
    b1, b2 = 1.0 / 6.0, 2.0 / 3.0                  # b_{S-1}, b_S
    a = {S - 1: t, S: (1.0 - t) / 4.0}
    C = lambda i: c[i - 1]
    for j in range(4, E):
        m = S - j + 2
        p2 = math.prod(a[k] for k in range(S - j + 3, S + 1))
        p1 = math.prod(a[k] for k in range(S - j + 3, S))
        a[m] = (alpha[j] - b2 * p2 * C(S - j + 2)) / (b1 * C(S - j + 1) * p1)
    first = S - E + 2
    last = b2 * math.prod(a[k] for k in range(first + 1, S + 1)) * C(first)
    return a, last - alpha[E]


def member_chain(p, c, S, E, alpha):
    """Sub-diagonal entries a_{i,i-1} (dict, 1-based rows) of the member with E
    evaluations whose stability polynomial has the coefficients alpha."""
    first = S - E + 2
    if p == 2:
        a, prod = {}, 1.0
        for j in range(3, E + 1):
            m = S - j + 3
            a[m] = alpha[j] / (c[S - j + 2 - 1] * prod)
            prod *= a[m]
        return a
    if p == 3:
        if E <= 3:
            return {S: 0.25}
        ts = np.linspace(-3.0, 3.0, 6001)
        f = []
        with np.errstate(all="ignore"):
            for t in ts:
                try:
                    f.append(float(_chain_p3(c, S, E, alpha, t)[1]))
                except ZeroDivisionError:
                    f.append(math.nan)
        f = np.array(f)
        roots = []
        for i in range(len(ts) - 1):
            if np.isfinite(f[i]) and np.isfinite(f[i + 1]) and f[i] * f[i + 1] <= 0.0:
                lo, hi = ts[i], ts[i + 1]
                flo = f[i]
                for _ in range(200):
                    mid = 0.5 * (lo + hi)
                    fm = _chain_p3(c, S, E, alpha, mid)[1]
                    if (fm <= 0.0) == (flo <= 0.0):
                        lo, flo = mid, fm
                    else:
                        hi = mid
                roots.append(0.5 * (lo + hi))
        if not roots:
            raise RuntimeError("no p = 3 chain reproduces this polynomial")
        # the root nearest the default a_{S-1,S-2} = 1/4
        t = min(roots, key=lambda r: abs(r - 0.25))
        return _chain_p3(c, S, E, alpha, t)[0]
    raise NotImplementedError("p = 4: the chain is optimised directly (optimised_family_p4)")


def optimised_tableau(p, E_list, alphas):
    """(c, b, a1, asub) of the family with each member's stability polynomial
    alphas[r]; shared c and b come from the library's builder."""
    from . import perrk_build_tableau
    c, b, a1, asub = perrk_build_tableau(p, E_list)
    S = len(c)
    for r, E in enumerate(E_list):
        first = S - E + 2
        a = member_chain(p, c, S, E, np.asarray(alphas[r], dtype=float))
        for i in range(3, S + 1):                  # rows 1 and 2 keep (0) and (c_2)
            v = a.get(i, 0.0) if i > first else 0.0
            asub[r, i - 1] = v
            a1[r, i - 1] = c[i - 1] - v
    return c, b, a1, asub


def _full_matrix(c, a1, asub, r):
    S = len(c)
    A = np.zeros((S, S))
    for i in range(1, S):
        A[i, 0] += a1[r, i]
        A[i, i - 1] += asub[r, i]
    return A


def _poly_of(b, A, E):
    """alpha_0..alpha_E of the member (alpha_j = b^T A^{j-1} 1)."""
    out = [1.0]
    v = np.ones(len(b))
    for _ in range(E):
        out.append(float(b @ v))
        v = A @ v
    return np.array(out)


def optimised_family_p4(spectrum, E_list, n_dir=32, max_eval=400):
    """(c, b, a1, asub, steps) of a p = 4 family whose members' free chain
    entries maximise the stable step on the spectrum; steps[r] is member r's
    stable step (>= the default chain's)."""
    from scipy.optimize import least_squares, minimize
    from . import perrk_build_tableau
    lam = _clean_spectrum(spectrum)
    c, b, a1, asub = perrk_build_tableau(4, E_list)
    S = len(c)
    steps = []
    for r, E in enumerate(E_list):
        first = S - E + 2
        rows = list(range(first + 1, S - 2))           # free rows (1-based); rows S-2 .. S are the base
        a_def = np.array([asub[r, i - 1] for i in rows])

        def set_chain(x):
            for i, v in zip(rows, x):
                asub[r, i - 1] = v
                a1[r, i - 1] = c[i - 1] - v

        def step_of(x, hi):
            set_chain(x)
            return stable_step(_poly_of(b, _full_matrix(c, a1, asub, r), E), lam, hi)

        h_lp, alpha_lp = optimal_polynomial(lam, 4, E, n_dir=n_dir, rel_tol=1e-3)
        h_def = step_of(a_def, 2.0 * h_lp)
        best_x, best_h = a_def, h_def
        if rows:
            def fit(x):
                set_chain(x)
                al = _poly_of(b, _full_matrix(c, a1, asub, r), E)
                return (al[5:] - alpha_lp[5:]) / np.abs(alpha_lp[5:]).clip(1e-300)
            x0 = least_squares(fit, a_def, xtol=1e-14, ftol=1e-14).x
            h0 = step_of(x0, 2.0 * h_lp)
            if h0 > best_h:
                best_x, best_h = x0, h0
            res = minimize(lambda x: -step_of(x, 2.0 * h_lp), best_x, method="Nelder-Mead",
                           options={"maxfev": max_eval, "xatol": 1e-8, "fatol": 1e-6 * best_h})
            if -res.fun > best_h:
                best_x, best_h = res.x, -res.fun
        set_chain(best_x)
        steps.append(best_h)
    return c, b, a1, asub, steps


def jacobian(solver, u=None, eps=1e-7):
    """dF/dU at the state u (default: the solver's state) from the library's
    right-hand side (perrk_rhs), one forward-difference column per degree of
    freedom (SoA order [V][n_elem][NP]); for the small meshes the optimiser is
    run on."""
    import torch
    from . import perrk_rhs
    u0 = solver.state() if u is None else np.asarray(u, dtype=np.float64)
    n = u0.size
    ud = torch.tensor(u0, device="cuda")
    f0 = torch.empty_like(ud)
    perrk_rhs(solver.h, ud.data_ptr(), f0.data_ptr())
    J = np.empty((n, n))
    step = eps * max(1.0, float(np.abs(u0).max()))
    flat = ud.view(-1)
    fk = torch.empty_like(ud)
    for k in range(n):
        old = float(flat[k])
        flat[k] = old + step
        perrk_rhs(solver.h, ud.data_ptr(), fk.data_ptr())
        flat[k] = old
        J[:, k] = ((fk - f0).view(-1) / step).cpu().numpy()
    return J


def jacobian_spectrum(solver, u=None, eps=1e-7):
    """Eigenvalues of dF/dU (see jacobian)."""
    return np.linalg.eigvals(jacobian(solver, u, eps))
