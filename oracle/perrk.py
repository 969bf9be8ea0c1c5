"""P-ERRK time stepping, written as the paper states it (oracle, float64).

Stage loop: eq. PartitionedRKSystem in full Butcher form.  For an element of
partition r,
    U_{n,i} = U_n + dt sum_{j<i} A^(r)_{ij} K_j ,   K_i = F(U_{n,i})
(F evaluated everywhere; only the rows of A^(r) decide which K_j matter, so
this equals evaluating F^(r) on its own index set), and
    d_n = sum_i b_i K_i                                     (Sec. 3).
Entropy change (eq. EntropyChange_EntropyVariables_ReArranged):
    Delta H = dt sum_i b_i sum_e sum_q omega_q J_q < w(U_{n,i,q}), K_{i,q} >.
Relaxation (eq. RelaxationEquation and its derivative, Sec. 3.1):
    r(g)  = H(U_n + g dt d) - H_target(g),
    r'(g) = < w(U_n + g dt d), dt d >_M - dH_target/dg,
with H_target = H_n + g Delta H (eq. EntropyConservationRRKM_Short), = H_n
(entropy kept from step to step, Sec. 4.1.1) or = H(U_0) (Sec. 4.1.2).
Newton-Raphson with unit step from the guess (gamma_{n-1}, 1 at the first
step); stop on |r| <= tol_r * A_n (A_n = sum omega J |s(U_n)|; the Newton
correction that pass yields is still applied, which costs no pass and makes
gamma insensitive to rounding at the threshold), on |dgamma| <= tol_g or
after max_it passes; if it did not stop by one of the
two tolerances, or gamma is not in (0.5, 1.5), take gamma = 1 (Sec. 3.2,
fallback of Sec. 3.2.1).  Relaxed update (eq. RRKM_Update):
U_{n+1} = U_n + gamma dt d, t_{n+1} = t_n + gamma dt.

The two other root finders the paper considers (Sec. 3.1), one evaluation of
r per full-state pass:
  bisection: r at the bracket ends [lo, hi] (Sec. 4.3.2 takes [0.8, 1.2]),
  which must differ in sign, then at midpoints, keeping the half whose ends
  differ in sign; stop on |r(mid)| <= tol_r A_n or a bracket of length
  <= tol_g (take that midpoint) or after max_it passes;
  secant: the two initial guesses lo and hi, then
  g_{k+1} = g_k - r_k (g_k - g_{k-1}) / (r_k - r_{k-1}); stop on
  |r_k| <= tol_r A_n or |g_{k+1} - g_k| <= tol_g (take g_k) or after max_it.
Both take an evaluated point, so H_{n+1} is that evaluation; the same
fallback applies.
"""
import dataclasses

import numpy as np

from . import dgsem, physics, tableau

GUESS_ONE, GUESS_PREV = "one", "prev"
SOLVER_NEWTON, SOLVER_BISECTION, SOLVER_SECANT = "newton", "bisection", "secant"
TARGET_DELTA_H, TARGET_PREV, TARGET_INITIAL = "delta_h", "prev", "initial"


@dataclasses.dataclass
class NewtonOptions:
    max_it: int = 10
    tol_r: float = 1e-14
    tol_g: float = 1e-14
    guess: str = GUESS_PREV
    target: str = TARGET_DELTA_H
    relax: bool = True
    solver: str = SOLVER_NEWTON
    lo: float = 0.8          # bisection bracket / secant initial guesses
    hi: float = 1.2


@dataclasses.dataclass
class StepRecord:
    gamma: float
    iters: int
    converged: bool
    H_n: float
    dH: float
    H_next: float
    t: float
    stage_dot: list          # per stage with b_i != 0: sum omega J <w, K_i>


class Solver:
    def __init__(self, wl, opts=None, p=None, E=None, alphas=None):
        self.wl = wl
        self.phys = physics.Physics(wl.equation, wl.surface_flux, wl.gamma_gas, getattr(wl, "mu", 0.0),
                                    getattr(wl, "prandtl", 0.75))
        self.geo = dgsem.Geometry(wl.coords, wl.faces, mortars=getattr(wl, "mortars", None))
        self.p = p or wl.order
        self.E = list(E or wl.E)
        if alphas is None:
            self.c, self.b, self.As = tableau.family(self.p, self.E)
        else:                      # members with the given stability polynomials
            self.c, self.b, self.As = tableau.family_from_poly(self.p, self.E, alphas)
        self.S = len(self.b)
        self.part = np.asarray(wl.part)
        self.opts = opts or NewtonOptions()
        self.U = wl.u0.copy()
        self.t = 0.0
        self.gamma_prev = 1.0
        self.H0 = self.entropy(self.U)

    # ---- functionals
    def entropy(self, U):
        return self.geo.integrate(self.phys.entropy(U))

    def abs_entropy(self, U):
        return self.geo.integrate(np.abs(self.phys.entropy(U)))

    def dot_w(self, U, K):
        return self.geo.integrate(np.sum(self.phys.entropy_vars(U) * K, axis=0))

    def rhs(self, U):
        return dgsem.rhs(self.geo, self.phys, U)

    # ---- one step
    def stages(self, U, dt):
        """Returns (d, Delta H, per-stage integrals) from the full Butcher stage loop."""
        S = self.S
        K = []
        dH = 0.0
        stage_dot = []
        A_e = np.stack([self.As[r] for r in self.part])        # [n_elem, S, S]
        for i in range(S):
            Ui = U.copy()
            for j in range(i):
                Ui += dt * A_e[None, :, i, j, None] * K[j]
            Ki = self.rhs(Ui)
            K.append(Ki)
            if self.b[i] != 0.0:
                s = self.dot_w(Ui, Ki)
                stage_dot.append(s)
                dH += self.b[i] * s
        d = sum(self.b[i] * K[i] for i in range(S) if self.b[i] != 0.0)
        return d, dt * dH, stage_dot

    def newton(self, U, d, dt, H_n, A_n, dH, guess):
        o = self.opts
        if o.target == TARGET_DELTA_H:
            tgt = lambda g: H_n + g * dH
            dtgt = dH
        elif o.target == TARGET_PREV:
            tgt = lambda g: H_n
            dtgt = 0.0
        else:
            tgt = lambda g: self.H0
            dtgt = 0.0
        if o.solver == SOLVER_BISECTION:
            return self._bisection(U, d, dt, A_n, tgt)
        if o.solver == SOLVER_SECANT:
            return self._secant(U, d, dt, A_n, tgt)
        g = guess
        converged = False
        it = 0
        while it < o.max_it:
            Ug = U + g * dt * d
            r = self.entropy(Ug) - tgt(g)
            rp = self.dot_w(Ug, dt * d) - dtgt
            it += 1
            if abs(r) <= o.tol_r * A_n:
                # residual small enough: no further pass, but the correction
                # this pass already yields is applied (Sec. 3.1 reading)
                if np.isfinite(r) and np.isfinite(rp) and rp != 0.0:
                    g = g - r / rp
                converged = True
                break
            if not np.isfinite(r) or not np.isfinite(rp) or rp == 0.0:
                break
            dg = -r / rp
            g = g + dg
            if abs(dg) <= o.tol_g:
                converged = True
                break
        if not converged or not np.isfinite(g) or not (0.5 < g < 1.5):
            return 1.0, it, False
        return g, it, True

    def _residual(self, U, d, dt, tgt, g):
        return self.entropy(U + g * dt * d) - tgt(g)

    @staticmethod
    def _accept(g, converged, it):
        if not converged or not np.isfinite(g) or not (0.5 < g < 1.5):
            return 1.0, it, False
        return g, it, True

    def _bisection(self, U, d, dt, A_n, tgt):
        o = self.opts
        lo, hi = o.lo, o.hi
        it = 0
        r_lo = r_hi = None
        while it < o.max_it:
            if r_lo is None:
                g = lo
            elif r_hi is None:
                g = hi
            else:
                g = 0.5 * (lo + hi)
            r = self._residual(U, d, dt, tgt, g)
            it += 1
            if not np.isfinite(r):
                return self._accept(g, False, it)
            if abs(r) <= o.tol_r * A_n:
                return self._accept(g, True, it)
            if r_lo is None:
                r_lo = r
            elif r_hi is None:
                r_hi = r
                if not (r_lo * r_hi < 0.0):        # no sign change: no bracketed root
                    return self._accept(g, False, it)
            else:
                if r * r_lo < 0.0:
                    hi, r_hi = g, r
                else:
                    lo, r_lo = g, r
                if hi - lo <= o.tol_g:
                    return self._accept(g, True, it)
        return self._accept(lo, False, it)

    def _secant(self, U, d, dt, A_n, tgt):
        o = self.opts
        g_prev, r_prev = None, None
        g = o.lo
        it = 0
        while it < o.max_it:
            r = self._residual(U, d, dt, tgt, g)
            it += 1
            if not np.isfinite(r):
                return self._accept(g, False, it)
            if abs(r) <= o.tol_r * A_n:
                return self._accept(g, True, it)
            if g_prev is None:
                g_prev, r_prev, g = g, r, o.hi
                continue
            den = r - r_prev
            if den == 0.0:
                return self._accept(g, False, it)
            g_new = g - r * (g - g_prev) / den
            if abs(g_new - g) <= o.tol_g:
                return self._accept(g, True, it)
            g_prev, r_prev, g = g, r, g_new
        return self._accept(g, False, it)

    def step(self, dt):
        U = self.U
        H_n = self.entropy(U)
        A_n = self.abs_entropy(U)
        d, dH, stage_dot = self.stages(U, dt)
        if self.opts.relax:
            guess = self.gamma_prev if self.opts.guess == GUESS_PREV else 1.0
            g, it, conv = self.newton(U, d, dt, H_n, A_n, dH, guess)
        else:
            g, it, conv = 1.0, 0, True
        self.U = U + g * dt * d
        self.t += g * dt
        if self.opts.relax and conv:
            self.gamma_prev = g
        rec = StepRecord(g, it, conv, H_n, dH, self.entropy(self.U), self.t, stage_dot)
        return rec

    def run(self, dt, nsteps):
        return [self.step(dt) for _ in range(nsteps)]
