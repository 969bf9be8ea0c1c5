"""P-ERK Butcher tableaux in full (S x S) form, order conditions, stability polynomials.

Archetypes (appendix A of the paper):
  p = 2  eq. PERK_ButcherTableauClassic_p2_E36: c_i = (i-1)/(2(S-1)) (read off the
         S = 6 example), b = e_S, rows (c_i - a_i, ..., a_i) with a_i = a_{i,i-1}.
  p = 3  eq. PERK_ButcherTableauOwn_p3: c_i = (i-1)/(S-3) for i <= S-2, c_{S-1} = 1,
         c_S = 1/2; b_1 = b_{S-1} = 1/6, b_S = 2/3.  Row S reads
         (1/2 - a_{S,S-1}, ..., a_{S,S-1}) (the printed '1 - a' contradicts
         eq. InternalConsistency with c_S = 1/2).  Order 3 forces
         a_{S-1,S-2}/6 + 2 a_{S,S-1}/3 = 1/6.  S = 3 is SSPRK3.
  p = 4  eq. PERK_ButcherTableau_p4 with the constants of eq.
         4thOrderPERK_BaseCoeffs, c_2..c_{S-3} = 1, b_{S-1} = b_S = 1/2; row S-1
         couples K_{S-2} (the printed a_{S-1,S-1} index is a typo).

Member r with E^(r) stage evaluations is active at stage 1 and at stages
S - E^(r) + 2 .. S (example after eq. PERK_ButcherTableauClassic_p2_E36).  At
inactive stages its row is (c_i, 0, ...), at its first active stage after
stage 1 the row is (c_i, 0, ...) as well (K_{i-1} of that member was not
evaluated).  Shared c and b (eq. InternalConsistency, eq. Conservation).

Free coefficients (not printed in the paper, Sec. 2.2): p = 2 matches the
Taylor coefficients 1/j! of exp(z) up to degree E (alpha_j =
c_{S-j+2} prod_{m=S-j+3}^S a_m solved top-down); p = 3 and p = 4 use
a_{i,i-1} = c_i / 8 on the free chain rows and a_{S-1,S-2} = 1/4 (p = 3),
a rule chosen so that every member is stable on a segment of the imaginary
axis (the paper's optimised coefficients are not printed).
"""
import itertools
import math

import numpy as np

P4_C_SM2 = 0.479274057836310
P4_A_SM2_PROD = 0.114851811257441      # a_{S-2,S-3} * c_{S-3}
P4_A_SM1 = 0.648906880894214
P4_A_S = 0.0283121635129678

MIN_E = {2: 2, 3: 3, 4: 5}


def active_stages(S, E):
    """1-based stage indices where a member with E evaluations is evaluated."""
    return [1] + list(range(S - E + 2, S + 1))


def abscissae(p, S):
    if p == 2:
        return np.array([(i - 1) / (2.0 * (S - 1)) for i in range(1, S + 1)])
    if p == 3:
        c = np.zeros(S)
        for i in range(1, S - 1):
            c[i - 1] = (i - 1) / (S - 3.0) if S > 3 else 0.0
        c[S - 2] = 1.0
        c[S - 1] = 0.5
        return c
    if p == 4:
        c = np.ones(S)
        c[0] = 0.0
        c[S - 3] = P4_C_SM2
        c[S - 2] = 0.5 + math.sqrt(3.0) / 6.0
        c[S - 1] = 0.5 - math.sqrt(3.0) / 6.0
        return c
    raise ValueError(p)


def weights(p, S):
    b = np.zeros(S)
    if p == 2:
        b[S - 1] = 1.0
    elif p == 3:
        b[0] = 1.0 / 6.0
        b[S - 2] = 1.0 / 6.0
        b[S - 1] = 2.0 / 3.0
    else:
        b[S - 2] = 0.5
        b[S - 1] = 0.5
    return b


def member(p, S, E):
    """Full Butcher matrix A (S x S, 0-based) of the member with E evaluations."""
    if E < MIN_E[p] or E > S:
        raise ValueError("E out of range for this archetype")
    c = abscissae(p, S)
    A = np.zeros((S, S))
    act = set(active_stages(S, E))
    first = S - E + 2                  # first active stage after stage 1 (1-based)
    sub = {}                           # 1-based row i -> a_{i,i-1}
    if p == 2:
        # Taylor-matching chain, solved from the last row upwards
        prod = 1.0
        for j in range(3, E + 1):
            m = S - j + 3              # row whose a_m is fixed by alpha_j
            a = (1.0 / math.factorial(j)) / (c[S - j + 2 - 1] * prod)
            sub[m] = a
            prod *= a
    elif p == 3:
        for i in range(first + 1, S - 1):
            sub[i] = c[i - 1] / 8.0
        if S - 1 > first:
            sub[S - 1] = 0.25
        a_sm1 = sub.get(S - 1, 0.0)
        sub[S] = (1.0 - a_sm1) / 4.0
    else:
        for i in range(first + 1, S - 2):
            sub[i] = c[i - 1] / 8.0
        sub[S - 2] = P4_A_SM2_PROD / c[S - 4]
        sub[S - 1] = P4_A_SM1
        sub[S] = P4_A_S
    for i in range(2, S + 1):
        a = sub.get(i, 0.0) if (i in act and i > first) else 0.0
        if i - 1 == 1:
            A[i - 1, 0] = c[i - 1]     # row 2: the only earlier stage is K_1
            continue
        A[i - 1, i - 2] = a
        A[i - 1, 0] = c[i - 1] - a
    return A


def family(p, E_list):
    """All members of a P-ERK family sharing S = max E; returns (c, b, [A^(r)])."""
    S = max(E_list)
    return abscissae(p, S), weights(p, S), [member(p, S, E) for E in E_list]


# -------------------------------------------------------- order conditions ---

def rooted_trees(n):
    """All rooted trees with n vertices as nested sorted tuples of children."""
    if n == 1:
        return [()]
    out = set()
    for parts in _partitions(n - 1):
        for combo in itertools.product(*[rooted_trees(k) for k in parts]):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def _partitions(n, maxv=None):
    maxv = maxv or n
    if n == 0:
        yield []
        return
    for k in range(min(n, maxv), 0, -1):
        for rest in _partitions(n - k, k):
            yield [k] + rest


def tree_size(t):
    return 1 + sum(tree_size(c) for c in t)


def tree_density(t):
    return tree_size(t) * math.prod(tree_density(c) for c in t)


def _coloured(t, R):
    """All colourings of the non-root vertices: yields nested (colour, children)."""
    child_options = [list(_coloured_full(c, R)) for c in t]
    for combo in itertools.product(*child_options):
        yield combo


def _coloured_full(t, R):
    for col in range(R):
        for kids in _coloured(t, R):
            yield (col, kids)


def _g(kids, As, S):
    """g_i = prod over children (sum_j A^(col child)_{ij} g_j(child))."""
    g = np.ones(S)
    for col, sub in kids:
        g = g * (As[col] @ _g(sub, As, S))
    return g


def order_residuals(c, b, As, p):
    """Max |b^T g(t) - 1/gamma(t)| over all coloured trees with <= p vertices,
    and over members the internal-consistency residual |A 1 - c|."""
    S = len(b)
    worst = 0.0
    for n in range(1, p + 1):
        for t in rooted_trees(n):
            dens = tree_density(t)
            for kids in _coloured(t, len(As)):
                worst = max(worst, abs(b @ _g(kids, As, S) - 1.0 / dens))
    cons = max(np.max(np.abs(A.sum(axis=1) - c)) for A in As)
    return worst, cons


def stability_coeffs(b, A):
    """alpha_j of P(z) = 1 + sum_j alpha_j z^j: alpha_j = b^T A^{j-1} 1."""
    S = len(b)
    out = [1.0]
    v = np.ones(S)
    for _ in range(S):
        out.append(float(b @ v))
        v = A @ v
    return np.array(out)


# ------------------------------------------- members from a stability polynomial ---

def _set_chain(A, c, m, a):
    """Row m (1-based) with K_{m-1} coefficient a and K_1 coefficient c_m - a."""
    A[m - 1, m - 2] = a
    A[m - 1, 0] = c[m - 1] - a


def _solve_row(A, c, b, m, j, target):
    """Set row m so that alpha_j = b^T A^{j-1} 1 equals target; alpha_j is
    affine in that row's entry (one evaluation at 0 and one at 1)."""
    _set_chain(A, c, m, 0.0)
    f0 = stability_coeffs(b, A)[j]
    _set_chain(A, c, m, 1.0)
    f1 = stability_coeffs(b, A)[j]
    a = (target - f0) / (f1 - f0)
    _set_chain(A, c, m, a)
    return a


def member_from_poly(p, S, E, alpha):
    """Member with E evaluations whose stability polynomial has the
    coefficients alpha[k], k = 0..E (alpha_k = 1/k! for k <= p; the E - p
    others free, Sec. 2.2), in the archetype's structure.

    p = 2: alpha_j fixes row S - j + 3, taken from the last row upwards.
    p = 3: for a trial t = a_{S-1,S-2} (row S then (1 - t)/4 by the order-3
    condition) alpha_j, j = 4 .. E-1, fixes row S - j + 2 in turn; alpha_E is
    then a scalar equation in t.  Of its roots on [-3, 3] the one nearest the
    default 1/4 is taken (a reading: the polynomial does not fix the chain
    uniquely).  p = 4 is not supported (its base stages fix one coefficient).
    Every coefficient is evaluated from the full Butcher matrix."""
    c, b = abscissae(p, S), weights(p, S)
    A = member(p, S, E)
    first = S - E + 2
    alpha = np.asarray(alpha, dtype=float)
    if p == 2:
        for j in range(3, E + 1):
            _solve_row(A, c, b, S - j + 3, j, alpha[j])
        return A
    if p != 3:
        raise NotImplementedError("p = 4")
    if E <= 3:
        return A

    A0 = A.copy()

    def resid(t):
        A[:] = A0                  # no entry of an earlier trial (possibly non-finite) survives
        _set_chain(A, c, S - 1, t)
        _set_chain(A, c, S, (1.0 - t) / 4.0)
        for j in range(4, E):
            _solve_row(A, c, b, S - j + 2, j, alpha[j])
        return stability_coeffs(b, A)[E] - alpha[E]

    ts = np.linspace(-3.0, 3.0, 6001)
    with np.errstate(all="ignore"):
        f = np.array([resid(t) for t in ts])
        roots = []
        for i in range(len(ts) - 1):
            if np.isfinite(f[i]) and np.isfinite(f[i + 1]) and f[i] * f[i + 1] <= 0.0:
                lo, hi, flo = ts[i], ts[i + 1], f[i]
                for _ in range(200):
                    mid = 0.5 * (lo + hi)
                    fm = resid(mid)
                    if (fm <= 0.0) == (flo <= 0.0):
                        lo, flo = mid, fm
                    else:
                        hi = mid
                roots.append(0.5 * (lo + hi))
    if not roots:
        raise ValueError("no chain of the p = 3 archetype has this stability polynomial")
    resid(min(roots, key=lambda r: abs(r - 0.25)))
    return A


def family_from_poly(p, E_list, alphas):
    S = max(E_list)
    return abscissae(p, S), weights(p, S), [member_from_poly(p, S, E, a) for E, a in zip(E_list, alphas)]
