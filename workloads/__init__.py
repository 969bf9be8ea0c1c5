"""Seeded synthetic workloads: meshes, partition assignment and initial states.

This module is the only code shared by the CUDA path and the CPU oracle.  It
holds none of the method's arithmetic (no DG operators, fluxes, Runge-Kutta
tableaux or relaxation); it only places mesh nodes, pairs faces, assigns
partitions by element size and evaluates initial conditions at the nodes.

Conventions (the input format of ``perrk_create``):

* polynomial degree N = 3, nodes per element NP = 4**dim, reference node
  positions are the four Legendre-Gauss-Lobatto points {-1, -1/sqrt5, 1/sqrt5, 1}
  (written here as the input format's fixed point set);
* node index inside an element: q = i + 4*j + 16*k (i along xi fastest);
* faces of an element: 0 = -xi, 1 = +xi, 2 = -eta, 3 = +eta, 4 = -zeta, 5 = +zeta;
* face list rows (eL, fL, eR, fR): fL is a '+' face (1, 3, 5) of eL, fR = fL - 1
  the matching '-' face of eR, face nodes in the same order on both sides;
* state layout SoA [V][n_elem][NP] in float64;
* partition 0 is the finest (largest stage-evaluation count E), ids 0..R-1.

Physical setups follow the paper's test cases: the isentropic vortex
(Sec. 4.1.2, eqs. for rho, v, p of the vortex), the Kelvin-Helmholtz
instability initial state (Sec. 3.2.2), the traveling viscous shock
(Sec. 4.3.2, eq. ViscousShockSolution) and the Taylor-Green vortex (standard
form, not in the paper).  A workload's ``mu`` > 0 (with ``prandtl``) asks for
the Navier-Stokes-Fourier viscous terms.  Partition assignment uses the shortest element edge
(Sec. 2.2, eq. CharSpeed_DG with h the minimal corner distance).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_POLY = 3
REF_NODES = np.array([-1.0, -1.0 / math.sqrt(5.0), 1.0 / math.sqrt(5.0), 1.0])
GAMMA_GAS = 1.4
BASE_SEED = 250704991


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    equation: str            # "burgers1d" | "euler2d" | "euler3d"
    coords: np.ndarray       # [n_elem, NP, dim] float64
    faces: np.ndarray        # [n_faces, 4] int32 (eL, fL, eR, fR)
    part: np.ndarray         # [n_elem] int32, 0 = finest
    E: list                  # stage evaluations per partition (descending)
    order: int               # P-ERK order p
    u0: np.ndarray           # [V, n_elem, NP] float64
    dt: float
    volume_flux: str         # "ec_burgers" | "ec_ranocha"
    surface_flux: str        # "ec" | "es_rusanov"
    gamma_gas: float = GAMMA_GAS
    info: dict = dataclasses.field(default_factory=dict)
    mu: float = 0.0          # dynamic viscosity (0: inviscid Euler)
    prandtl: float = 0.75    # Prandtl number of the viscous runs
    # 2:1 non-conforming interfaces: rows (coarse element, its face, fine
    # element on the face's lower half, fine element on the upper half)
    mortars: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 4), dtype=np.int32))

    @property
    def n_elem(self):
        return self.coords.shape[0]

    @property
    def nvar(self):
        return self.u0.shape[0]

    @property
    def n_dof(self):
        return int(self.u0.size)

    def dof_stage_per_step(self):
        """Sum over partitions of E^(r) * M^(r) (M = nodes x variables), the
        paper's count of scalar RHS evaluations per step (eq. RHSEvals)."""
        per_elem = self.u0.shape[0] * self.u0.shape[2]
        counts = np.bincount(self.part, minlength=len(self.E))
        return int(sum(e * c for e, c in zip(self.E, counts)) * per_elem)


# ----------------------------------------------------------------------------
# structured (logically Cartesian, periodic) meshes
# ----------------------------------------------------------------------------

def _elem_index(ix, iy, iz, n):
    return ix + n[0] * (iy + n[1] * iz)


def structured_faces(n):
    """Periodic face list for an n[0] x n[1] x n[2] element grid (missing dims = 1)."""
    dim = len(n)
    nn = list(n) + [1] * (3 - dim)
    iz, iy, ix = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    e = _elem_index(ix, iy, iz, nn)
    cols = [np.stack([e, np.full_like(e, 1), _elem_index((ix + 1) % nn[0], iy, iz, nn), np.zeros_like(e)], 1)]
    if dim >= 2:
        cols.append(np.stack([e, np.full_like(e, 3), _elem_index(ix, (iy + 1) % nn[1], iz, nn), np.full_like(e, 2)], 1))
    if dim >= 3:
        cols.append(np.stack([e, np.full_like(e, 5), _elem_index(ix, iy, (iz + 1) % nn[2], nn), np.full_like(e, 4)], 1))
    # rows ordered element by element, directions in turn
    return np.stack(cols, 1).reshape(-1, 4).astype(np.int32)


def tensor_coords(edges):
    """Node coordinates of an axis-aligned tensor mesh from per-axis cell edges."""
    dim = len(edges)
    n = [len(e) - 1 for e in edges]
    nn = n + [1] * (3 - dim)
    t = 0.5 * (REF_NODES + 1.0)
    per_axis = []
    for a in range(dim):
        lo = np.asarray(edges[a][:-1])
        hi = np.asarray(edges[a][1:])
        per_axis.append(lo[:, None] + (hi - lo)[:, None] * t[None, :])  # [n_a, 4]
    iz, iy, ix = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    idx = [ix.ravel(), iy.ravel(), iz.ravel()]
    NP = 4 ** dim
    q = np.arange(NP)
    loc = [q % 4, (q // 4) % 4, q // 16]
    out = np.empty((int(np.prod(n)), NP, dim))
    for a in range(dim):
        out[:, :, a] = per_axis[a][idx[a][:, None], loc[a][None, :]]
    return out


def min_corner_edge(coords, dim):
    """Shortest distance between adjacent corner nodes of each element."""
    c = coords
    if dim == 1:
        return np.abs(c[:, 3, 0] - c[:, 0, 0])
    corner = lambda i, j, k=0: c[:, (3 if i else 0) + 4 * (3 if j else 0) + 16 * (3 if k else 0), :]
    pairs = []
    ks = (0, 1) if dim == 3 else (0,)
    for k in ks:
        for j in (0, 1):
            pairs.append((corner(0, j, k), corner(1, j, k)))
        for i in (0, 1):
            pairs.append((corner(i, 0, k), corner(i, 1, k)))
    if dim == 3:
        for i in (0, 1):
            for j in (0, 1):
                pairs.append((corner(i, j, 0), corner(i, j, 1)))
    d = np.stack([np.linalg.norm(a - b, axis=-1) for a, b in pairs], axis=1)
    return d.min(axis=1)


def levels_from_h(h, h_ref, n_levels):
    """Refinement level of each element: round(log2(h_ref / h)), clipped.
    Level L elements get partition id n_levels-1-L so that 0 is the finest."""
    lev = np.clip(np.rint(np.log2(h_ref / h)), 0, n_levels - 1).astype(np.int32)
    return (n_levels - 1 - lev).astype(np.int32)


# ----------------------------------------------------------------------------
# initial states
# ----------------------------------------------------------------------------

def prim_to_cons(rho, v, p, gamma=GAMMA_GAS):
    v = np.asarray(v)
    kin = 0.5 * rho * np.sum(v * v, axis=0)
    return np.concatenate([rho[None], rho[None] * v, (p / (gamma - 1.0) + kin)[None]], axis=0)


def isentropic_vortex(x, y, t, center, strength, L=10.0, R=1.5, mach=0.4, gamma=GAMMA_GAS):
    """Isentropic vortex of Sec. 4.1.2 (background rho=1, v=(1,1), p=rho^g/(g Ma^2)),
    vortex centre translated with v_inf and wrapped to the nearest periodic image.
    The velocity perturbation is the rotated vector (-c_y, c_x)."""
    vinf = np.array([1.0, 1.0])
    cx = x - center[0] - vinf[0] * t
    cy = y - center[1] - vinf[1] * t
    cx = (cx + L) % (2 * L) - L
    cy = (cy + L) % (2 * L) - L
    g = np.exp((1.0 - (cx * cx + cy * cy)) / (2.0 * R * R))
    rho = (1.0 - strength ** 2 * mach ** 2 * (gamma - 1.0) * g * g / (8.0 * math.pi ** 2)) ** (1.0 / (gamma - 1.0))
    amp = strength * g / (2.0 * math.pi * R)
    vx = vinf[0] - amp * cy
    vy = vinf[1] + amp * cx
    p = rho ** gamma / (gamma * mach ** 2)
    return prim_to_cons(rho, np.stack([vx, vy]), p, gamma)


def kelvin_helmholtz(x, y, phase=0.0, amp=0.1, gamma=GAMMA_GAS):
    """Kelvin-Helmholtz initial state of Sec. 3.2.2 with a seeded phase."""
    b = np.tanh(15.0 * y + 7.5) - np.tanh(15.0 * y - 7.5)
    rho = 0.5 + 0.75 * b
    vx = 0.5 * (b - 1.0)
    vy = amp * np.sin(2.0 * math.pi * x + phase)
    p = np.ones_like(x)
    return prim_to_cons(rho, np.stack([vx, vy]), p, gamma)


def taylor_green(x, y, z, mach=0.1, gamma=GAMMA_GAS):
    """Taylor-Green vortex (Brachet/DeBonis form), rho = 1, V0 = 1."""
    vx = np.sin(x) * np.cos(y) * np.cos(z)
    vy = -np.cos(x) * np.sin(y) * np.cos(z)
    vz = np.zeros_like(x)
    p = 1.0 / (gamma * mach ** 2) + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return prim_to_cons(np.ones_like(x), np.stack([vx, vy, vz]), p, gamma)


def viscous_shock_prims(s, gamma=5.0 / 3.0, mu=0.15, rho0=1.0, vs=1.0):
    """Traveling viscous shock of Sec. 4.3.2 (eq. ViscousShockSolution) at the
    signed distance s = x0 along the shock normal (x0 = x - v t), for the
    Mach number Ma = 2 / sqrt(3 - gamma) at which the profile is explicit:
    c0 = v / Ma, p0 = c0^2 rho0 / gamma, chi = 2 exp(s / (2 l)),
    w = 1 + (1 - sqrt(1 + 2 chi^2)) / (2 chi^2);  rho = rho0 / w,
    u = v (1 - w), p = p0 / w (1 + (gamma - 1) / 2 Ma^2 (1 - w^2)).
    This w solves dw/ds = -(w - 1)(w - 1/2) / (l w).  The momentum balance of
    the Navier-Stokes-Fourier equations across the profile (Stokes'
    hypothesis; Pr = 3/4 keeps the total enthalpy constant) requires
    l = 8 gamma mu / (3 (gamma + 1) rho0 v), which is taken here: the printed
    length mu / (gamma-1) * 2 gamma / (gamma-1) / (rho0 v) is larger by
    2 / (gamma - 1)^2 (4.5 at gamma = 5/3), and with it the profile is not a
    solution at the stated viscosity.
    s may be complex (complex-step derivatives).  Returns (rho, u_n, p)."""
    ma = 2.0 / math.sqrt(3.0 - gamma)
    c0 = vs / ma
    p0 = c0 * c0 * rho0 / gamma
    ell = 8.0 * gamma * mu / (3.0 * (gamma + 1.0) * rho0 * vs)
    chi = 2.0 * np.exp(s / (2.0 * ell))
    w = 1.0 + (1.0 - np.sqrt(1.0 + 2.0 * chi * chi)) / (2.0 * chi * chi)
    return rho0 / w, vs * (1.0 - w), p0 / w * (1.0 + 0.5 * (gamma - 1.0) * ma * ma * (1.0 - w * w))


def to_soa(u_nodes):
    """[V, n_elem, NP] from an array already shaped that way (copy, contiguous)."""
    return np.ascontiguousarray(u_nodes, dtype=np.float64)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def burgers_1d(n_coarse_each_side=24, n_fine=16, E=(8, 4), dt=None):
    """64 periodic elements on [0, 1]: 24 of width h, 16 central of width h/4,
    24 of width h (h = 1/52).  u0 = 1 + 0.5 sin(2 pi x)."""
    n_total_width = 2 * n_coarse_each_side + n_fine / 4.0
    h = 1.0 / n_total_width
    widths = [h] * n_coarse_each_side + [h / 4] * n_fine + [h] * n_coarse_each_side
    edges = np.concatenate([[0.0], np.cumsum(widths)])
    edges[-1] = 1.0
    coords = tensor_coords([edges])
    n = len(widths)
    faces = structured_faces([n])
    hmin = min_corner_edge(coords, 1)
    part = levels_from_h(hmin, h, 2)
    x = coords[:, :, 0]
    u0 = (1.0 + 0.5 * np.sin(2 * math.pi * x))[None]
    if dt is None:
        dt = 0.25 * h / 1.5 / 7.0 * 2.0
    return Workload("burgers1d_64", 1, "burgers1d", coords, faces, part, list(E), 2, to_soa(u0), dt,
                    "ec_burgers", "ec", info=dict(h=h, t_end=0.1))


def _radial_contraction(X, Y, R0=6.0, B=0.75):
    """Smooth, compactly supported, monotone radial map r -> r (1 - B (1 - (r/R0)^4)^3):
    identity for r >= R0, element size reduced by 1 - B = 1/4 around the centre."""
    r = np.sqrt(X * X + Y * Y)
    s = np.minimum(r / R0, 1.0)
    fac = 1.0 - B * (1.0 - s ** 4) ** 3
    return X * fac, Y * fac


def vortex_2d(n=64, L=10.0, seed=1, n_levels=3, E=(12, 6, 3), order=3, cfl=0.5, mixed_note=None, mu=0.0):
    """Isentropic vortex on an n x n periodic curvilinear mesh of [-L, L]^2: a
    central patch contracted by 4 (two refinement levels), then a seeded
    smooth periodic displacement of at most 10% of the logical cell size."""
    rng = np.random.default_rng(BASE_SEED + 2 + 1000 * seed)
    H = 2 * L / n
    k = rng.integers(1, 4, size=4)
    ph = rng.uniform(0, 2 * math.pi, size=4)
    t = 0.5 * (REF_NODES + 1.0)
    NP = 16
    coords = np.empty((n * n, NP, 2))
    for iy in range(n):
        for ix in range(n):
            e = ix + n * iy
            for q in range(NP):
                i, j = q % 4, q // 4
                X = -L + (ix + t[i]) * H
                Y = -L + (iy + t[j]) * H
                sx = (X + L) / (2 * L)
                sy = (Y + L) / (2 * L)
                dX = 0.1 * H * math.sin(2 * math.pi * k[0] * sx + ph[0]) * math.sin(2 * math.pi * k[1] * sy + ph[1])
                dY = 0.1 * H * math.sin(2 * math.pi * k[2] * sx + ph[2]) * math.sin(2 * math.pi * k[3] * sy + ph[3])
                x, y = _radial_contraction(np.float64(X + dX), np.float64(Y + dY))
                coords[e, q, 0] = x
                coords[e, q, 1] = y
    faces = structured_faces([n, n])
    hmin = min_corner_edge(coords, 2)
    part = levels_from_h(hmin, H, n_levels)
    center = rng.uniform(-2.0, 2.0, size=2)
    strength = rng.uniform(3.0, 5.0)
    u0 = isentropic_vortex(coords[:, :, 0], coords[:, :, 1], 0.0, center, strength, L=L)
    # characteristic speed |v| + c <= ~2.2 for this vortex; finest h ~ H/4
    dt = cfl * (H / 4) / (2 * N_POLY + 1) / 2.5
    return Workload(f"vortex2d_{n}x{n}", 2, "euler2d", coords, faces, part, list(E), order, to_soa(u0), dt,
                    "ec_ranocha", "es_rusanov",
                    info=dict(center=center, strength=strength, L=L, H=H, perturb_k=k, perturb_phase=ph), mu=mu)


def graded_edges(n, lo, hi, bands, n_levels, fine_counts):
    """1D edges of n cells on [lo, hi] refined towards the band centres.
    Around each band centre: fine_counts[l] cells of width h0 / 2^(l) on each
    side for l = n_levels-1 .. 1 (innermost finest), the rest coarse and
    uniform.  Returns (edges, level per cell)."""
    per_band = []
    for l in range(n_levels - 1, 0, -1):
        per_band.append((l, fine_counts[l]))
    # cells per band: innermost level counted once on each side
    band_cells = []
    for c in bands:
        seq = []
        for l, cnt in per_band:
            seq = [l] * cnt + seq + [l] * cnt
        band_cells.append((c, seq))
    n_fine = sum(len(s) for _, s in band_cells)
    n_coarse = n - n_fine
    assert n_coarse > 0
    # solve for the coarse width h0' so that the total length fits, with the
    # fine cells measured in units of the nominal coarse size h0 = (hi-lo)/n
    h0 = (hi - lo) / n
    fine_len = sum(h0 / 2 ** l for _, s in band_cells for l in s)
    hc = ((hi - lo) - fine_len) / n_coarse
    # lay out: coarse cells evenly distributed between bands
    band_lengths = [sum(h0 / 2 ** l for l in s) for _, s in band_cells]
    widths, levels = [], []
    centres = [c for c, _ in band_cells]
    # compute coarse counts between band edges proportional to gap length
    starts = [c - bl / 2 for c, bl in zip(centres, band_lengths)]
    ends = [c + bl / 2 for c, bl in zip(centres, band_lengths)]
    gaps = [starts[0] - lo] + [starts[i + 1] - ends[i] for i in range(len(centres) - 1)] + [hi - ends[-1]]
    total_gap = sum(gaps)
    counts = [int(round(g / total_gap * n_coarse)) for g in gaps]
    counts[-1] = n_coarse - sum(counts[:-1])
    for bi in range(len(centres)):
        widths += [hc] * counts[bi]
        levels += [0] * counts[bi]
        for l in band_cells[bi][1]:
            widths.append(h0 / 2 ** l)
            levels.append(l)
    widths += [hc] * counts[-1]
    levels += [0] * counts[-1]
    edges = np.concatenate([[lo], lo + np.cumsum(widths)])
    edges[-1] = hi
    return edges, np.asarray(levels, dtype=np.int32), h0


def khi_2d(n=256, seed=1, E=(16, 10, 7, 5), order=4, n_levels=4, fine_counts=None, cfl=0.4):
    """Kelvin-Helmholtz on [-1, 1]^2, n x n quads, uniform in x and graded in y
    with 4 levels around the shear layers y = +-0.5 (partition by shortest edge)."""
    rng = np.random.default_rng(BASE_SEED + 3 + 1000 * seed)
    if fine_counts is None:
        s = n // 256 if n >= 256 else 0
        fine_counts = {1: max(1, n // 32), 2: max(1, n // 32), 3: max(1, n // 32)}
    ex = np.linspace(-1.0, 1.0, n + 1)
    ey, ylev, h0 = graded_edges(n, -1.0, 1.0, [-0.5, 0.5], n_levels, fine_counts)
    coords = tensor_coords([ex, ey])
    faces = structured_faces([n, n])
    hx = 2.0 / n
    hmin = min_corner_edge(coords, 2)
    part = levels_from_h(hmin, hx, n_levels)
    phase = rng.uniform(0, 2 * math.pi)
    u0 = kelvin_helmholtz(coords[:, :, 0], coords[:, :, 1], phase=phase)
    hfine = hmin.min()
    dt = cfl * hfine / (2 * N_POLY + 1) / 2.0
    return Workload(f"khi2d_{n}x{n}", 2, "euler2d", coords, faces, part, list(E), order, to_soa(u0), dt,
                    "ec_ranocha", "es_rusanov", info=dict(phase=phase, hx=hx))


def tgv_3d(n=64, n_fine=16, E=(8, 4), order=3, cfl=0.5, mu=0.0):
    """Taylor-Green vortex on [0, 2 pi]^3, n^3 affine boxes, the central n_fine
    cells per axis at half width (partition by shortest edge: cross of slabs)."""
    nc = n - n_fine
    hc = 2 * math.pi / (nc + n_fine / 2.0)
    w = [hc] * (nc // 2) + [hc / 2] * n_fine + [hc] * (nc - nc // 2)
    e1 = np.concatenate([[0.0], np.cumsum(w)])
    e1[-1] = 2 * math.pi
    coords = tensor_coords([e1, e1, e1])
    faces = structured_faces([n, n, n])
    hmin = min_corner_edge(coords, 3)
    part = levels_from_h(hmin, hc, 2)
    u0 = taylor_green(coords[:, :, 0], coords[:, :, 1], coords[:, :, 2])
    c = math.sqrt(1.0 / 0.01)  # speed of sound for Ma = 0.1, rho = 1
    dt = cfl * (hc / 2) / (2 * N_POLY + 1) / (c + 1.0)
    return Workload(f"tgv3d_{n}^3", 3, "euler3d", coords, faces, part, list(E), order, to_soa(u0), dt,
                    "ec_ranocha", "ec", info=dict(hc=hc), mu=mu)


def viscous_shock_2d(n=16, angle=0.0, L=2.0, gamma=5.0 / 3.0, mu=0.15, E=(4,), order=2):
    """The viscous shock of Sec. 4.3.2 on the periodic square [-L, L]^2 of n x n
    boxes, its normal rotated by `angle` in the plane (the state jumps across
    the periodic seams; away from them it is the traveling profile)."""
    e = np.linspace(-L, L, n + 1)
    coords = tensor_coords([e, e])
    faces = structured_faces([n, n])
    nrm = np.array([math.cos(angle), math.sin(angle)])
    sx = coords[:, :, 0] * nrm[0] + coords[:, :, 1] * nrm[1]
    rho, un, p = viscous_shock_prims(sx, gamma, mu)
    u0 = prim_to_cons(rho, un[None] * nrm[:, None, None], p, gamma)
    h = 2 * L / n
    dt = 0.035 * (h / (N_POLY + 1)) ** 2
    part = np.zeros(n * n, np.int32)
    return Workload(f"viscous_shock2d_{n}", 2, "euler2d", coords, faces, part, list(E), order, to_soa(u0), dt,
                    "ec_ranocha", "es_rusanov", gamma_gas=gamma, info=dict(angle=angle, L=L, normal=nrm), mu=mu,
                    prandtl=0.75)


def small_box_2d(n=8, seed=0, R=2, E=(6, 3), order=3, ic="vortex", surface="es_rusanov", random_parts=False, mu=0.0):
    """Small tensor mesh on [-L, L]^2 for tests, optionally with random partition ids."""
    rng = np.random.default_rng(BASE_SEED + 7 + 1000 * seed)
    L = 5.0
    edges, lev, h0 = graded_edges(n, -L, L, [0.0], R, {l: 1 for l in range(1, R)}) if R > 1 else (np.linspace(-L, L, n + 1), None, 2 * L / n)
    ex = np.linspace(-L, L, n + 1)
    coords = tensor_coords([ex, edges])
    faces = structured_faces([n, n])
    hmin = min_corner_edge(coords, 2)
    part = levels_from_h(hmin, 2 * L / n, R) if R > 1 else np.zeros(n * n, np.int32)
    if random_parts:
        part = rng.integers(0, R, size=n * n).astype(np.int32)
    if ic == "vortex":
        u0 = isentropic_vortex(coords[:, :, 0], coords[:, :, 1], 0.0, rng.uniform(-1, 1, 2), 4.0, L=L, R=1.0)
    else:
        u0 = kelvin_helmholtz(coords[:, :, 0] / L, coords[:, :, 1] / L, phase=rng.uniform(0, 6.28))
    dt = 0.2 * hmin.min() / (2 * N_POLY + 1) / 2.5
    return Workload(f"box2d_{n}", 2, "euler2d", coords, faces, part, list(E), order, to_soa(u0), dt,
                    "ec_ranocha", surface, mu=mu)


def batched_2d(n_inst=256, seed=1, n_min=16, n_max=128, S=12, order=3):
    """Independent 2D Euler instances: sizes n x n with n ~ U{n_min..n_max},
    2-4 partitions from a refinement band of seeded position and width (tensor
    mesh graded in y around the band, partition by shortest edge), and an
    isentropic vortex or a Kelvin-Helmholtz state by a seeded coin flip.  All
    members use the same P-ERK family size S (order 3)."""
    rng = np.random.default_rng(BASE_SEED + 5 + 1000 * seed)
    E_by_R = {2: [S, 6], 3: [S, 6, 3], 4: [S, 8, 5, 3]}
    out = []
    for k in range(n_inst):
        n = int(rng.integers(n_min, n_max + 1))
        R = int(rng.integers(2, 5))
        L = 5.0
        centre = float(rng.uniform(-0.5 * L, 0.5 * L))
        per_level = max(1, n // 32)
        ex = np.linspace(-L, L, n + 1)
        ey, _, _ = graded_edges(n, -L, L, [centre], R, {l: per_level for l in range(1, R)})
        coords = tensor_coords([ex, ey])
        faces = structured_faces([n, n])
        hmin = min_corner_edge(coords, 2)
        part = levels_from_h(hmin, 2 * L / n, R)
        if rng.uniform() < 0.5:
            u0 = isentropic_vortex(coords[:, :, 0], coords[:, :, 1], 0.0, rng.uniform(-1, 1, 2), float(rng.uniform(3, 5)),
                                   L=L, R=1.0)
            ic = "vortex"
        else:
            u0 = kelvin_helmholtz(coords[:, :, 0] / L, coords[:, :, 1] / L, phase=float(rng.uniform(0, 2 * math.pi)))
            ic = "khi"
        dt = 0.3 * hmin.min() / (2 * N_POLY + 1) / 2.5
        out.append(Workload(f"batch{k}_{ic}_{n}x{n}_R{R}", 2, "euler2d", coords, faces, part, list(E_by_R[R]), order,
                            to_soa(u0), dt, "ec_ranocha", "es_rusanov", info=dict(n=n, R=R, ic=ic)))
    return out


# ------------------------------------------------------------- quadtree meshes

class Quadtree:
    """A 2:1-balanced quadtree of periodic square cells on [-L, L]^2 over an
    n x n base grid.  A leaf is (level, ix, iy) with 0 <= ix, iy < n 2^level;
    its cell is [-L + ix h, -L + (ix + 1) h] x [...], h = 2L / (n 2^level).
    Mesh construction only: cell boxes, conforming face pairs, 2:1 mortars."""

    def __init__(self, n, L, leaves):
        self.n, self.L = n, L
        self.leaves = sorted(set(leaves))
        self._index = {c: i for i, c in enumerate(self.leaves)}

    @classmethod
    def uniform(cls, n, L):
        return cls(n, L, [(0, ix, iy) for iy in range(n) for ix in range(n)])

    def cells_at(self, lev):
        return self.n << lev

    def h(self, lev):
        return 2.0 * self.L / self.cells_at(lev)

    def centre(self, c):
        lev, ix, iy = c
        h = self.h(lev)
        return -self.L + (ix + 0.5) * h, -self.L + (iy + 0.5) * h

    def leaf_covering(self, lev, ix, iy):
        """The leaf that contains cell (lev, ix, iy) (it or an ancestor), or None if that cell is refined."""
        m = self.cells_at(lev)
        ix, iy = ix % m, iy % m
        for l in range(lev, -1, -1):
            c = (l, ix >> (lev - l), iy >> (lev - l))
            if c in self._index:
                return c
        return None

    def refine(self, marks):
        """Split the marked leaves into four children, then refine further
        until every face neighbour differs by at most one level."""
        leaves = set(self.leaves)
        todo = [c for c in marks if c in leaves]
        while todo:
            for c in todo:
                if c in leaves:
                    leaves.remove(c)
                    lev, ix, iy = c
                    leaves.update((lev + 1, 2 * ix + a, 2 * iy + b) for a in (0, 1) for b in (0, 1))
            tree = Quadtree(self.n, self.L, leaves)
            todo = tree._unbalanced()
        return Quadtree(self.n, self.L, leaves)

    def coarsen(self, marks):
        """Merge each family of four sibling leaves that are all marked into
        their parent, unless that would break the 2:1 balance."""
        leaves = set(self.leaves)
        marked = set(marks)
        parents = {(l - 1, ix >> 1, iy >> 1) for (l, ix, iy) in marked if l > 0}
        for (l, px, py) in sorted(parents, reverse=True):
            kids = [(l + 1, 2 * px + a, 2 * py + b) for a in (0, 1) for b in (0, 1)]
            if not all(k in leaves and k in marked for k in kids):
                continue
            trial = (leaves - set(kids)) | {(l, px, py)}
            if not Quadtree(self.n, self.L, trial)._unbalanced():
                leaves = trial
        return Quadtree(self.n, self.L, leaves)

    def adapt(self, refine_marks, coarsen_marks):
        """Coarsen the families whose four leaves are all in coarsen_marks
        (where the 2:1 balance allows), then refine refine_marks (and
        whatever the balance then requires).  Returns the new tree and the
        map of its leaves to this tree's: rows (kind, a0, a1, a2, a3) with
        kind 0 = the same leaf a0, 1 = child a1 (a + 2 b) of leaf a0,
        2 = parent of leaves a0..a3 (child order a + 2 b)."""
        refine_marks = set(refine_marks)
        coarsen_marks = set(coarsen_marks) - refine_marks
        families = {}
        for (l, ix, iy) in coarsen_marks:
            if l > 0:
                families.setdefault((l - 1, ix >> 1, iy >> 1), []).append((l, ix, iy))
        keep = set()
        for par, kids in families.items():
            sibs = [(par[0] + 1, 2 * par[1] + a, 2 * par[2] + b) for a in (0, 1) for b in (0, 1)]
            if any(k in refine_marks for k in sibs):
                keep.update(kids)
        tree = self.coarsen(coarsen_marks - keep).refine(refine_marks)
        old = self._index
        rows = []
        for (l, ix, iy) in tree.leaves:
            if (l, ix, iy) in old:
                rows.append((0, old[(l, ix, iy)], 0, 0, 0))
            elif l > 0 and (l - 1, ix >> 1, iy >> 1) in old:
                rows.append((1, old[(l - 1, ix >> 1, iy >> 1)], (ix & 1) + 2 * (iy & 1), 0, 0))
            else:
                kids = [(l + 1, 2 * ix + (c & 1), 2 * iy + (c >> 1)) for c in range(4)]
                if not all(k in old for k in kids):
                    raise ValueError("adapt changed a leaf by more than one level")
                rows.append((2,) + tuple(old[k] for k in kids))
        return tree, np.asarray(rows, dtype=np.int32)

    def _unbalanced(self):
        """Leaves with a face neighbour two or more levels finer (to be split)."""
        out = set()
        for c in self.leaves:
            lev, ix, iy = c
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                nb = self.leaf_covering(lev, ix + dx, iy + dy)
                if nb is not None and nb[0] < lev - 1:
                    out.add(nb)
        return sorted(out)

    def mesh(self):
        """(coords [n_elem, 16, 2], faces [n_faces, 4], mortars [n_m, 4], level [n_elem])."""
        t = 0.5 * (REF_NODES + 1.0)
        ne = len(self.leaves)
        coords = np.empty((ne, 16, 2))
        q = np.arange(16)
        for e, (lev, ix, iy) in enumerate(self.leaves):
            h = self.h(lev)
            coords[e, :, 0] = -self.L + (ix + t[q % 4]) * h
            coords[e, :, 1] = -self.L + (iy + t[q // 4]) * h
        faces, mortars = [], []
        for e, (lev, ix, iy) in enumerate(self.leaves):
            m = self.cells_at(lev)
            # (face, neighbour cell offset, the two finer cells of a refined
            # neighbour that touch this face: lower then upper half)
            for f, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
                nx, ny = (ix + dx) % m, (iy + dy) % m
                nb = (lev, nx, ny)
                if nb in self._index:
                    if f & 1:
                        faces.append((e, f, self._index[nb], f - 1))
                    continue
                if self.leaf_covering(lev, nx, ny) is not None:
                    continue                            # coarser neighbour: its mortar row covers this face
                if f < 2:
                    col = 2 * nx + (1 if f == 0 else 0)   # the neighbour's column next to this face
                    kids = [(lev + 1, col, 2 * ny), (lev + 1, col, 2 * ny + 1)]
                else:
                    row = 2 * ny + (1 if f == 2 else 0)
                    kids = [(lev + 1, 2 * nx, row), (lev + 1, 2 * nx + 1, row)]
                mortars.append((e, f, self._index[kids[0]], self._index[kids[1]]))
        levels = np.array([c[0] for c in self.leaves])
        return (coords, np.asarray(faces, dtype=np.int32).reshape(-1, 4),
                np.asarray(mortars, dtype=np.int32).reshape(-1, 4), levels)


def quadtree_workload(tree, name, E, order, ic="vortex", surface="es_rusanov", seed=0, cfl=0.3, levels_to_parts=None):
    """Workload on a quadtree mesh: partition = refinement level (finest =
    partition 0, Sec. 2.2: the stable step scales with the cell size),
    initial state the translating isentropic vortex or the KHI state."""
    coords, faces, mortars, levels = tree.mesh()
    lmax = int(levels.max())
    part = (lmax - levels).astype(np.int32) if levels_to_parts is None else np.asarray(levels_to_parts(levels), np.int32)
    R = int(part.max()) + 1
    rng = np.random.default_rng(BASE_SEED + 7 + seed)
    x, y = coords[:, :, 0], coords[:, :, 1]
    if ic == "vortex":
        u0 = isentropic_vortex(x, y, 0.0, rng.uniform(-1, 1, 2), float(rng.uniform(3, 5)), L=tree.L, R=1.0)
    else:
        u0 = kelvin_helmholtz(x / tree.L, y / tree.L, phase=float(rng.uniform(0, 2 * math.pi)))
    hmin = tree.h(lmax)
    dt = cfl * hmin / (2 * N_POLY + 1) / 2.5
    return Workload(name, 2, "euler2d", coords, faces, part, list(E[:R]), order, to_soa(u0), dt, "ec_ranocha", surface,
                    info=dict(levels=levels, tree=tree), mortars=mortars)


def amr_marks(tree, alpha, thresholds=(0.01, 0.5), levels=(0, 1, 2)):
    """Three-level controller: the target level of a leaf is levels[2] where
    the indicator is at least thresholds[1], levels[1] where it is at least
    thresholds[0], else levels[0]; leaves below their target are marked for
    refinement, leaves above it for coarsening."""
    ref, coa = [], []
    for c, a in zip(tree.leaves, alpha):
        target = levels[2] if a >= thresholds[1] else (levels[1] if a >= thresholds[0] else levels[0])
        if c[0] < target:
            ref.append(c)
        elif c[0] > target:
            coa.append(c)
    return ref, coa


def quadtree_patch_2d(n=8, L=5.0, patch=0.35, depth=1, E=(6, 3), order=3, ic="vortex", surface="es_rusanov", seed=0):
    """n x n base cells with the cells whose centre lies within patch * L of
    the origin (in the max norm) refined `depth` times: 2:1 mortars around
    each refined band."""
    tree = Quadtree.uniform(n, L)
    for _ in range(depth):
        marks = [c for c in tree.leaves if max(abs(v) for v in tree.centre(c)) < patch * L]
        tree = tree.refine(marks)
    return quadtree_workload(tree, f"quadtree{n}_d{depth}", E, order, ic=ic, surface=surface, seed=seed)


def by_name(name, **kw):
    table = {
        "burgers1d": burgers_1d,
        "vortex2d": vortex_2d,
        "khi2d": khi_2d,
        "tgv3d": tgv_3d,
        "box2d": small_box_2d,
    }
    return table[name](**kw)
