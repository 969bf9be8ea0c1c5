"""Adaptive mesh refinement for the P-ERRK stage loop on 2D quadtree meshes.

The paper runs its multirate schemes on adaptively refined meshes (Sec.
3.2.2, Sec. 5.3): every few steps the mesh is refined where the
shock-capturing indicator of Hennemann et al. on the density is large and
coarsened where it is small, the solution is carried to the new mesh, and the
partitions are re-derived from the new element sizes (Sec. 2.2: a cell of
half the size gets the member with twice the stage evaluations).  Interfaces
between cells of different levels are 2:1 mortars.

Host logic only (argument preparation for the library): the quadtree with
its 2:1 balance, the three-level controller, the mesh arrays of the C ABI and
the partition ids.  The two computations on the state run in the library's
kernels: the indicator (perrk_amr_indicator) and the transfer
(perrk_amr_transfer).

Canonical orders: leaves sorted by (level, ix, iy); a leaf's cell is
[-L + ix h, -L + (ix + 1) h] x [-L + iy h, ...], h = 2L / (n 2^level), on the
periodic square [-L, L]^2 over an n x n base grid.
"""
from __future__ import annotations

import math

import numpy as np

from . import Solver, perrk_amr_indicator, perrk_amr_transfer, perrk_set_dt

_LGL = np.array([-1.0, -1.0 / math.sqrt(5.0), 1.0 / math.sqrt(5.0), 1.0])


class QuadMesh:
    """A 2:1-balanced periodic quadtree (see the module docstring)."""

    def __init__(self, n, L, leaves):
        self.n, self.L = int(n), float(L)
        self.leaves = sorted(set(leaves))
        self.pos = {c: k for k, c in enumerate(self.leaves)}

    @classmethod
    def uniform(cls, n, L):
        return cls(n, L, [(0, i, j) for i in range(n) for j in range(n)])

    def size(self, lev):
        return 2.0 * self.L / (self.n << lev)

    def _wrap(self, lev, i, j):
        m = self.n << lev
        return lev, i % m, j % m

    def owner(self, lev, i, j, leaves=None):
        """Leaf containing cell (lev, i, j), or None where that cell is split."""
        leaves = self.pos if leaves is None else leaves
        lev, i, j = self._wrap(lev, i, j)
        while lev >= 0:
            if (lev, i, j) in leaves:
                return (lev, i, j)
            lev, i, j = lev - 1, i // 2, j // 2
        return None

    @staticmethod
    def _children(c):
        lev, i, j = c
        return [(lev + 1, 2 * i + (k & 1), 2 * j + (k >> 1)) for k in range(4)]   # child index a + 2 b

    def _balance(self, leaves):
        """Split leaves until no face neighbour is two levels finer."""
        leaves = set(leaves)
        queue = sorted(leaves, reverse=True)
        while queue:
            c = queue.pop()
            if c not in leaves:
                continue
            lev, i, j = c
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                o = self.owner(lev, i + di, j + dj, leaves)
                if o is not None and o[0] < lev - 1:
                    leaves.discard(o)
                    kids = self._children(o)
                    leaves.update(kids)
                    queue.extend(kids)
                    queue.append(c)
        return leaves

    def adapt(self, refine, coarsen):
        """New mesh and the map of its leaves (rows kind, a0..a3 as in
        perrk_amr_transfer): families all marked for coarsening (and none of
        whose members is marked for refinement) merge unless that breaks the
        balance, marked leaves split, and the balance is restored."""
        refine = set(refine)
        coarsen = set(coarsen) - refine
        leaves = set(self.leaves)
        parents = sorted({(l - 1, i // 2, j // 2) for (l, i, j) in coarsen if l > 0}, reverse=True)
        for p in parents:
            kids = self._children(p)
            if not all(k in leaves and k in coarsen for k in kids):
                continue
            trial = (leaves - set(kids)) | {p}
            if self._balance(trial) == trial:
                leaves = trial
        for c in refine:
            if c in leaves:
                leaves.discard(c)
                leaves.update(self._children(c))
        new = QuadMesh(self.n, self.L, self._balance(leaves))
        rows = []
        for c in new.leaves:
            if c in self.pos:
                rows.append((0, self.pos[c], 0, 0, 0))
                continue
            lev, i, j = c
            par = (lev - 1, i // 2, j // 2)
            if lev > 0 and par in self.pos:
                rows.append((1, self.pos[par], (i & 1) + 2 * (j & 1), 0, 0))
                continue
            kids = self._children(c)
            if not all(k in self.pos for k in kids):
                raise ValueError("a leaf changed by more than one level in one adaptation")
            rows.append((2,) + tuple(self.pos[k] for k in kids))
        return new, np.asarray(rows, dtype=np.int32).reshape(-1, 5)

    def levels(self):
        return np.array([c[0] for c in self.leaves], dtype=np.int32)

    def arrays(self):
        """(node coordinates [n_elem, 16, 2], conforming faces [n, 4],
        mortars [n, 4]) in the conventions of perrk_mesh_desc."""
        t = 0.5 * (_LGL + 1.0)
        q = np.arange(16)
        coords = np.empty((len(self.leaves), 16, 2))
        faces, mortars = [], []
        for e, (lev, i, j) in enumerate(self.leaves):
            h = self.size(lev)
            coords[e, :, 0] = -self.L + (i + t[q & 3]) * h
            coords[e, :, 1] = -self.L + (j + t[q >> 2]) * h
            # face 0: -x, 1: +x, 2: -y, 3: +y
            for f, (di, dj) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
                nb = self._wrap(lev, i + di, j + dj)
                if nb in self.pos:
                    if f % 2 == 1:
                        faces.append((e, f, self.pos[nb], f - 1))
                    continue
                o = self.owner(*nb)
                if o is not None:
                    continue                          # a coarser neighbour lists this face in its mortar row
                ni, nj = nb[1], nb[2]
                if f in (0, 1):                       # the finer column touching this face, lower y first
                    ci = 2 * ni + (1 if f == 0 else 0)
                    pair = ((lev + 1, ci, 2 * nj), (lev + 1, ci, 2 * nj + 1))
                else:                                 # the finer row touching this face, lower x first
                    cj = 2 * nj + (1 if f == 2 else 0)
                    pair = ((lev + 1, 2 * ni, cj), (lev + 1, 2 * ni + 1, cj))
                mortars.append((e, f, self.pos[pair[0]], self.pos[pair[1]]))
        return (coords, np.asarray(faces, dtype=np.int32).reshape(-1, 4),
                np.asarray(mortars, dtype=np.int32).reshape(-1, 4))


def controller(mesh, alpha, thresholds=(0.01, 0.5), levels=(0, 1, 2)):
    """Three-level controller: target level levels[2] where alpha >=
    thresholds[1], levels[1] where alpha >= thresholds[0], else levels[0];
    returns (leaves to refine, leaves to coarsen)."""
    ref, coa = [], []
    for c, a in zip(mesh.leaves, alpha):
        target = levels[2] if a >= thresholds[1] else (levels[1] if a >= thresholds[0] else levels[0])
        if c[0] < target:
            ref.append(c)
        elif c[0] > target:
            coa.append(c)
    return ref, coa


class _Problem:
    """The fields Solver reads (a workload-like record)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def partitions(levels, max_level):
    """Partition id of each element: the finest level allowed is partition
    0 (most stage evaluations), one partition per level coarser."""
    return (max_level - np.asarray(levels)).astype(np.int32)


class AmrRun:
    """A P-ERRK run on an adaptive quadtree mesh: one library context per
    mesh; adapt() evaluates the indicator on the device, adapts the mesh,
    creates the context of the new mesh (partitions from the levels) and
    carries the state over on the device.  E_by_offset[r] is the stage
    count of partition r = max_level - level; dt is the caller's and stays
    fixed (it is limited by the finest level allowed)."""

    def __init__(self, mesh, u0, E_by_offset, order, dt, opts, max_level, surface="es_rusanov", gamma_gas=1.4,
                 tableaux=None):
        self.mesh, self.E, self.order, self.dt, self.opts = mesh, list(E_by_offset), order, dt, opts
        self.max_level, self.surface, self.gamma_gas = max_level, surface, gamma_gas
        self.solver = self._solver(mesh, u0)
        self.adapt_seconds = 0.0
        self.adapt_parts = {"indicator": 0.0, "mesh": 0.0, "context": 0.0, "transfer": 0.0}

    def _problem(self, mesh, u0=None):
        coords, faces, mortars = mesh.arrays()
        return _Problem(coords=coords, faces=faces, mortars=mortars, part=partitions(mesh.levels(), self.max_level),
                        E=self.E, order=self.order, equation="euler2d", surface_flux=self.surface,
                        gamma_gas=self.gamma_gas, dt=self.dt, u0=u0)

    def _solver(self, mesh, u0=None):
        return Solver(self._problem(mesh, u0), self.opts)

    def step(self, nsteps=1, info=True, stream=0):
        return self.solver.step(nsteps, info, stream)

    def adapt(self, thresholds=(0.01, 0.5), levels=None):
        """One adaptation; returns (alpha on the old mesh, refine marks,
        coarsen marks, transfer map)."""
        import time
        t0 = time.perf_counter()
        levels = levels or (0, max(0, self.max_level - 1), self.max_level)
        alpha = perrk_amr_indicator(self.solver.h)
        t1 = time.perf_counter()
        ref, coa = controller(self.mesh, alpha, thresholds, levels)
        new, amap = self.mesh.adapt(ref, coa)
        t2 = time.perf_counter()
        nxt = self._solver(new)
        perrk_set_dt(nxt.h, self.dt)
        t3 = time.perf_counter()
        perrk_amr_transfer(self.solver.h, nxt.h, amap)
        self.solver.close()
        self.solver, self.mesh = nxt, new
        t4 = time.perf_counter()
        for k, v in zip(("indicator", "mesh", "context", "transfer"), (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
            self.adapt_parts[k] += v
        self.adapt_seconds += t4 - t0
        return alpha, ref, coa, amap

    def state(self):
        return self.solver.state()

    def close(self):
        self.solver.close()
