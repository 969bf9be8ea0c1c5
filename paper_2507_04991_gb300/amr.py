"""Adaptive mesh refinement for the P-ERRK stage loop on 2D quadtree meshes.

The paper runs its multirate schemes on adaptively refined meshes (Sec.
3.2.2, Sec. 5.3): every few steps the mesh is refined where the
shock-capturing indicator of Hennemann et al. on the density is large and
coarsened where it is small, the solution is carried to the new mesh, and the
partitions are re-derived from the new element sizes (Sec. 2.2: a cell of
half the size gets the member with twice the stage evaluations).  Interfaces
between cells of different levels are 2:1 mortars.

The quadtree with its 2:1 balance, its adaptation and the mesh arrays of the
C ABI are the library's native host code (perrk_quadtree_*); this module adds
the three-level controller, the partition ids and the driver.  The two
computations on the state run in the library's kernels: the indicator
(perrk_amr_indicator) and the transfer (perrk_amr_transfer).

Canonical orders: leaves sorted by (level, ix, iy); a leaf's cell is
[-L + ix h, -L + (ix + 1) h] x [-L + iy h, ...], h = 2L / (n 2^level), on the
periodic square [-L, L]^2 over an n x n base grid.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import Solver, _check, _ptr, load as _lib, perrk_amr_indicator, perrk_amr_transfer, perrk_set_dt


class QuadMesh:
    """A 2:1-balanced periodic quadtree (see the module docstring), held by
    the library's native quadtree (perrk_quadtree_*).  `leaves` lists
    (level, ix, iy) in the canonical order; adapt() hands the native tree on
    to the mesh it returns."""

    def __init__(self, n, L, handle):
        self.n, self.L = int(n), float(L)
        self._h = handle
        cnt = _lib().perrk_quadtree_size(handle)
        buf = np.empty((cnt, 3), dtype=np.int32)
        _check(_lib().perrk_quadtree_leaves(handle, _ptr(buf)), "perrk_quadtree_leaves")
        self.leaf_array = buf                      # [n_leaves][3] = (level, ix, iy)
        self._leaves = None
        self._pos = None

    def __len__(self):
        return len(self.leaf_array)

    @property
    def leaves(self):
        """(level, ix, iy) tuples in the canonical order (built on first use)."""
        if self._leaves is None:
            self._leaves = [tuple(r) for r in self.leaf_array.tolist()]
        return self._leaves

    @property
    def pos(self):
        if self._pos is None:
            self._pos = {c: k for k, c in enumerate(self.leaves)}
        return self._pos

    @classmethod
    def uniform(cls, n, L):
        h = C.c_void_p()
        _check(_lib().perrk_quadtree_create(int(n), float(L), C.byref(h)), "perrk_quadtree_create")
        return cls(n, L, h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib().perrk_quadtree_destroy(h)
            except Exception:
                pass
            self._h = None

    def size(self, lev):
        return 2.0 * self.L / (self.n << lev)

    def owner(self, lev, i, j):
        """Leaf containing cell (lev, i, j) (periodic), or None where that cell is split."""
        m = self.n << lev
        i, j = i % m, j % m
        while lev >= 0:
            if (lev, i, j) in self.pos:
                return (lev, i, j)
            lev, i, j = lev - 1, i // 2, j // 2
        return None

    def adapt(self, refine, coarsen):
        """New mesh and the map of its leaves (rows kind, a0..a3 as in
        perrk_amr_transfer): families all marked for coarsening (and none of
        whose members is marked for refinement) merge unless that breaks the
        balance, marked leaves split, and the balance is restored.  This
        mesh object is spent (the native tree moves to the new one)."""
        marks = np.zeros(len(self), dtype=np.int8)
        for c in coarsen:
            marks[self.pos[c]] = -1
        for c in refine:
            marks[self.pos[c]] = 1
        return self.adapt_marks(marks)

    def adapt_marks(self, marks):
        """adapt() with the marks as an array over the leaves (+1 refine,
        -1 coarsen, 0 keep)."""
        if not self._h:
            raise RuntimeError("this quadtree mesh was already adapted")
        marks = np.ascontiguousarray(marks, dtype=np.int8)
        cap = 4 * len(self)
        amap = np.empty((cap, 5), dtype=np.int32)
        n_new = C.c_int(0)
        _check(_lib().perrk_quadtree_adapt(self._h, _ptr(marks), _ptr(amap), cap, C.byref(n_new)),
               "perrk_quadtree_adapt")
        h, self._h = self._h, None
        return QuadMesh(self.n, self.L, h), amap[:n_new.value].copy()

    def levels(self):
        return self.leaf_array[:, 0].copy()

    def arrays(self):
        """(node coordinates [n_elem, 16, 2], conforming faces [n, 4],
        mortars [n, 4]) in the conventions of perrk_mesh_desc."""
        lib = _lib()
        nf, nm = C.c_int(0), C.c_int(0)
        _check(lib.perrk_quadtree_mesh(self._h, None, None, C.byref(nf), None, C.byref(nm), None), "perrk_quadtree_mesh")
        coords = np.empty((len(self), 16, 2))
        faces = np.empty((nf.value, 4), dtype=np.int32)
        mortars = np.empty((nm.value, 4), dtype=np.int32)
        _check(lib.perrk_quadtree_mesh(self._h, _ptr(coords), _ptr(faces) if nf.value else None, C.byref(nf),
                                       _ptr(mortars) if nm.value else None, C.byref(nm), None), "perrk_quadtree_mesh")
        return coords, faces, mortars


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


def controller_marks(mesh, alpha, thresholds=(0.01, 0.5), levels=(0, 1, 2)):
    """The controller's decisions as marks over the leaves (+1 refine,
    -1 coarsen, 0 keep), vectorised."""
    a = np.asarray(alpha)
    target = np.where(a >= thresholds[1], levels[2], np.where(a >= thresholds[0], levels[1], levels[0]))
    lev = mesh.leaf_array[:, 0]
    return np.where(lev < target, 1, np.where(lev > target, -1, 0)).astype(np.int8)


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
        marks = controller_marks(self.mesh, alpha, thresholds, levels)
        leaves = self.mesh.leaf_array
        new, amap = self.mesh.adapt_marks(marks)
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
        ref = [tuple(c) for c in leaves[marks > 0].tolist()]
        coa = [tuple(c) for c in leaves[marks < 0].tolist()]
        return alpha, ref, coa, amap

    def state(self):
        return self.solver.state()

    def close(self):
        self.solver.close()
