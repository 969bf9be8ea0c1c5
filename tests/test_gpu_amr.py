"""Adaptive mesh refinement on the GPU against the oracle: the refinement
indicator, the solution transfer, the package's quadtree adaptation (exact
against the generator's) and whole adaptive runs (Sec. 3.2.2: the mesh
changes every few steps and the partitions follow the new element sizes)."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
from paper_2507_04991_gb300 import amr as pamr
import workloads
from oracle import amr as oamr, dgsem, perrk as operrk
from test_gpu_parity import gamma_explained_tol, rel_linf

pytestmark = pytest.mark.gpu

E_BY_OFFSET = [12, 6, 3]
MAX_LEVEL = 2
THRESH = (0.3, 0.9)
LEVELS = (0, 1, 2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _dt(n=8, L=1.0):
    h_min = 2 * L / (n << MAX_LEVEL)
    return 0.3 * h_min / 7 / 2.5


def _oracle_workload(tree, U, dt, surface="es_rusanov"):
    coords, faces, mortars, levels = tree.mesh()
    return workloads.Workload("amr", 2, "euler2d", coords, faces, (MAX_LEVEL - levels).astype(np.int32),
                              list(E_BY_OFFSET), 3, U, dt, "ec_ranocha", surface, mortars=mortars)


def _same_mesh(pmesh, tree, pmap=None, omap=None):
    assert pmesh.leaves == tree.leaves
    pc, pf, pm = pmesh.arrays()
    oc, of, om, _ = tree.mesh()
    assert np.abs(pc - oc).max() == 0.0
    assert sorted(map(tuple, pf)) == sorted(map(tuple, of))
    assert sorted(map(tuple, pm)) == sorted(map(tuple, om))
    if pmap is not None:
        assert np.array_equal(pmap, omap)


def test_indicator_matches_oracle():
    tree = workloads.Quadtree.uniform(8, 1.0)
    wl = workloads.quadtree_workload(tree, "khi", (3,), 3, ic="khi")
    rng = np.random.default_rng(2)
    for U in (wl.u0, wl.u0 * (1 + 0.05 * rng.standard_normal(wl.u0.shape))):
        wl.u0 = U
        for prec in (pk.FP64, pk.MIXED):
            s = pk.Solver(wl, pk.options(precision=prec))
            a_dev = pk.perrk_amr_indicator(s.h)
            s.close()
            a_ref = oamr.indicator(U[0])
            tol = 1e-9 if prec == pk.FP64 else 1e-3
            assert np.abs(a_dev - a_ref).max() <= tol, np.abs(a_dev - a_ref).max()


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_transfer_matches_oracle(precision):
    tree = workloads.Quadtree.uniform(8, 1.0)
    wl = workloads.quadtree_workload(tree, "khi", (3,), 3, ic="khi")
    dt = _dt()
    U = wl.u0
    for cycle in range(3):
        alpha = oamr.indicator(U[0])
        ref, coa = workloads.amr_marks(tree, alpha, THRESH, LEVELS)
        if cycle == 2:
            ref, coa = [], [c for c in tree.leaves if c[0] > 0]
        new, amap = tree.adapt(ref, coa)
        src = pk.Solver(_oracle_workload(tree, U, dt), pk.options(precision=precision))
        dst = pk.Solver(_oracle_workload(new, np.zeros((4, len(new.leaves), 16)), dt), pk.options(precision=precision))
        pk.perrk_amr_transfer(src.h, dst.h, amap)
        got = dst.state()
        src.close()
        dst.close()
        U = oamr.transfer(U, amap)
        assert rel_linf(got, U) <= (1e-14 if precision == pk.FP64 else 1e-7)
        tree = new


def test_transfer_rejects_bad_maps():
    tree = workloads.Quadtree.uniform(4, 1.0)
    wl = workloads.quadtree_workload(tree, "v", (3,), 3)
    a = pk.Solver(wl)
    b = pk.Solver(wl)
    m = np.zeros((wl.n_elem, 5), np.int32)
    m[:, 1] = np.arange(wl.n_elem)
    m[3, 1] = wl.n_elem
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_amr_transfer(a.h, b.h, m)
    assert ei.value.status == pk.PERRK_INVALID_ARG
    a.close()
    b.close()


def test_adaptive_run_matches_oracle():
    """Three adaptation cycles of four relaxed float64 steps each on a KHI
    state: the device run (package AMR driver) and the oracle run take the
    same decisions, reach the same state, and keep mass to round-off."""
    dt = _dt()
    tree = workloads.Quadtree.uniform(8, 1.0)
    wl0 = workloads.quadtree_workload(tree, "khi", (3,), 3, ic="khi")
    opts = pk.options(precision=pk.FP64)
    run = pamr.AmrRun(pamr.QuadMesh.uniform(8, 1.0), wl0.u0, E_BY_OFFSET, 3, dt, opts, MAX_LEVEL)
    U = wl0.u0.copy()
    t, g_prev = 0.0, 1.0
    geo0 = dgsem.Geometry(wl0.coords, wl0.faces)
    m0 = geo0.integrate(U[0])
    grec_all, rrec_all = [], []
    for cycle in range(3):
        alpha, pref, pcoa, pmap = run.adapt(THRESH, LEVELS)
        a_ref = oamr.indicator(U[0])
        assert np.abs(alpha - a_ref).max() <= 1e-9
        ref, coa = workloads.amr_marks(tree, a_ref, THRESH, LEVELS)
        assert sorted(ref) == sorted(pref) and sorted(coa) == sorted(pcoa)
        tree, omap = tree.adapt(ref, coa)
        _same_mesh(run.mesh, tree, pmap, omap)
        U = oamr.transfer(U, omap)
        wl = _oracle_workload(tree, U, dt)
        o = operrk.Solver(wl)
        o.t, o.gamma_prev = t, g_prev
        rrec = []
        for _ in range(4):
            before = o.U.copy()
            r = o.step(dt)
            r.du_inf = float(np.abs(o.U - before).max())     # gamma dt |d|_inf, for the explained bound
            rrec.append(r)
        grec = [r[0] for r in run.step(4)]
        U, t, g_prev = o.U, o.t, o.gamma_prev
        grec_all += grec
        rrec_all += rrec
        for a, b in zip(grec, rrec):
            assert a["flags"] == 0 and b.converged
        assert rel_linf(run.state(), U) < gamma_explained_tol(grec_all, rrec_all, U)
        # t accumulates gamma dt: it differs by the gamma differences the root's conditioning explains
        dt_explained = sum(abs(a["gamma"] - b.gamma) for a, b in zip(grec_all, rrec_all)) * dt
        assert abs(grec[-1]["t"] - t) < 1e-14 + 1.5 * dt_explained
    coords, faces, mortars, _ = tree.mesh()
    geo = dgsem.Geometry(coords, faces, mortars=mortars)
    assert abs(geo.integrate(run.state()[0]) - m0) <= 1e-13 * abs(m0)
    assert len(mortars) > 0
    print("adaptation seconds", run.adapt_seconds)
    run.close()


def test_adaptive_run_mixed_conserves():
    """The mixed form under adaptation (its own indicator decisions): no
    flags, and mass kept to the FP32 rounding of its flux arithmetic: the
    stage registers K_i carry ~6e-8 relative rounding of the flux terms,
    so twelve steps of dt ~ 1e-3 move the total mass by ~1e-10 of itself
    (float64 keeps it to 1e-13, test_adaptive_run_matches_oracle)."""
    dt = _dt()
    wl0 = workloads.quadtree_workload(workloads.Quadtree.uniform(8, 1.0), "khi", (3,), 3, ic="khi")
    run = pamr.AmrRun(pamr.QuadMesh.uniform(8, 1.0), wl0.u0, E_BY_OFFSET, 3, dt, pk.options(precision=pk.MIXED),
                      MAX_LEVEL)
    geo0 = dgsem.Geometry(wl0.coords, wl0.faces)
    m0 = geo0.integrate(wl0.u0[0])
    for cycle in range(3):
        run.adapt(THRESH, LEVELS)
        assert all(r[0]["flags"] == 0 for r in run.step(4))
    coords, faces, mortars = run.mesh.arrays()
    geo = dgsem.Geometry(coords, faces, mortars=mortars)
    assert abs(geo.integrate(run.state()[0]) - m0) <= 1e-8 * abs(m0)
    run.close()
