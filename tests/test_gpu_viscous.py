"""GPU parity of the Navier-Stokes-Fourier path (BR1 viscous terms on
entropy-variable gradients, Sec. 4.3.2) against the oracle: the right-hand side
on box, curved and 3D meshes; the multirate stage loop with relaxation under
random partition ids (the gradient set of a stage includes the inactive
neighbours of the active elements); a batch of two instances; entropy decay
and linear invariants."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import dgsem, perrk as operrk, physics

pytestmark = pytest.mark.gpu

TOL = {pk.FP64: 1e-12, pk.MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    __graft_entry__.build()
    torch.zeros(1, device="cuda")


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _phys(wl):
    return physics.Physics(wl.equation, wl.surface_flux, wl.gamma_gas, wl.mu, wl.prandtl)


RHS_CASES = {
    "box": lambda: workloads.small_box_2d(n=8, seed=41, R=2, E=[6, 3], order=3, mu=0.05),
    "curved": lambda: workloads.vortex_2d(n=12, mu=0.02),
    "tgv": lambda: workloads.tgv_3d(n=4, n_fine=2, mu=0.01),
    "shock": lambda: workloads.viscous_shock_2d(n=8, angle=0.6),
}


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
@pytest.mark.parametrize("name", list(RHS_CASES))
def test_viscous_rhs_parity(name, precision):
    import torch
    wl = RHS_CASES[name]()
    rng = np.random.default_rng(43)
    u = wl.u0 * (1.0 + 0.02 * rng.standard_normal(wl.u0.shape))
    geo = dgsem.Geometry(wl.coords, wl.faces)
    K_ref = dgsem.rhs(geo, _phys(wl), u)
    Kv_ref = dgsem.viscous_rhs(geo, _phys(wl), u)
    s = pk.Solver(wl, pk.options(precision=precision))
    ud = torch.tensor(u, device="cuda")
    kd = torch.empty_like(ud)
    pk.perrk_rhs(s.h, ud.data_ptr(), kd.data_ptr())
    torch.cuda.synchronize()
    K = kd.cpu().numpy()
    s.close()
    err = rel_linf(K, K_ref)
    assert np.abs(Kv_ref).max() > 1e-3 * np.abs(K_ref).max()     # the viscous part is not negligible
    assert err < (1e-12 if precision == pk.FP64 else 2e-5), err


def oracle_run(wl, nsteps, **kw):
    s = operrk.Solver(wl, operrk.NewtonOptions(**kw))
    recs = []
    for _ in range(nsteps):
        u0 = s.U.copy()
        r = s.step(wl.dt)
        r.du_inf = float(np.abs(s.U - u0).max())
        recs.append(r)
    return s, recs


def gamma_explained_tol(grec, rrec, u_ref, base=1e-12):
    """A gamma difference dg_n (rounding in Delta H, amplified by the
    relaxation root's conditioning) moves the state by dg_n dt |d_n|; the rest
    must agree to `base`."""
    scale = float(np.abs(u_ref).max())
    extra = sum(abs(a["gamma"] - b.gamma) * b.du_inf / b.gamma for a, b in zip(grec, rrec))
    return base + 1.5 * extra / scale


STEP_CASES = {
    "box_p2_random": lambda: workloads.small_box_2d(n=6, seed=44, R=3, E=[6, 4, 2], order=2, random_parts=True,
                                                    mu=0.05),
    "box_p3_graded": lambda: workloads.small_box_2d(n=8, seed=45, R=2, E=[6, 3], order=3, mu=0.05),
    "box_p4_random": lambda: workloads.small_box_2d(n=6, seed=46, R=3, E=[8, 6, 5], order=4, random_parts=True,
                                                    mu=0.05),
    "curved_p3": lambda: workloads.vortex_2d(n=12, E=(8, 5, 3), mu=0.02),
    "tgv_p3": lambda: workloads.tgv_3d(n=4, n_fine=2, mu=0.01),
}


def gpu_run(wl, nsteps, precision, relax=True, target=pk.TARGET_DELTA_H):
    opts = pk.options(precision=precision, relaxation=relax, max_it=10, tol_r=1e-14, tol_g=1e-14, target=target)
    s = pk.Solver(wl, opts)
    recs = s.step(nsteps)
    u = s.state()
    s.close()
    return u, [r[0] for r in recs]


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
@pytest.mark.parametrize("case", list(STEP_CASES))
def test_viscous_stage_loop_parity_unrelaxed(case, precision):
    wl = STEP_CASES[case]()
    n = 6 if case != "tgv_p3" else 3
    ref, _ = oracle_run(wl, n, relax=False)
    u, _ = gpu_run(wl, n, precision, relax=False)
    assert rel_linf(u, ref.U) < TOL[precision]


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
@pytest.mark.parametrize("case", list(STEP_CASES))
def test_viscous_step_parity(case, precision):
    wl = STEP_CASES[case]()
    n = 6 if case != "tgv_p3" else 3
    ref, rrec = oracle_run(wl, n)
    u, grec = gpu_run(wl, n, precision)
    err = rel_linf(u, ref.U)
    tol = gamma_explained_tol(grec, rrec, ref.U) if precision == pk.FP64 else TOL[precision]
    assert err < tol, (case, err, tol)
    for a, b in zip(grec, rrec):
        assert abs(a["gamma"] - b.gamma) < (1e-7 if precision == pk.FP64 else 5e-4)
        assert b.dH < 0.0                       # viscous dissipation
        assert a["flags"] & pk.FLAG_NONPHYSICAL == 0


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_viscous_batched_parity(precision):
    """Two instances of different sizes, partitions and viscosity-free
    inviscid settings shared (one context holds one viscosity)."""
    wls = [workloads.small_box_2d(n=6, seed=47, R=3, E=[6, 4, 3], order=3, random_parts=True, mu=0.05),
           workloads.small_box_2d(n=4, seed=48, R=2, E=[6, 3], order=3, mu=0.05)]
    s = pk.Solver(wls, pk.options(precision=precision, max_it=10, tol_r=1e-14, tol_g=1e-14))
    s.step(4)
    u = s.state()
    s.close()
    off = 0
    for wl in wls:
        ref, rrec = oracle_run(wl, 4)
        ue = u[:, off:off + wl.n_elem]
        off += wl.n_elem
        assert rel_linf(ue, ref.U) < (1e-9 if precision == pk.FP64 else TOL[precision])


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_viscous_entropy_decay_and_invariants(precision):
    """EC fluxes plus BR1: the only entropy change is viscous dissipation, so
    H decreases every step; mass, momentum and energy stay conserved."""
    wl = workloads.small_box_2d(n=8, seed=49, R=2, E=[6, 3], order=3, surface="ec", random_parts=True, mu=0.05)
    geo = dgsem.Geometry(wl.coords, wl.faces)
    u, grec = gpu_run(wl, 8, precision)
    for r in grec:
        assert r["dH"] < 0.0 and r["H_next"] < r["H_n"]
    tol = 1e-13 if precision == pk.FP64 else 1e-8
    for v in range(4):
        m0, m1 = geo.integrate(wl.u0[v]), geo.integrate(u[v])
        assert abs(m1 - m0) < tol * (abs(m0) + 1.0)


def _edge_case(name):
    if name == "one_element":
        # one periodic element: every face pairs it with itself, and its
        # gradient uses its own opposite face traces
        return workloads.small_box_2d(n=1, seed=71, R=1, E=[4], order=2, mu=0.05)
    if name == "empty_partition":
        # member 1 owns no element: no stage has a ring from it
        wl = workloads.small_box_2d(n=6, seed=72, R=2, E=[6, 3], order=3, mu=0.05)
        wl.part = np.zeros_like(wl.part)
        return wl
    if name == "ragged_prefix":
        # random partitions: prefixes and rings of every size, none a
        # multiple of the elements per CTA
        return workloads.small_box_2d(n=7, seed=73, R=3, E=[8, 6, 3], order=3, random_parts=True, mu=0.05)
    raise KeyError(name)


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
@pytest.mark.parametrize("name", ["one_element", "empty_partition", "ragged_prefix"])
def test_viscous_edge_case_meshes(name, precision):
    wl = _edge_case(name)
    ref, rrec = oracle_run(wl, 4)
    tested = 0
    for variant in (0, 1):
        for epb in (4, 8, 16):
            s = pk.Solver(wl, pk.options(precision=precision, max_it=10, tol_r=1e-14, tol_g=1e-14))
            pk.perrk_set_tuning(s.h, epb, 0, 128, variant)
            try:
                recs = [r[0] for r in s.step(4)]
            except pk.PerrkError as err:
                assert "invalid configuration" in str(err)      # a mapping whose shared memory does not fit
                s.close()
                continue
            u = s.state()
            s.close()
            tested += 1
            tol = gamma_explained_tol(recs, rrec, ref.U) if precision == pk.FP64 else TOL[precision]
            assert rel_linf(u, ref.U) < tol, (name, variant, epb, rel_linf(u, ref.U), tol)
    assert tested >= 2
