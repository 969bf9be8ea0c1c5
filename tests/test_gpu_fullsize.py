"""Parity at the full configuration sizes, in the launch configuration the
bench uses (autotuned mapping, CUDA graph, mixed form): sampled outputs that
the oracle computes element by element, and invariants that hold at any size.

* batched (256 instances, 1.04e8 DOF): the smallest instances against oracle
  runs, linear invariants of every instance;
* KHI 256^2 (4.2M DOF) and TGV 64^3 (84M DOF): the right-hand side at sampled
  elements against the oracle on a local patch (the sampled elements and their
  face neighbours), and one or two steps' invariants."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import dgsem, perrk as operrk, physics
from oracle.lgl import lgl as lgl_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _patch_rhs(wl, u, sample):
    """Oracle RHS at the sampled elements: a patch of the sampled elements and
    their face neighbours, with the faces that touch sampled elements."""
    faces = wl.faces
    touch = np.isin(faces[:, 0], sample) | np.isin(faces[:, 2], sample)
    fsel = faces[touch]
    patch = np.unique(np.concatenate([sample, fsel[:, 0], fsel[:, 2]]))
    loc = {int(e): i for i, e in enumerate(patch)}
    lf = np.array([[loc[int(a)], b, loc[int(c)], d] for a, b, c, d in fsel], dtype=np.int32)
    geo = dgsem.Geometry(wl.coords[patch], lf)
    ph = physics.Physics(wl.equation, wl.surface_flux)
    K = dgsem.rhs(geo, ph, u[:, patch])
    return K[:, [loc[int(e)] for e in sample]]


def _device_rhs(wl, u, precision):
    import torch
    s = pk.Solver(wl, pk.options(precision=precision))
    ud = torch.tensor(u, device="cuda")
    kd = torch.empty_like(ud)
    pk.perrk_rhs(s.h, ud.data_ptr(), kd.data_ptr())
    torch.cuda.synchronize()
    s.close()
    return kd


def _term_scale(wl, sample):
    """Per sampled element, the magnitude of the terms whose sum is the
    right-hand side on a box element: max |f(u)| over the element's nodes (any
    direction, any variable) times (2/h) (dim ||D||_inf + 1/w_0), the largest
    volume plus surface contribution before the cancellations that leave
    dU/dt.  Returns (T_e, ||D||_inf, h_e)."""
    x, w, D = lgl_nodes(3)
    u = wl.u0[:, sample]
    d = wl.dim
    rho = u[0]
    v = u[1:1 + d] / rho
    p = (wl.gamma_gas - 1.0) * (u[-1] - 0.5 * rho * np.sum(v * v, axis=0))
    F = np.maximum(np.abs(u[1:1 + d]).max(axis=(0, 2)),
                   np.maximum(np.abs(rho * v[:, None] * v[None]).max(axis=(0, 1, 3)) + np.abs(p).max(axis=1),
                              np.abs((u[-1] + p) * v).max(axis=(0, 2))))
    h = np.min([wl.coords[sample, 3 * 4 ** a, a] - wl.coords[sample, 0, a] for a in range(d)], axis=0)
    Dn = float(np.abs(D).sum(axis=1).max())
    return F * (2.0 / h) * (d * Dn + 1.0 / w[0]), Dn, h


@pytest.mark.parametrize("name", ["khi", "tgv"])
def test_fullsize_rhs_sampled(name):
    """Sampled right-hand side at full size against the oracle.

    Tolerances follow from the conditioning of flux differencing, not from the
    size of dU/dt: the sum over a node's volume and surface terms of magnitude
    T (``_term_scale``) cancels to |dU/dt| << T (T/|dU/dt| ~ 1e4 for KHI 256^2,
    ~5e5 for the Mach 0.1 TGV, whose pressure flux is ~250).
    * float64: the library takes a box element's metric from its first node,
      the oracle evaluates D x at every node; both carry the rounding of the
      node coordinates, eps |x|_max / (h/2) ||D||_inf relative, which the
      cancellation amplifies by T.  The bound is that metric error times T.
    * mixed (FP32 fluxes): each two-point flux carries a few FP32 ulps, so the
      bound is 8 * 2^-24 * T.  Times dt this is the size of the FP32 rounding
      of U itself."""
    wl = workloads.khi_2d(n=256) if name == "khi" else workloads.tgv_3d(n=64)
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(wl.n_elem, 48, replace=False))
    u = wl.u0
    K_ref = _patch_rhs(wl, u, sample)
    T, Dn, h = _term_scale(wl, sample)
    xmax = float(np.abs(wl.coords).max())
    tol = {pk.FP64: 2.0 ** -52 * xmax / (h / 2.0) * Dn * T, pk.MIXED: 8.0 * 2.0 ** -24 * T}
    ratio = {}
    for prec in (pk.FP64, pk.MIXED):
        kd = _device_rhs(wl, u, prec)
        K = kd[:, sample].cpu().numpy()
        del kd
        err = np.abs(K - K_ref).max(axis=(0, 2))            # per sampled element
        ratio[prec] = float((err / tol[prec]).max())
        k = int(np.argmax(err / tol[prec]))
        print(f"{name} precision {prec}: worst element err {err[k]:.3e} tol {tol[prec][k]:.3e} "
              f"T {T[k]:.3e} max|K| {np.abs(K_ref[:, k]).max():.3e}; max err {err.max():.3e}")
    assert ratio[pk.FP64] < 1.0 and ratio[pk.MIXED] < 1.0, (name, ratio)


@pytest.mark.parametrize("name", ["khi", "tgv"])
def test_fullsize_steps_invariants(name):
    """Mixed form, bench launch configuration (autotuned, graph): mass to FP32
    round-off, entropy non-increasing with ES fluxes (KHI) or kept to 1e-12
    with EC fluxes and the H_{n+1} = H_n target (TGV)."""
    wl = workloads.khi_2d(n=256) if name == "khi" else workloads.tgv_3d(n=64)
    target = pk.TARGET_DELTA_H if name == "khi" else pk.TARGET_PREV
    s = pk.Solver(wl, pk.options(precision=pk.MIXED, use_graph=True, target=target))
    pk.perrk_autotune(s.h)
    s.set_state(wl.u0)
    recs = [r[0] for r in s.step(2)]
    u = s.state()
    s.close()
    # omega J from the oracle's geometry on box elements: per-element constant Jacobian
    w1 = np.array([1.0, 5.0, 5.0, 1.0]) / 6.0
    d = wl.dim
    wq = w1 if d == 1 else (np.outer(w1, w1).ravel() if d == 2 else np.einsum("k,j,i->kji", w1, w1, w1).ravel())
    ext = [wl.coords[:, 3 * 4 ** a, a] - wl.coords[:, 0, a] for a in range(d)]
    J = np.prod(ext, axis=0) / 2 ** d
    wJ = wq[None, :] * J[:, None]
    # scale: the variable's own magnitude, for momentum components the total momentum
    mom = float(np.sum(wJ * np.sqrt(np.sum(wl.u0[1:-1] ** 2, axis=0))))
    for v in range(wl.nvar):
        m0 = float(np.sum(wJ * wl.u0[v]))
        m1 = float(np.sum(wJ * u[v]))
        scale = float(np.sum(wJ * np.abs(wl.u0[v]))) + (mom if 0 < v < wl.nvar - 1 else 0.0)
        assert abs(m1 - m0) < 1e-8 * scale, (name, v)
    A = float(np.sum(wJ * np.abs(physics.euler_entropy(wl.u0, 1.4))))
    for r in recs:
        assert r["flags"] & (pk.FLAG_NONPHYSICAL | pk.FLAG_NONFINITE) == 0
        if name == "tgv":
            assert abs(r["H_next"] - r["H_n"]) <= 1e-12 * A
        else:
            assert r["dH"] < 0 and r["H_next"] <= r["H_n"] + 1e-13 * A


def test_fullsize_batched_sampled_instances():
    """The bench's batched workload (256 instances) in the bench's launch
    configuration; the four smallest instances against oracle runs and the
    linear invariants of all instances."""
    insts = workloads.batched_2d(n_inst=256, seed=1)
    s = pk.Solver(insts, pk.options(precision=pk.MIXED, use_graph=True))
    pk.perrk_autotune(s.h)
    s.set_state(np.concatenate([w.u0 for w in insts], axis=1))
    recs = s.step(3)
    u = s.state()
    s.close()
    offs = np.cumsum([0] + [w.n_elem for w in insts])
    smallest = np.argsort([w.n_elem for w in insts])[:4]
    for k in smallest:
        wl = insts[k]
        ref = operrk.Solver(wl)
        for _ in range(3):
            ref.step(wl.dt)
        ug = u[:, offs[k]:offs[k + 1]]
        assert np.abs(ug - ref.U).max() / np.abs(ref.U).max() < 1e-5
    for k, wl in enumerate(insts):
        hx = wl.coords[:, 3, 0] - wl.coords[:, 0, 0]
        hy = wl.coords[:, 12, 1] - wl.coords[:, 0, 1]
        w1 = np.array([1.0, 5.0, 5.0, 1.0]) / 6.0
        wJ = np.outer(w1, w1).ravel()[None, :] * (hx * hy / 4)[:, None]
        m0 = float(np.sum(wJ * wl.u0[0]))
        m1 = float(np.sum(wJ * u[0, offs[k]:offs[k + 1]]))
        assert abs(m1 - m0) < 1e-8 * abs(m0)
        assert all(row[k]["flags"] & (pk.FLAG_NONPHYSICAL | pk.FLAG_NONFINITE) == 0 for row in recs)
