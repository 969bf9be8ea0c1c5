"""Semi-discrete pins of the oracle's DGSEM: conservation, entropy conservation /
stability, free-stream preservation, metric identities, spectral accuracy."""
import numpy as np
import pytest

import workloads
from oracle import dgsem, physics


def _perturbed(u, rng, amp=0.05):
    return u * (1.0 + amp * rng.standard_normal(u.shape))


CASES = [
    ("burgers1d", lambda: workloads.burgers_1d()),
    ("euler2d_box", lambda: workloads.small_box_2d(n=6)),
    ("euler2d_curved", lambda: workloads.vortex_2d(n=12)),
    ("euler3d", lambda: workloads.tgv_3d(n=4, n_fine=2)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_conservation_and_entropy(name, make):
    wl = make()
    rng = np.random.default_rng(5)
    g = dgsem.Geometry(wl.coords, wl.faces)
    u = _perturbed(wl.u0, rng)
    for surf in ("ec", "es_rusanov" if wl.equation != "burgers1d" else "es"):
        ph = physics.Physics(wl.equation, surf)
        K = dgsem.rhs(g, ph, u)
        scale = g.integrate(np.sum(np.abs(K), axis=0)) + 1.0
        for v in range(K.shape[0]):
            assert abs(g.integrate(K[v])) < 1e-13 * scale, (name, surf, v)
        rate = g.integrate(np.sum(ph.entropy_vars(u) * K, axis=0))
        if surf == "ec":
            assert abs(rate) < 1e-13 * scale
        else:
            assert rate < -1e-6 * scale


@pytest.mark.parametrize("name,make", CASES[1:])
def test_free_stream(name, make):
    wl = make()
    g = dgsem.Geometry(wl.coords, wl.faces)
    ph = physics.Physics(wl.equation, "es_rusanov")
    u = np.ones_like(wl.u0)
    u[1:-1] = np.arange(1, wl.dim + 1)[:, None, None] * 0.3
    u[-1] = 4.0
    K = dgsem.rhs(g, ph, u)
    assert np.abs(K).max() < 1e-11


def test_metric_identities_curved():
    wl = workloads.vortex_2d(n=12)
    g = dgsem.Geometry(wl.coords, wl.faces)
    for comp in range(2):
        div = g.dxi(g.Ja[0][comp], 0) + g.dxi(g.Ja[1][comp], 1)
        assert np.abs(div).max() < 1e-12
    assert np.all(g.J > 0)
    # total area = (2L)^2
    assert abs(np.sum(g.wJ) - 400.0) < 1e-9


def test_spectral_accuracy_burgers_rhs():
    """For smooth data the DG RHS approximates -(u^2/2)_x with pointwise error ~ h^N."""
    errs = []
    for n in (16, 32):
        edges = np.linspace(0, 1, n + 1)
        coords = workloads.tensor_coords([edges])
        g = dgsem.Geometry(coords, workloads.structured_faces([n]))
        x = coords[:, :, 0]
        u = (1 + 0.5 * np.sin(2 * np.pi * x))[None]
        K = dgsem.rhs(g, physics.Physics("burgers1d", "ec"), u)
        exact = -u[0] * 0.5 * 2 * np.pi * np.cos(2 * np.pi * x)
        errs.append(np.abs(K[0] - exact).max())
    assert errs[0] / errs[1] > 0.8 * 2 ** 3
