"""Matched error: both forms against the exact solutions of the Burgers and
vortex configurations.  The mixed form's FP32 rounding must stay far below
the discretisation error at the same time step and mesh, so that its speed
is not bought with accuracy."""
import math

import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    __graft_entry__.build()
    torch.zeros(1, device="cuda")


def _run(wl, nsteps, precision):
    s = pk.Solver(wl, pk.options(precision=precision, max_it=10, tol_r=1e-14 if precision == pk.FP64 else 1e-12,
                                 tol_g=1e-14))
    recs = s.step(nsteps)
    u = s.state()
    s.close()
    return u, recs[-1][0]["t"]


def _burgers_exact(x, t):
    """u(x, t) = u0(x - u t), u0 = 1 + sin(2 pi x) / 2, before the shock time
    1 / pi: Newton on the characteristic equation node by node."""
    u = 1.0 + 0.5 * np.sin(2 * math.pi * x)
    for _ in range(60):
        g = u - 1.0 - 0.5 * np.sin(2 * math.pi * (x - u * t))
        dg = 1.0 + math.pi * t * np.cos(2 * math.pi * (x - u * t))
        u = u - g / dg
    return u


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_burgers_error_against_exact(precision):
    wl = workloads.burgers_1d()
    n = int(round(wl.info["t_end"] / wl.dt))
    u, t = _run(wl, n, precision)
    ex = _burgers_exact(wl.coords[:, :, 0], t)
    err = np.abs(u[0] - ex).max()
    u64, t64 = _run(wl, n, pk.FP64)
    err64 = np.abs(u64[0] - _burgers_exact(wl.coords[:, :, 0], t64)).max()
    assert err64 < 1e-3                                  # resolved smooth solution
    assert abs(err - err64) < 0.05 * err64, (err, err64)


def test_vortex_error_against_exact():
    """The 64 x 64 curved vortex, 40 relaxed steps: both forms' L_inf errors
    against the translating vortex at each run's own final time agree to 5%
    of their size (the FP32 rounding is a small part of the error)."""
    wl = workloads.vortex_2d()
    errs = {}
    for prec in (pk.FP64, pk.MIXED):
        u, t = _run(wl, 40, prec)
        inf = wl.info
        ex = workloads.isentropic_vortex(wl.coords[:, :, 0], wl.coords[:, :, 1], t, inf["center"], inf["strength"],
                                         L=inf["L"])
        errs[prec] = float(np.abs(u - ex).max() / np.abs(ex).max())
    assert errs[pk.FP64] < 1e-2
    assert abs(errs[pk.MIXED] - errs[pk.FP64]) < 0.05 * errs[pk.FP64], errs


def test_vortex_convergence_order():
    """Observed order of the relaxed multirate scheme on the curved vortex
    configuration (p = 3, N = 3, three partitions), refining space and time
    together against the exact translating vortex (the paper's convergence
    study design, Sec. 4.3.1)."""
    T = 0.5
    errs = []
    for n in (24, 48, 96):
        wl = workloads.vortex_2d(n=n)
        nsteps = int(math.ceil(T / wl.dt))
        wl.dt = T / nsteps
        u, t = _run(wl, nsteps, pk.FP64)
        inf = wl.info
        ex = workloads.isentropic_vortex(wl.coords[:, :, 0], wl.coords[:, :, 1], t, inf["center"], inf["strength"],
                                         L=inf["L"])
        errs.append(float(np.abs(u - ex).max() / np.abs(ex).max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > 2.5 and errs[-1] < errs[0], (errs, rates)
