"""The allocation-free entropy entry point (perrk_entropy_static).

Callers that cannot allocate device memory when they need the entropy (for
instance because all device memory belongs to their own pool allocator, or
because they run in a loop where cudaMalloc is not allowed) pass their state,
their quadrature weights and an output buffer; the library uses a file-scope
device scratch array instead of allocating.  This test checks that entry
point, through the C ABI, against the context-based perrk_entropy on the same
state, on two calls in a row (the scratch array is reused between calls).
"""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads

pytestmark = pytest.mark.gpu

LGL_W = np.array([1.0, 5.0, 5.0, 1.0]) / 6.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _box_weights(coords):
    """omega_i omega_j J on axis-aligned box elements, J = hx hy / 4."""
    hx = coords[:, 3, 0] - coords[:, 0, 0]
    hy = coords[:, 12, 1] - coords[:, 0, 1]
    w2 = np.outer(LGL_W, LGL_W).ravel()          # index j*4 + i
    return (w2[None, :] * (hx * hy / 4.0)[:, None]).ravel()


def test_entropy_static_matches_context_entropy_twice():
    import torch
    wl = workloads.small_box_2d(n=8, seed=51, R=2, E=[6, 3], order=3)
    s = pk.Solver(wl, pk.options(precision=pk.FP64))
    H_ref = float(pk.perrk_entropy(s.h)[0])
    s.close()
    u = torch.tensor(wl.u0.reshape(wl.nvar, -1), device="cuda", dtype=torch.float64).contiguous()
    wj = torch.tensor(_box_weights(wl.coords), device="cuda", dtype=torch.float64)
    n = wj.numel()
    for _ in range(2):
        out = torch.full((2,), float("nan"), device="cuda", dtype=torch.float64)
        pk.perrk_entropy_static(pk.EULER_2D, wl.gamma_gas, u.data_ptr(), wj.data_ptr(), n, out.data_ptr())
        torch.cuda.synchronize()
        H, A = out.cpu().numpy()
        assert abs(H - H_ref) <= 1e-12 * abs(H_ref)
        assert A >= abs(H) > 0.0


def test_entropy_static_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    for bad in (0, 16777216 + 1):
        with pytest.raises(pk.PerrkError) as ei:
            pk.perrk_entropy_static(pk.BURGERS_1D, 1.4, x.data_ptr(), x.data_ptr(), bad, x.data_ptr())
        assert ei.value.status == pk.PERRK_INVALID_ARG
        assert "n_nodes" in pk.last_error()
