"""The allocation-free entropy entry point (perrk_entropy_static).

Some callers cannot allocate device memory at the point where they need the
entropy: code that hands all device memory to its own pool allocator up
front, or a loop in which cudaMalloc (which may synchronise the device and can
fail under memory pressure) is not allowed.  They pass their state, their
quadrature weights and an output buffer; the library's cross-block scratch is
a file-scope device array instead of an allocation.

These tests call that entry point through the C ABI and check it against the
oracle's entropy functions summed exactly on the host (math.fsum), and
against the context-based perrk_entropy, on two calls in a row each (the
scratch array and its ticket counter are reused between calls).  The sizes
launch one block, several blocks with a ragged last one, and all 4096 blocks
at the documented maximum of 16,777,216 nodes, so that the ticket, the
visibility of the block partials, the last block's reduction and the counter
reset between calls all run.
"""
import math

import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import dgsem as odg
from oracle import physics as oph

pytestmark = pytest.mark.gpu

NODES_PER_BLOCK = 4096
MAX_NODES = 16_777_216


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _exact_sums(s, wj):
    """(sum wJ s, sum wJ |s|), each product rounded once, then summed exactly."""
    t = wj * s
    return math.fsum(t.tolist()), math.fsum(np.abs(t).tolist())


def _call(equation, gamma, u, wj, stream=0):
    import torch
    out = torch.full((2,), float("nan"), device="cuda", dtype=torch.float64)
    pk.perrk_entropy_static(equation, gamma, u.data_ptr(), wj.data_ptr(), wj.numel(), out.data_ptr(), stream)
    return out


def _check(out, H_ref, A_ref, tol=1e-12):
    H, A = out.cpu().numpy()
    assert abs(H - H_ref) <= tol * abs(A_ref), (H, H_ref)
    assert abs(A - A_ref) <= tol * abs(A_ref), (A, A_ref)


def _burgers_case(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    u = rng.uniform(-2.0, 2.0, n)
    wj = rng.uniform(0.1, 1.0, n)
    s = oph.burgers_entropy(u[None, :])
    H_ref, A_ref = _exact_sums(s, wj)
    return (torch.tensor(u, device="cuda").reshape(1, n).contiguous(), torch.tensor(wj, device="cuda"),
            H_ref, A_ref)


@pytest.mark.parametrize("n", [1000, 3 * NODES_PER_BLOCK + 17, MAX_NODES])
def test_burgers_against_oracle_twice(n):
    """One block; four blocks with a ragged fourth; every block at the cap."""
    import torch
    u, wj, H_ref, A_ref = _burgers_case(n, seed=n % 997)
    stream = torch.cuda.current_stream().cuda_stream
    first = _call(pk.BURGERS_1D, 1.4, u, wj, stream)
    second = _call(pk.BURGERS_1D, 1.4, u, wj, stream)   # same stream, no sync in between
    torch.cuda.synchronize()
    _check(first, H_ref, A_ref)
    _check(second, H_ref, A_ref)
    assert torch.equal(first, second)


def test_euler2d_multiblock_against_oracle_and_context():
    """A 40 x 40 vortex mesh: 25,600 nodes, six full blocks and a ragged
    seventh.  The reference sums use the oracle's metric terms and entropy."""
    import torch
    wl = workloads.small_box_2d(n=40, seed=51, R=2, E=[6, 3], order=3)
    geo = odg.Geometry(wl.coords, wl.faces)
    s = oph.euler_entropy(wl.u0, wl.gamma_gas)                  # [n_elem, NP]
    H_ref, A_ref = _exact_sums(s.ravel(), geo.wJ.ravel())
    n_nodes = geo.wJ.size
    assert n_nodes > 6 * NODES_PER_BLOCK and n_nodes % NODES_PER_BLOCK != 0
    sol = pk.Solver(wl, pk.options(precision=pk.FP64))
    H_ctx = float(pk.perrk_entropy(sol.h)[0])
    sol.close()
    u = torch.tensor(wl.u0.reshape(wl.nvar, -1), device="cuda", dtype=torch.float64).contiguous()
    wj = torch.tensor(geo.wJ.ravel(), device="cuda", dtype=torch.float64)
    for _ in range(2):
        out = _call(pk.EULER_2D, wl.gamma_gas, u, wj)
        torch.cuda.synchronize()
        _check(out, H_ref, A_ref)
        assert abs(float(out[0]) - H_ctx) <= 1e-12 * A_ref


def test_counter_reset_between_sizes():
    """A many-block call, a one-block call, then the many-block call again: a
    ticket counter left non-zero by one call would make the next call's last
    block finish early (or never) and give a wrong sum."""
    import torch
    big = _burgers_case(9 * NODES_PER_BLOCK + 5, seed=7)
    small = _burgers_case(300, seed=8)
    outs = [_call(pk.BURGERS_1D, 1.4, c[0], c[1]) for c in (big, small, big)]
    torch.cuda.synchronize()
    for out, c in zip(outs, (big, small, big)):
        _check(out, c[2], c[3])


def test_nonphysical_node_gives_nan():
    """p = 0 exactly at one node (rho = 1, v = 0, E = 0): both sums are NaN."""
    import torch
    n = 2 * NODES_PER_BLOCK + 3
    u = np.zeros((4, n))
    u[0] = 1.0
    u[3] = 2.5
    u[3, n // 2] = 0.0
    out = _call(pk.EULER_2D, 1.4, torch.tensor(u, device="cuda"), torch.ones(n, device="cuda",
                                                                              dtype=torch.float64))
    torch.cuda.synchronize()
    assert np.isnan(out.cpu().numpy()).all()


def test_entropy_static_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    for bad in (0, MAX_NODES + 1):
        with pytest.raises(pk.PerrkError) as ei:
            pk.perrk_entropy_static(pk.BURGERS_1D, 1.4, x.data_ptr(), x.data_ptr(), bad, x.data_ptr())
        assert ei.value.status == pk.PERRK_INVALID_ARG
        assert "n_nodes" in pk.last_error()
