"""Batched form: independent instances of different sizes, partition counts,
time steps and initial data advanced by one context (one launch per stage over
all instances' active elements, per-instance Newton solves)."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import perrk as operrk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _instances():
    return workloads.batched_2d(n_inst=5, seed=7, n_min=6, n_max=12)


def _batched_run(insts, steps, precision, use_graph=False, tune=False):
    s = pk.Solver(insts, pk.options(precision=precision, use_graph=use_graph))
    if tune:
        pk.perrk_autotune(s.h)
        s.set_state(np.concatenate([w.u0 for w in insts], axis=1))
    recs = s.step(steps)
    u = s.state()
    s.close()
    return u, recs


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_batched_matches_oracle_per_instance(precision):
    insts = _instances()
    assert len({w.info["R"] for w in insts}) > 1 and len({w.info["n"] for w in insts}) > 1
    steps = 6
    u, recs = _batched_run(insts, steps, precision)
    off = 0
    for k, wl in enumerate(insts):
        ref = operrk.Solver(wl)
        rrec = []
        for _ in range(steps):
            u0 = ref.U.copy()
            r = ref.step(wl.dt)
            r.du_inf = float(np.abs(ref.U - u0).max())
            rrec.append(r)
        ug = u[:, off:off + wl.n_elem]
        off += wl.n_elem
        grec = [row[k] for row in recs]
        err = float(np.abs(ug - ref.U).max() / np.abs(ref.U).max())
        if precision == pk.FP64:
            extra = sum(abs(a["gamma"] - b.gamma) * b.du_inf / b.gamma for a, b in zip(grec, rrec))
            assert err < 1e-12 + 1.5 * extra / np.abs(ref.U).max(), (k, err)
            assert all(abs(a["gamma"] - b.gamma) < 1e-7 for a, b in zip(grec, rrec))
        else:
            assert err < 1e-5, (k, err)
        assert abs(grec[-1]["t"] - ref.t) < (1e-10 if precision == pk.FP64 else 1e-6)


def test_batched_graph_and_autotune_bitwise():
    insts = _instances()
    u1, r1 = _batched_run(insts, 4, pk.MIXED)
    u2, r2 = _batched_run(insts, 4, pk.MIXED, use_graph=True, tune=True)
    assert np.array_equal(u1, u2)
    assert [[x["gamma"] for x in row] for row in r1] == [[x["gamma"] for x in row] for row in r2]


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_many_instances_one_block_each(precision):
    """With at least as many instances as SMs, each instance's Delta H is
    summed by one block of its own; fewer instances use the work chunks.
    The same instances in one context of 160 and in two of 80: the first
    step's Delta H (identical element sums, only their order differs) agrees
    to round-off; gamma and the state agree to the root's conditioning (the
    two contexts also chunk their Newton passes differently)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = max(160, sms + 8)
    insts = workloads.batched_2d(n_inst=n, seed=11, n_min=8, n_max=12)
    big, rb = _batched_run(insts, 3, precision)
    halves = [insts[: n // 2], insts[n // 2:]]
    parts = [_batched_run(h, 3, precision) for h in halves]
    small = np.concatenate([p[0] for p in parts], axis=1)
    rs = [row_a + row_b for row_a, row_b in zip(parts[0][1], parts[1][1])]
    dh_b = np.array([x["dH"] for x in rb[0]])
    dh_s = np.array([x["dH"] for x in rs[0]])
    # (mixed form: the element integrands carry FP32 noise of both signs and
    # Delta H is a small remainder of them, so the double-float sums' order
    # shows at ~1e-9 of it)
    tol_dh = 1e-12 if precision == pk.FP64 else 1e-8
    assert np.abs(dh_b - dh_s).max() <= tol_dh * np.abs(dh_s).max(), np.abs(dh_b - dh_s).max()
    gb = np.array([[x["gamma"] for x in row] for row in rb])
    gs = np.array([[x["gamma"] for x in row] for row in rs])
    # (mixed form: its root moves by ~3e-5 from step to step on the FP32
    # rounding in Delta H, so a different summation order moves it as much)
    assert np.abs(gb - gs).max() <= (1e-6 if precision == pk.FP64 else 1e-3), np.abs(gb - gs).max()
    scale = np.abs(small).max()
    assert np.abs(big - small).max() <= (1e-9 if precision == pk.FP64 else 1e-6) * scale
    assert all(x["flags"] == 0 for row in rb for x in row)
