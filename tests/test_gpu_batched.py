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
