"""Checkpoint/resume: a run stopped after n steps, saved (state and relaxation
history), restored into a fresh context and continued must reproduce the
uninterrupted run bit for bit: state, gamma, Delta H and Newton counts."""
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


def _problems():
    return [workloads.small_box_2d(n=6, seed=31, R=3, E=[7, 5, 3], order=3, random_parts=True),
            workloads.small_box_2d(n=6, seed=32, R=2, E=[4, 3], order=3)]


def _fields(recs):
    keys = ("gamma", "dH", "H_next", "t", "gamma_guess", "iters", "flags")
    return [tuple(r[k] for k in keys) for step in recs for r in step]


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
@pytest.mark.parametrize("guess", [pk.GUESS_PREV, pk.GUESS_MLP])
@pytest.mark.parametrize("target", [pk.TARGET_DELTA_H, pk.TARGET_INITIAL])
def test_resumed_run_is_bitwise_identical(precision, guess, target):
    opts = lambda: pk.options(precision=precision, guess=guess, target=target, use_graph=True, max_it=8,
                              tol_r=1e-13, tol_g=1e-14)
    w = pk.mlp_init(seed=5)
    ref = pk.Solver(_problems(), opts())
    ref.set_mlp(w)
    rec_ref = ref.step(7)
    u_ref = ref.state()
    ref.close()

    a = pk.Solver(_problems(), opts())
    a.set_mlp(w)
    rec_a = a.step(3)
    ckpt = a.checkpoint()
    a.close()
    assert all(h.steps == 3 for h in ckpt[1])

    b = pk.Solver(_problems(), opts())
    b.set_mlp(w)
    b.resume(ckpt)
    rec_b = b.step(4)
    u_b = b.state()
    hist = pk.perrk_get_resume(b.h)
    b.close()

    assert np.array_equal(u_b, u_ref)
    assert _fields(rec_a) + _fields(rec_b) == _fields(rec_ref)
    assert all(h.steps == 7 for h in hist)


def test_resume_rejects_mismatched_history():
    s = pk.Solver(_problems(), pk.options())
    hist = pk.perrk_get_resume(s.h)
    hist[1].steps = hist[0].steps + 1
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_set_resume(s.h, hist)
    assert ei.value.status == pk.PERRK_INVALID_ARG
    s.close()
