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
    hd, hist = pk.checkpoint_history(ckpt)
    assert hd.magic == 0x4b435250 and hd.precision == precision and hd.n_inst == 2
    assert all(h.steps == 3 for h in hist)

    b = pk.Solver(_problems(), opts())
    b.set_mlp(w)
    b.resume(ckpt)
    rec_b = b.step(4)
    u_b = b.state()
    _, hist = pk.checkpoint_history(b.checkpoint())
    b.close()

    assert np.array_equal(u_b, u_ref)
    assert _fields(rec_a) + _fields(rec_b) == _fields(rec_ref)
    assert all(h.steps == 7 for h in hist)


def test_checkpoint_rejects_mismatch():
    """A checkpoint loads only into a context of the same precision and
    shapes, and only with consistent step counts; the context is unchanged
    after a refused load."""
    s = pk.Solver(_problems(), pk.options())
    data = bytearray(s.checkpoint())
    u0 = s.state()
    other = pk.Solver(_problems(), pk.options(precision=pk.MIXED))
    with pytest.raises(pk.PerrkError) as ei:
        other.resume(bytes(data))
    assert ei.value.status == pk.PERRK_INVALID_ARG
    other.close()
    bad = bytearray(data)
    off = pk.C.sizeof(pk.perrk_checkpoint_header) + pk.C.sizeof(pk.perrk_resume_info) + \
        pk.perrk_resume_info.steps.offset
    bad[off:off + 8] = (5).to_bytes(8, "little")          # instance 1 at another step count
    with pytest.raises(pk.PerrkError):
        s.resume(bytes(bad))
    with pytest.raises(pk.PerrkError):
        s.resume(bytes(data[:-8]))                         # truncated
    assert np.array_equal(s.state(), u0)
    s.close()


def test_async_state_copies_match_synchronous():
    """on_device = 2: asynchronous host copies on a side stream, two contexts
    in flight at once, give the same result as the synchronous path."""
    import torch
    wl = _problems()
    u0 = np.concatenate([w.u0 for w in wl], axis=1)
    ref = pk.Solver(wl, pk.options(precision=pk.MIXED))
    ref.set_state(u0)
    ref.step(3, info=False)
    u_ref = ref.state()
    ref.close()
    host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    ctx = [pk.Solver(wl, pk.options(precision=pk.MIXED)) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    for X in range(2):
        s = streams[X].cuda_stream
        pk.perrk_set_state(ctx[X].h, host_in.data_ptr(), on_device=pk.STATE_HOST_ASYNC, stream=s)
        pk.perrk_step(ctx[X].h, 3, info=False, stream=s)
        pk.perrk_get_state(ctx[X].h, outs[X].data_ptr(), on_device=pk.STATE_HOST_ASYNC, stream=s)
    torch.cuda.synchronize()
    for X in range(2):
        assert np.array_equal(outs[X].numpy(), u_ref)
    with pytest.raises(ValueError):             # an ndarray may not outlive an asynchronous call
        pk.perrk_set_state(ctx[0].h, u0, on_device=pk.STATE_HOST_ASYNC)
    for X in range(2):
        ctx[X].close()
