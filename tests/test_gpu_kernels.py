"""GPU checks of building blocks: the double-float logarithm of the mixed
form against CUDA's float64 log (error bound 2^-46), and the relaxation
kernels' determinism."""
import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()


def test_df_log_against_cuda_log():
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([np.exp(rng.uniform(-30, 30, 200000)), 1 + rng.uniform(-1e-4, 1e-4, 50000),
                        rng.uniform(0.2, 5.0, 200000), [1.0, 2.0, 0.5, 1.0 + 2.0 ** -20]])
    xd = torch.tensor(x, device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    pk.perrk_df_log(xd.data_ptr(), yd.data_ptr(), xd.numel())
    ref = torch.log(xd)
    err = (yd - ref).abs()
    small = ref.abs() < 1
    assert float(err[small].max()) < 2.0 ** -46                 # absolute, |log x| < 1
    assert float((err[~small] / ref[~small].abs()).max()) < 2.0 ** -46
    assert float(yd[-4]) == 0.0


def test_repeatable_bitwise():
    wl = workloads.small_box_2d(n=8, seed=41, R=2, E=[6, 3], order=3)
    outs = []
    for _ in range(2):
        s = pk.Solver(wl, pk.options(precision=pk.MIXED))
        recs = s.step(5)
        outs.append((s.state(), [r[0]["gamma"] for r in recs]))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_autotune_keeps_results_bitwise(precision):
    wl = workloads.small_box_2d(n=8, seed=43, R=2, E=[6, 3], order=3)
    s1 = pk.Solver(wl, pk.options(precision=precision))
    r1 = s1.step(4)
    u1 = s1.state()
    s1.close()
    s2 = pk.Solver(wl, pk.options(precision=precision, use_graph=True))
    pk.perrk_autotune(s2.h)
    s2.set_state(wl.u0)
    tuning = pk.perrk_tuning(s2.h)
    r2 = s2.step(4)
    u2 = s2.state()
    s2.close()
    assert tuning["elems_per_cta"] in (4, 8, 16) and tuning["relax_threads"] in (128, 256)
    assert tuning["stage_variant"] in (0, 1, 2, 3, 4)
    # grid candidates: one CTA per element group, 2, 4 or 8 CTAs per SM, and
    # for the box kernels (mixed form) the one-wave grids of 20, 10, 5 per SM
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_sm = (2, 4, 8) + ((5, 10, 20) if precision == pk.MIXED else ())
    assert tuning["persistent_grid"] in [0] + [k * sms for k in per_sm]
    assert np.array_equal(u1, u2)
    assert [a[0]["gamma"] for a in r1] == [a[0]["gamma"] for a in r2]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_mixed_stage_kernel_variants_bitwise(dim, mu):
    """The mixed form's stage kernels (generic, float4 box kernel, box kernel
    with cp.async staging and, in 2D, the box kernel fed by a producer warp
    through bulk copies) under every elements-per-CTA and grid choice give
    bit-identical steps (same arithmetic in the same order), with and without
    the viscous terms."""
    if dim == 2:
        wl = workloads.small_box_2d(n=12, seed=47, R=2, E=[6, 3], order=3, ic="khi", mu=mu)
        epbs = (4, 8, 16)
    else:
        wl = workloads.tgv_3d(n=8, n_fine=4, mu=mu)
        epbs = (1, 2, 4)
    ref = None
    configs = [(v, e, g) for v in (0, 1, 2) for e in epbs for g in (0, 152)]
    if dim == 2:
        # the staged kernel: its ring of buffers wraps around several times
        # when a small persistent grid covers all element groups
        configs += [(v, e, g) for v in (3, 4) for e in (4, 8) for g in (0, 1, 3)]
    for variant, epb, grid in configs:
        s = pk.Solver(wl, pk.options(precision=pk.MIXED, use_graph=True))
        try:
            pk.perrk_set_tuning(s.h, epb, grid, 128, variant)
            s.set_state(wl.u0)
            recs = s.step(3)
        except pk.PerrkError as err:
            # a mapping whose shared memory does not fit is refused at launch
            assert "invalid configuration" in str(err) or "configuration" in pk.last_error()
            s.close()
            continue
        out = (s.state(), [r[0]["gamma"] for r in recs])
        s.close()
        if ref is None:
            ref = out
        assert np.array_equal(out[0], ref[0]), (variant, epb, grid)
        assert out[1] == ref[1], (variant, epb, grid)
    assert ref is not None


@pytest.mark.parametrize("precision", [pk.FP64, pk.MIXED])
def test_fused_direction_bitwise(precision):
    """d formed once at the last stage from K_1, K_{S-1}, K_S equals d
    accumulated stage by stage, bit for bit (same sums in the same order), for
    p = 2, 3 and 4 families."""
    for order, E in ((2, [6, 3]), (3, [6, 3]), (4, [8, 5])):
        wl = workloads.small_box_2d(n=8, seed=53, R=2, E=E, order=order, ic="khi")
        outs = []
        for fuse in (True, False):
            s = pk.Solver(wl, pk.options(precision=precision, fuse_direction=fuse))
            recs = s.step(3)
            outs.append((s.state(), [r[0]["gamma"] for r in recs], [r[0]["dH"] for r in recs]))
            s.close()
        assert np.array_equal(outs[0][0], outs[1][0]), order
        assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2], order


def _run_variant(wls, variant, epb, grid, steps=3, fuse=True):
    s = pk.Solver(wls, pk.options(precision=pk.MIXED, use_graph=True, fuse_direction=fuse))
    pk.perrk_set_tuning(s.h, epb, grid, 128, variant)
    s.set_state(np.concatenate([w.u0 for w in wls], axis=1))
    recs = s.step(steps)
    out = (s.state(), [[r["gamma"] for r in row] for row in recs], [[r["dH"] for r in row] for row in recs])
    s.close()
    return out


@pytest.mark.parametrize("fuse", [True, False])
def test_staged_kernel_batched_bitwise(fuse):
    """Batched instances of uneven sizes (ragged active prefixes in every
    stage) through the staged kernel against the box kernel, bit for bit, with
    the direction fused or accumulated, for two family sizes."""
    for order, S in ((3, 12), (3, 10)):
        wls = workloads.batched_2d(n_inst=6, seed=5 + order, n_min=6, n_max=20, S=S, order=order)
        ref = _run_variant(wls, 1, 8, 0, fuse=fuse)
        for variant, epb, grid in ((3, 8, 0), (3, 8, 5), (3, 4, 0), (4, 4, 2), (4, 8, 0), (4, 8, 3)):
            out = _run_variant(wls, variant, epb, grid, fuse=fuse)
            assert np.array_equal(out[0], ref[0]), (order, variant, epb, grid)
            assert out[1] == ref[1] and out[2] == ref[2], (order, variant, epb, grid)


def test_staged_kernel_bounded_wait_reports_timeout_and_recovers():
    """The staged kernel's waits are bounded: with its producer told to fill
    nothing, the consumers give up after about a second, the step reports
    PERRK_TIMEOUT, and the same context then steps normally again."""
    import time
    wl = workloads.small_box_2d(n=12, seed=47, R=2, E=[6, 3], order=3, ic="khi")
    ref = _run_variant([wl], 1, 8, 0)
    s = pk.Solver(wl, pk.options(precision=pk.MIXED))
    pk.perrk_set_tuning(s.h, 8, 0, 128, 3)
    pk.perrk_test_stall_producer(s.h, True)
    t0 = time.perf_counter()
    with pytest.raises(pk.PerrkError) as ei:
        s.step(1)
    assert ei.value.status == pk.PERRK_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    pk.perrk_test_stall_producer(s.h, False)
    s.set_state(wl.u0)
    recs = s.step(3)
    assert np.array_equal(s.state(), ref[0])
    assert [r[0]["gamma"] for r in recs] == [g[0] for g in ref[1]]
    s.close()
