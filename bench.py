"""Throughput of the P-ERRK multirate stage loop on GB300 (DOF-stage updates/s).

A step is one full P-ERRK step of every instance of the workload: all stages
over their active elements, the Delta H reduction, the Newton passes and the
relaxed update.  The unit counts sum_r E^(r) M^(r) scalar right-hand-side
evaluations per step (the paper's eq. RHSEvals), M^(r) = nodes x variables of
partition r, summed over instances.

Chosen form: all instances in one batched context (one launch per stage over
every instance's active elements, per-instance Newton solves), FP32 fluxes
and stage registers, the state, direction, entropy passes and update as
float pairs (~48-bit significand), float64 Newton scalars and Delta H, the
learned Newton guess (trained during set-up on gamma traces of the plain
method), autotuned CTA mapping, one CUDA graph per step.  It is compared with
the plain float64 form looped per instance and with the plain float64 form
batched.

  python bench.py [--gpus N --steps K --warmup W] [--workload batched2d|vortex2d|khi2d|tgv3d|burgers1d]
                  [--impl native|reference]

Multi-GPU runs are independent replicas (one per rank, seeded by rank,
launched with torch.distributed.run): value = DOF-stage updates of all ranks
/ max rank time.  ``--impl reference`` times the CPU oracle (plain float64
numpy) on the host, one bounded sample per step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-stage updates/s per GB300, chosen vs plain FP64 form, at matched error"
# what the chosen form computes in: FP32 flux differencing, surface fluxes and
# stage registers K_i; the state U, the direction d and the entropy passes as
# float pairs (hi + lo, ~48-bit significand) on the FP32 pipe; the Newton
# scalars, Delta H and the step records in float64
DTYPE_CHOSEN = "f32 fluxes/K + f32x2 (~48-bit) state, d, entropy + f64 scalars"
UNIT = "DOF-stage updates/s"


def make_workload(name, rank=0, instances=None, size=None):
    import workloads
    if size and name in ("khi2d", "tgv3d"):
        # a smaller mesh of the same configuration (profiling captures)
        if name == "khi2d":
            return [workloads.khi_2d(n=size, seed=1 + rank)], (f"Kelvin-Helmholtz, {size}x{size} quads graded in y "
                                                                "(4 levels), N=3, 4 partitions E={16,10,7,5}, p=4, ES")
        return [workloads.tgv_3d(n=size, n_fine=size // 4)], (f"Taylor-Green vortex Ma 0.1, {size}^3 boxes, central "
                                                               f"{size // 4} per axis at h/2, N=3, 2 partitions "
                                                               "E={8,4}, p=3, EC")
    if name == "batched2d":
        insts = workloads.batched_2d(n_inst=256, seed=1 + rank)[:(instances or 256)]
        return insts, ("256 independent 2D Euler instances, n x n quads with n ~ U{16..128} (1.63M elements, "
                       "1.04e8 DOF), 2-4 partitions by a graded refinement band, vortex or KHI initial data, "
                       "N=3, p=3 P-ERRK (S=12), Ranocha EC volume + Rusanov ES surface")
    if name == "vortex2d":
        return [workloads.vortex_2d(n=64, seed=1 + rank)], ("isentropic vortex, 64x64 curved quads on [-10,10]^2, "
                                                             "N=3, 3 partitions E={12,6,3}, p=3, Ranocha EC volume "
                                                             "+ Rusanov ES surface")
    if name == "khi2d":
        return [workloads.khi_2d(n=256, seed=1 + rank)], ("Kelvin-Helmholtz, 256x256 quads graded in y (4 levels), "
                                                           "N=3, 4 partitions E={16,10,7,5}, p=4, ES")
    if name == "tgv3d":
        return [workloads.tgv_3d(n=64)], ("Taylor-Green vortex Ma 0.1, 64^3 boxes, central 16 per axis at h/2, "
                                          "N=3, 2 partitions E={8,4}, p=3, EC")
    if name == "tgv3d_visc":
        wl = workloads.tgv_3d(n=64, mu=1.0 / 1600.0)
        wl.prandtl = 0.71
        return [wl], ("viscous Taylor-Green vortex, Re 1600 (mu = 1/1600), Pr 0.71, Ma 0.1, 64^3 boxes, central 16 "
                      "per axis at h/2, N=3, 2 partitions E={8,4}, p=3, EC volume and surface fluxes, "
                      "Navier-Stokes-Fourier viscous terms by BR1 on entropy-variable gradients")
    if name == "burgers1d":
        return [workloads.burgers_1d()], "Burgers 1D, 64 elements (16 at h/4), N=3, p=2 E={8,4}, EC"
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 50 ms."""

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        num = lambda x: x.replace(".", "").isdigit()
        sm = [float(s[1]) for s in self.samples if num(s[1])]
        mx = [float(s[2]) for s in self.samples if num(s[2])]
        pw = [float(s[3]) for s in self.samples if num(s[3])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(self.samples)}


_BACKEND = None


def dist_setup(backend=None):
    """Ranks from the torch.distributed.run environment; NCCL on GPUs, gloo
    on CPU (replica bookkeeping only: the data path has no collective)."""
    global _BACKEND
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        _BACKEND = backend
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(x, world, op):
    """Max or sum of a host scalar over the ranks."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _BACKEND == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# DRAM traffic of the roofline kernel (all-active last stage of the batched 2D
# workload) per stage kernel variant, from one ncu capture of each full-size
# launch.  It is reported only while the stage kernel sources are the ones
# those captures measured (code digest without comments and whitespace).
STAGE_TRAFFIC = {"workload": "batched2d",
                 # DRAM bytes per active element of the box kernel (8 elements
                 # per CTA, persistent grid of 3,040 CTAs) at the all-active
                 # last stage, from a capture of the first 128 instances
                 # (inputs well above L2); a launch's traffic scales with its
                 # elements
                 "bytes_per_element": {1: (764970240 + 370747136) / 763942},   # 128 instances, 0.994 of algorithmic
                 "sources_sha256": "3f331e99f58b8cdd5b3b767d7482a70af7c5be78e201fcc42c4213c2d9da5536"}
STAGE_SOURCES = ["stage.cuh", "stage_box.cuh", "physics.cuh", "dfloat.cuh", "kernels_stage2d.cu", "stage_launch.cu"]


def code_digest(paths):
    """sha256 of C++/CUDA sources with comments and whitespace removed: a
    comment edit leaves the digest (and the captured traffic) valid, any code
    change does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for path in paths:
        with open(path, "r", encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)      # block comments
        src = re.sub(r"//[^\n]*", "", src)                   # line comments
        h.update("".join(src.split()).encode())
    return h.hexdigest()


def stage_traffic(workload, variant, n_active):
    h = code_digest([os.path.join(ROOT, "paper_2507_04991_gb300", "csrc", f) for f in STAGE_SOURCES])
    ok = (workload == STAGE_TRAFFIC["workload"] and variant in STAGE_TRAFFIC["bytes_per_element"]
          and h == STAGE_TRAFFIC["sources_sha256"])
    return STAGE_TRAFFIC["bytes_per_element"][variant] * n_active if ok else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "of measured"
    return 6800.0, "of fallback"


def sample_instances(name, insts):
    """Instances the CPU oracle is timed on: the workload's own, except where
    one step of a single large instance would take minutes, where the same
    configuration at reduced resolution stands in (the oracle's cost per
    DOF-stage update does not depend on the mesh size)."""
    import workloads
    if name in ("tgv3d", "tgv3d_visc"):
        wl = workloads.tgv_3d(n=16, n_fine=4, mu=insts[0].mu)
        wl.prandtl = insts[0].prandtl
        return [wl], "the same configuration on 16^3 boxes (4 per axis at h/2)"
    if name == "khi2d":
        return [workloads.khi_2d(n=64)], "the same configuration on 64^2 quads"
    return insts, None


def _oracle_worker(insts, barrier, cmds, results, widx):
    """One host process of the all-cores oracle timing.  It builds the oracle
    solvers of its instances (untimed), then for every command `window`
    waits at a barrier shared by all processes and takes whole oracle steps
    of its instances in turn until `window` seconds have passed; it reports
    the DOF-stage updates of the completed steps and the time they took."""
    from oracle import perrk as operrk
    solvers = [(operrk.Solver(wl), wl) for wl in insts]
    k = 0
    while True:
        window = cmds.get()
        if window is None:
            return
        barrier.wait()
        t0 = time.clock_gettime(time.CLOCK_MONOTONIC)
        units, t1 = 0, t0
        while t1 - t0 < window:
            s, wl = solvers[k % len(solvers)]
            s.step(wl.dt)
            units += wl.dof_stage_per_step()
            k += 1
            t1 = time.clock_gettime(time.CLOCK_MONOTONIC)
        results.put((widx, units, t1 - t0))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The CPU oracle on all host cores: one spawned process per core (never
    forked after CUDA use), one numpy thread each.  Process w owns instances
    w, w + cores, ... of the first cores * per_core instances.  A round
    starts every process at a barrier and runs for a fixed window; its
    throughput is the sum over processes of completed DOF-stage updates over
    their own busy time (all processes are busy for the whole window, so the
    sum is the machine's aggregate rate, with the contention of all cores
    running at once)."""

    def __init__(self, insts, per_core, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        n = self.cores * per_core
        take = [insts[k % len(insts)] for k in range(n)]
        self.n_inst = min(n, len(insts))
        ctx = mp.get_context("spawn")
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"        # inherited at spawn
        self.barrier = ctx.Barrier(self.cores)
        self.results = ctx.Queue()
        self.cmds = [ctx.Queue() for _ in range(self.cores)]
        self.procs = [ctx.Process(target=_oracle_worker, args=(take[w::self.cores], self.barrier, self.cmds[w],
                                                                self.results, w), daemon=True)
                      for w in range(self.cores)]
        for p in self.procs:
            p.start()

    def round(self, window):
        for q in self.cmds:
            q.put(window)
        out = [self.results.get(timeout=900) for _ in self.procs]
        return sum(u / t for _, u, t in out), max(t for _, _, t in out)

    def close(self):
        for q in self.cmds:
            q.put(None)
        for p in self.procs:
            p.join(timeout=60)


def oracle_sample(insts, seconds_cap):
    """Time the CPU oracle on a bounded sample: whole steps of the workload's
    instances in order until about seconds_cap of work."""
    from oracle import perrk as operrk
    units, el, done = 0, 0.0, 0
    for wl in insts:
        s = operrk.Solver(wl)
        t0 = time.perf_counter()
        s.step(wl.dt)
        el += time.perf_counter() - t0
        units += wl.dof_stage_per_step()
        done += 1
        if el > seconds_cap:
            break
    return units / el, done, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    insts, desc = make_workload(args.workload)
    insts, s_note = sample_instances(args.workload, insts)
    from oracle import perrk as operrk
    solvers = {}

    def one(k):   # one bounded sample: one oracle step of instance k
        i = k % len(insts)
        wl = insts[i]
        if i not in solvers:
            solvers[i] = operrk.Solver(wl)
        t0 = time.perf_counter()
        solvers[i].step(wl.dt)
        return wl.dof_stage_per_step(), time.perf_counter() - t0

    cores = host_cores()
    if args.ref_cores == 1 or cores == 1:
        for k in range(args.warmup):
            one(k)
        units, el = 0, 0.0
        for k in range(args.steps):
            u, t = one(args.warmup + k)
            units += u
            el += t
        val = units / el
        used = 1
        sample = (f"{args.steps} oracle steps, each of one instance in turn (numpy float64, one host thread), "
                  f"after {args.warmup} warm-up steps" + (f"; {s_note}" if s_note else ""))
    else:
        # each timed step: a window of ref_window seconds in which every host
        # core takes whole oracle steps of its own instances
        pool = OraclePool(insts, 2, cores)
        # the timed windows of the whole run stay near 150 s whatever --steps
        # is (a window still completes at least one oracle step per process)
        window = min(args.ref_window, max(0.5, 150.0 / max(1, args.steps)))
        for _ in range(args.warmup):
            pool.round(min(1.0, window))
        rates, el = [], 0.0
        for _ in range(args.steps):
            r, t = pool.round(window)
            rates.append(r)
            el += t
        pool.close()
        val = float(np.mean(rates))
        used = cores
        sample = (f"{args.steps} timed windows of {window:g} s, in each every one of {cores} host processes "
                  f"(numpy float64, one thread each, started together at a barrier) takes whole oracle steps of its "
                  f"own instances ({pool.n_inst} instances in all); after {args.warmup} warm-up windows"
                  + (f"; {s_note}" if s_note else ""))
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {desc}"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch
    import paper_2507_04991_gb300 as pk
    import __graft_entry__
    world, rank, local = dist_setup()
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    pk.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    insts, desc = make_workload(args.workload, rank, args.instances, args.size)
    if args.instances:
        desc = f"the first {len(insts)} of: " + desc
    u0 = np.concatenate([w.u0 for w in insts], axis=1)
    dof_stage = sum(w.dof_stage_per_step() for w in insts)
    dof = sum(w.n_dof for w in insts)

    # ---- set-up (untimed): plain float64 batched context, gamma traces, learned guess
    plain = pk.Solver(insts, pk.options(precision=pk.FP64, use_graph=True, max_it=args.max_it))
    pk.perrk_autotune(plain.h, stream=sh)
    plain.set_state(u0)
    trace = plain.step(args.train_steps)
    X, T = pk.mlp_dataset(trace)
    W, mlp_loss = pk.mlp_fit(X, T, epochs=600, lr=3e-3)
    plain.set_state(u0)

    # The mixed form's Delta H carries FP32 rounding, which moves its root gamma
    # by ~1e-5..1e-4 from step to step; residuals below ~1e-13 A are below the
    # double-float entropy noise, so the mixed form stops at 1e-12 A.
    mixed_opts = dict(precision=pk.MIXED, use_graph=True, max_it=args.max_it, tol_r=args.mixed_tol_r)
    chosen = pk.Solver(insts, pk.options(guess=pk.GUESS_MLP, **mixed_opts))
    if args.tuning:
        epb, grid, var = (int(x) for x in args.tuning.split(","))
        pk.perrk_set_tuning(chosen.h, epb, grid, 128, var)
    else:
        pk.perrk_autotune(chosen.h, stream=sh)
    chosen.set_state(u0)
    chosen.set_mlp(W)
    tuning = pk.perrk_tuning(chosen.h)
    info0 = pk.perrk_stage_info(chosen.h, 0)
    S = info0["n_stages"]
    assert info0["dof_stage_per_step"] == dof_stage
    kernels_per_step = info0["kernels_per_step"]

    big_l2 = dof * 8 > 4 * 135 * 2 ** 20
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def ranged(name, fn):
        # an NVTX range around the launches, so a profiler can select them (ncu --nvtx --nvtx-include)
        def run():
            torch.cuda.nvtx.range_push(name)
            fn()
            torch.cuda.nvtx.range_pop()
        return run

    def timed(fn, nsteps):
        evs = []
        for _ in range(nsteps):
            l2_flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3

    for _ in range(args.warmup):
        pk.perrk_step(chosen.h, 1, info=False, stream=sh)
        pk.perrk_step(plain.h, 1, info=False, stream=sh)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t_chosen = timed(ranged("chosen_step", lambda: pk.perrk_step(chosen.h, 1, info=False, stream=sh)), args.steps)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_max = reduce_over_ranks(t_chosen, world, "max")
    value = reduce_over_ranks(dof_stage * args.steps, world, "sum") / t_max

    n_plain = max(2, args.steps // 4)
    t_plain = timed(lambda: pk.perrk_step(plain.h, 1, info=False, stream=sh), n_plain)
    plain_batched = dof_stage * n_plain / t_plain
    loop_value = None
    if len(insts) > 1:
        # the plain float64 form looped per instance (one context per instance)
        loop = [pk.Solver(w, pk.options(precision=pk.FP64, use_graph=True, max_it=args.max_it)) for w in insts]
        for sv in loop:
            pk.perrk_step(sv.h, 1, info=False, stream=sh)
        torch.cuda.synchronize()
        t_loop = timed(lambda: [pk.perrk_step(sv.h, 1, info=False, stream=sh) for sv in loop], 2)
        loop_value = dof_stage * 2 / t_loop
        for sv in loop:
            sv.close()

    # ---- matched error: both forms from u0, 10 steps
    chosen.set_state(u0)
    plain.set_state(u0)
    rc = chosen.step(10)
    rp = plain.step(10)
    uc, up = chosen.state(), plain.state()
    rel, off = 0.0, 0
    for w in insts:
        a, b = uc[:, off:off + w.n_elem], up[:, off:off + w.n_elem]
        rel = max(rel, float(np.abs(a - b).max() / np.abs(b).max()))
        off += w.n_elem
    def passes(recs):
        return float(np.mean([r["iters"] for row in recs[3:] for r in row]))

    def guess_err(recs):
        return float(np.mean([abs(r["gamma_guess"] - r["gamma"]) for row in recs[3:] for r in row]))

    passes_chosen = passes(rc)
    passes_plain = passes(rp)
    # the same mixed form with the method's own guesses: what the learned guess changes
    guesses = {"mlp": {"passes": passes_chosen, "mean_abs_guess_error": guess_err(rc)}}
    for gname, g in (("gamma_prev", pk.GUESS_PREV), ("one", pk.GUESS_ONE)):
        sv = pk.Solver(insts, pk.options(guess=g, **mixed_opts))
        sv.set_state(u0)
        r_ = sv.step(10)
        sv.close()
        guesses[gname] = {"passes": passes(r_), "mean_abs_guess_error": guess_err(r_)}
    guesses["fp64_gamma_prev"] = {"passes": passes_plain, "mean_abs_guess_error": guess_err(rp)}

    # ---- phases (the paper reports runtime shares of the relaxation and the
    # entropy integrand): the S stage launches of a step timed on their own,
    # the relaxation (relax_init, learned guess, Newton passes, update) as the
    # rest of the step
    t_stages = timed(lambda: [pk.perrk_launch_stage(chosen.h, i, stream=sh) for i in range(S)], 10) / 10
    phases = {"stages_ms": 1e3 * t_stages, "step_ms": 1e3 * t_max / args.steps,
              "relaxation_ms": max(0.0, 1e3 * (t_max / args.steps - t_stages)),
              "relaxation_share": max(0.0, 1.0 - t_stages / (t_max / args.steps))}

    # ---- dominant kernel: an all-active stage of the chosen form, timed live on the launching stream
    st = pk.perrk_stage_info(chosen.h, S - 1)
    k_s = timed(ranged("stage_all_active", lambda: pk.perrk_launch_stage(chosen.h, S - 1, stream=sh)), 20) / 20
    peak, peak_src = measured_peaks()
    achieved = st["bytes"] / k_s / 1e9
    # the plain float64 form's all-active last stage, timed live (its per-node
    # logarithms and divisions run on the FP64 pipe), and the FMA peaks of
    # this GPU measured by the library's probe
    st_p = pk.perrk_stage_info(plain.h, S - 1)
    k_p = timed(ranged("plain_stage_all_active", lambda: pk.perrk_launch_stage(plain.h, S - 1, stream=sh)), 5) / 5
    alu_peaks = {"fp32_tflops": pk.perrk_fma_peak(0, stream=sh), "fp64_tflops": pk.perrk_fma_peak(1, stream=sh)}

    # ---- end to end through the C ABI with host buffers (pinned): every step
    # copies its whole input state in and its whole result state out.  Three
    # contexts take the steps in turn on three streams with asynchronous
    # copies: a context's chain (copy in, set-up, step, copy out) is about
    # three steps long, so the host link and the kernels both stay busy.
    n_ctx = 3
    host_u = torch.from_numpy(np.ascontiguousarray(uc)).pin_memory()
    host_out = [torch.empty_like(host_u).pin_memory() for _ in range(n_ctx)]
    state_bytes = host_u.numel() * 8
    ctxs = [chosen]
    for _ in range(n_ctx - 1):
        extra = pk.Solver(insts, pk.options(guess=pk.GUESS_MLP, **mixed_opts))
        pk.perrk_set_tuning(extra.h, tuning["elems_per_cta"], tuning["persistent_grid"], tuning["relax_threads"],
                            tuning["stage_variant"])
        extra.set_mlp(W)
        ctxs.append(extra)
    # side streams for every context (the current stream may be the legacy
    # default stream, which would serialise with the others)
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_ctx)]
    for X in range(n_ctx):                                 # capture each context's graph outside the timing
        pk.perrk_set_state(ctxs[X].h, host_u.data_ptr(), on_device=pk.STATE_HOST_ASYNC, stream=streams[X].cuda_stream)
        pk.perrk_step(ctxs[X].h, 1, info=False, stream=streams[X].cuda_stream)
    torch.cuda.synchronize()
    # a fixed number of steps, independent of --steps: a short pipeline is
    # mostly fill and drain (the first copy in and the last copy out overlap
    # nothing)
    # the host link's rate on these pinned buffers in this process (untimed,
    # reported beside e2e: it bounds the pipeline and varies between boxes)
    link = {}
    dev_tmp = torch.empty_like(host_u, device=dev)
    for name, fn in (("h2d", lambda: dev_tmp.copy_(host_u, non_blocking=True)),
                     ("d2h", lambda: host_out[0].copy_(dev_tmp, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        t_l = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        link[name + "_gbs"] = 3 * state_bytes / (time.perf_counter() - t_l) / 1e9
    dev_tmp2 = torch.empty_like(dev_tmp)
    torch.cuda.synchronize()
    t_l = time.perf_counter()
    for _ in range(3):
        with torch.cuda.stream(streams[0]):
            dev_tmp.copy_(host_u, non_blocking=True)
        with torch.cuda.stream(streams[1]):
            host_out[0].copy_(dev_tmp2, non_blocking=True)
    torch.cuda.synchronize()
    link["both_gbs"] = 6 * state_bytes / (time.perf_counter() - t_l) / 1e9
    del dev_tmp, dev_tmp2
    # Each step waits for the previous context's step (an event), so the
    # steps run one after another while the copies, the split and the join of
    # the other contexts overlap them; left to themselves the three streams
    # can fall into computing together and then copying together.
    e2e_steps = args.e2e_steps
    done_ev = [torch.cuda.Event() for _ in range(e2e_steps)]
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        X = k % n_ctx
        sX = streams[X].cuda_stream
        pk.perrk_set_state(ctxs[X].h, host_u.data_ptr(), on_device=pk.STATE_HOST_ASYNC, stream=sX)
        if k > 0:
            streams[X].wait_event(done_ev[k - 1])
        pk.perrk_step(ctxs[X].h, 1, info=False, stream=sX)
        done_ev[k].record(streams[X])
        pk.perrk_get_state(ctxs[X].h, host_out[X].data_ptr(), on_device=pk.STATE_HOST_ASYNC, stream=sX)
    torch.cuda.synchronize()
    e2e_time = reduce_over_ranks(time.perf_counter() - t0, world, "max")
    e2e_value = reduce_over_ranks(dof_stage * e2e_steps, world, "sum") / e2e_time
    e2e_match = all(bool(torch.equal(host_out[0], o)) for o in host_out[1:])   # all contexts stepped the same input
    for extra in ctxs[1:]:
        extra.close()

    if rank != 0:
        return
    s_insts, s_note = sample_instances(args.workload, insts)
    cpu = oracle_sample(s_insts, args.cpu_seconds) if args.cpu_seconds > 0 else (None, 0, 0.0)
    if args.cpu_per_core > 0:
        pool = OraclePool(s_insts, args.cpu_per_core)
        pool.round(1.0)                                   # warm-up window
        cpu_all = (pool.round(args.cpu_window)[0], pool.cores, pool.n_inst, args.cpu_window)
        pool.close()
    else:
        cpu_all = (None, 1, 0, 0.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_CHOSEN, "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "instances": len(insts), "dof": dof,
                   "dof_stage_per_step": dof_stage,
                   "form": "chosen: batched instances, FP32 flux differencing, surface fluxes and stage registers "
                           "K_i; state, direction, entropy passes and update as float pairs (~48-bit); float64 "
                           "Newton scalars and Delta H; learned Newton guess, autotuned mapping, one CUDA graph "
                           "per step",
                   "autotuned_mapping": tuning, "newton_max_it": args.max_it,
                   "l2": ("inputs larger than L2; " if big_l2 else "") + "L2 flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "plain_fp64": {"per_instance_loop": loop_value, "batched": plain_batched,
                       "stage_all_active_ms": 1e3 * k_p, "stage_all_active_gbs": st_p["bytes"] / k_p / 1e9,
                       "alu_peaks_measured": alu_peaks,
                       "ratio_chosen_vs_loop": (value / world / loop_value) if loop_value else None,
                       "ratio_chosen_vs_batched": value / world / plain_batched},
        "matched_error": {"chosen_vs_fp64_max_rel_linf_after_10_steps": rel,
                          "fp64_vs_oracle": "tests/test_gpu_parity.py, tests/test_gpu_batched.py",
                          "newton_passes_per_step_chosen": passes_chosen,
                          "newton_passes_per_step_fp64_prev_guess": passes_plain, "mlp_train_loss": mlp_loss,
                          "newton_guess_comparison_steps_4_to_10": guesses,
                          "newton_tol_r": {"mixed": args.mixed_tol_r, "fp64": 1e-14}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": stage_traffic(args.workload, tuning["stage_variant"], st["n_active"]), "kernel": f"k_stage (stage {S}, {st['n_active']} elements, all active)",
                     "algorithmic_bytes": st["bytes"], "kernel_ms": 1e3 * k_s, "peak_source": peak_src},
        "cpu_baseline": {"value": cpu_all[0], "unit": UNIT, "cores": cpu_all[1], "kind": "oracle",
                         "sample": f"a {cpu_all[3]:g} s window in which each of {cpu_all[1]} host processes "
                                   f"(numpy float64, one thread each, started together at a barrier) takes whole "
                                   f"oracle steps of its own share of the first {cpu_all[2]} instances, after a 1 s "
                                   f"warm-up window" + (f"; {s_note}" if s_note else ""),
                         "one_core": {"value": cpu[0], "cores": 1,
                                      "sample": f"one oracle step each of the first {cpu[1]} instances "
                                                f"({cpu[2]:.1f} s, one thread)"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "pipeline": f"{n_ctx} contexts, {n_ctx} streams, asynchronous pinned copies",
                "results_agree": e2e_match, "host_link": link},
        "phases": phases,
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_amr(args):
    """Adaptive KHI run (Sec. 3.2.2: the mesh changes every 7th step): a
    16 x 16 quadtree on [-1, 1]^2 refined once where the density indicator
    is large (thresholds 2e-4 / 1e-3 of the three-level controller, which
    keep one refined band around each shear layer), partitions from the
    levels (E = 6, 3 for levels 1, 0), the chosen numerics (mixed form, CUDA
    graph, default box-kernel mapping).  value = DOF-stage updates of all steps over the wall time of
    steps and adaptations together; the adaptation share is reported."""
    import torch
    import paper_2507_04991_gb300 as pk
    from paper_2507_04991_gb300 import amr as pamr
    import __graft_entry__
    import workloads
    __graft_entry__.build()
    pk.load()
    sh = torch.cuda.current_stream().cuda_stream
    n, L, max_level, every = 16, 1.0, 1, 7
    dt = 0.3 * (2 * L / (n << max_level)) / 7 / 2.5
    u0 = workloads.quadtree_workload(workloads.Quadtree.uniform(n, L), "khi", (3,), 3, ic="khi").u0
    opts = pk.options(precision=pk.MIXED, use_graph=True, max_it=args.max_it, tol_r=args.mixed_tol_r)
    thresholds, levels = (2e-4, 1e-3), (0, 1, 1)
    run = pamr.AmrRun(pamr.QuadMesh.uniform(n, L), u0, [6, 3], 3, dt, opts, max_level)
    for _ in range(2):                                   # reach the refined mesh before timing
        run.adapt(thresholds, levels)
    cycles = max(1, (args.steps + every - 1) // every)
    units, t_adapt, launches = 0, 0.0, 0
    for _ in range(args.warmup):
        pk.perrk_step(run.solver.h, 1, info=False, stream=sh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(cycles):
        # the adaptation: indicator, mesh, context of the new mesh, transfer,
        # and the new context's first step (which captures its step graph)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        run.adapt(thresholds, levels)
        pk.perrk_step(run.solver.h, 1, info=False, stream=sh)
        torch.cuda.synchronize()
        t_adapt += time.perf_counter() - ta
        info = pk.perrk_stage_info(run.solver.h, 0)
        pk.perrk_step(run.solver.h, every - 1, info=False, stream=sh)
        units += every * info["dof_stage_per_step"]
        launches += every * info["kernels_per_step"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lv = np.bincount(run.mesh.levels(), minlength=2).tolist()
    line = {"metric": METRIC, "value": units / wall, "unit": UNIT, "n_gpus": 1, "steps": cycles * every,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / (cycles * every), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_CHOSEN, "data": "synthetic",
            "config": {"workload": "khi2d_amr: Kelvin-Helmholtz on a 16x16 quadtree over [-1,1]^2, one level of refinement "
                                   "by the density indicator (thresholds 2e-4, 1e-3), adapted every 7th step, "
                                   "partitions from the levels (E = 6, 3), p=3, ES, mixed form, CUDA graph",
                       "elements_at_end": len(run.mesh.leaves), "level_histogram_at_end": lv,
                       "mortars_at_end": int(run.mesh.arrays()[2].shape[0]),
                       "includes": "adaptation (indicator, mesh, context creation, transfer) inside the wall time; "
                                   "default stage mapping (box kernel, 8 elements per CTA)"},
            "amr": {"adapt_seconds": t_adapt, "adapt_share": t_adapt / wall, "cycles": cycles,
                    "parts_seconds": dict(run.adapt_parts),
                    "note": "adapt_seconds include each new context's first step (graph capture)"},
            "gpu_launches": launches}
    run.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batched2d")
    ap.add_argument("--size", type=int, default=None,
                    help="khi2d / tgv3d: cells per direction instead of 256 / 64 (smaller cases for profiling)")
    ap.add_argument("--instances", type=int, default=None,
                    help="batched2d: use only the first N instances (profiling on a reduced case)")
    ap.add_argument("--max-it", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bound of the one-thread oracle sample")
    ap.add_argument("--cpu-per-core", type=int, default=2,
                    help="instances per host process in the all-cores oracle sample (0: skip)")
    ap.add_argument("--ref-cores", type=int, default=0, help="--impl reference: 1 = one thread, 0 = all host cores")
    ap.add_argument("--e2e-steps", type=int, default=48, help="steps of the end-to-end pipeline (fixed)")
    ap.add_argument("--cpu-window", type=float, default=6.0, help="seconds of the all-cores oracle window")
    ap.add_argument("--ref-window", type=float, default=3.0, help="--impl reference: seconds per timed window")
    ap.add_argument("--mixed-tol-r", type=float, default=1e-12)
    ap.add_argument("--tuning", default=None,
                    help="EPB,GRID,VARIANT: pin the chosen form's stage mapping instead of autotuning it "
                         "(reproducible profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "khi2d_amr":
        run_amr(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
