"""Host-side helpers of bench.py (no GPU): the code digest that keeps a
captured DRAM-traffic figure valid only while the kernel code is unchanged,
and the bounded CPU-oracle samples."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_digest_ignores_comments_not_code(tmp_path):
    b = _bench()
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(float *x) {\n  x[0] = 1.0f; /* one */\n}\n")
    ref = b.code_digest([str(a)])
    a.write_text("// another header\n\n__global__ void k(float *x)  {\n\tx[0] = 1.0f;   // set\n}\n")
    assert b.code_digest([str(a)]) == ref
    a.write_text("__global__ void k(float *x) {\n  x[0] = 2.0f;\n}\n")
    assert b.code_digest([str(a)]) != ref


def test_stage_traffic_only_for_its_workload():
    b = _bench()
    assert b.stage_traffic("khi2d", 1, 100) is None
    assert b.stage_traffic("batched2d", 7, 100) is None


def test_cpu_samples_are_bounded():
    """Single large instances are sampled at reduced resolution; batched
    instances are sampled as they are."""
    b = _bench()
    import workloads
    big = [workloads.tgv_3d(n=8, n_fine=2, mu=0.01)]
    s, note = b.sample_instances("tgv3d_visc", big)
    assert note and s[0].n_elem == 16 ** 3 and s[0].mu == big[0].mu
    small = [workloads.small_box_2d(n=4)]
    assert b.sample_instances("batched2d", small) == (small, None)


def test_all_cores_oracle_pool_runs_windows():
    """The all-cores oracle timing: spawned processes, a barrier per window,
    a positive aggregate rate from every process's completed steps."""
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b          # by name: the spawned processes import it the same way
    import workloads
    insts = [workloads.small_box_2d(n=4, seed=k) for k in range(3)]
    pool = b.OraclePool(insts, per_core=1, cores=2)
    try:
        rate, busy = pool.round(0.2)
        assert rate > 0 and busy >= 0.2
        rate2, _ = pool.round(0.2)
        assert rate2 > 0
    finally:
        pool.close()
    assert all(not p.is_alive() for p in pool.procs)


def test_make_workload_size_option():
    """--size gives the same single-mesh configuration on a smaller mesh
    (profiling captures): cells per direction, partitions and schemes kept."""
    import bench
    (k,), _ = bench.make_workload("khi2d", size=16)
    (t,), _ = bench.make_workload("tgv3d", size=8)
    assert k.n_elem == 16 * 16 and k.E == [16, 10, 7, 5] and k.order == 4
    assert t.n_elem == 8 ** 3 and t.E == [8, 4] and t.order == 3
    assert set(t.part.tolist()) == {0, 1}
    (b,), _ = bench.make_workload("khi2d")
    assert b.n_elem == 256 * 256
