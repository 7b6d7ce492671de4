"""Host-side logic of bench.py on the CPU: the multi-rank reduction (two gloo
ranks), the workload bookkeeping and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_BACKEND="gloo")
    w, r, _ = bench.dist_setup(world)
    v = bench.reduce_max(10.0 + r, w, device="cpu")
    bench.barrier(w)
    q.put((r, v))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert got == [(0, 11.0), (1, 11.0)]


def test_workload_sizes():
    items, desc = bench.workload_items("config2")
    assert len(items) == 100 and "128x64x64" in desc
    assert bench.point_steps(items) == 100 * 128 * 64 * 64 * 400
    items, _ = bench.workload_items("config3")
    assert len(items) == 256


@pytest.mark.parametrize("scheme,code", [("cs", 1), ("mcs", 2), ("hv", 3)])
def test_workload_scheme_option(scheme, code):
    items, desc = bench.workload_items("config2", instruments=3, march_steps=10, scheme=scheme)
    assert all(x["grid"]["scheme"] == code for x in items)
    assert abs(items[0]["grid"]["theta_adi"] - bench.SCHEMES[scheme][1]) == 0.0
    assert scheme.upper() + " scheme" in desc
    plain, _ = bench.workload_items("config2", instruments=3, march_steps=10)
    assert all(x["grid"]["scheme"] == 0 and x["grid"]["theta_adi"] == 0.5 for x in plain)


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--workload", "config1",
                        "--ref-steps-per-step", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_source_digest_is_stable():
    assert bench.source_digest() == bench.source_digest()
    assert len(bench.source_digest()) == 16


def test_kernel_names_of_launch_shapes():
    # the roofline line names the kernel a launch shape runs
    assert bench.kernel_name("pass1", (16, 8, 8, 1, 4, 0, 0)) == "k_pass1_r96"
    assert bench.kernel_name("pass1", (16, 8, 8, 1, 4, 0, 0), "fp64") == "k_pass1"
    assert bench.kernel_name("pass1", (16, 8, 8, 1, 4, 0, 0), "fp32", 3) == "k_pass1"
    assert bench.kernel_name("pass1", (32, 16, 8, 8, 8, 0, 0)) == "k_pass1"
    assert bench.kernel_name("pass1", (8, 16, 1, 1, 4, 1, 16)) == "k_pass1s"
    assert bench.kernel_name("pass1", (16, 8, 1, 1, 4, 1, 16)) == "k_pass1s_r96"
    assert bench.kernel_name("pass2", (16, 8, 8, 1, 4, 0, 0)) == "k_pass2"
    assert bench.kernel_name("pass3", (16, 8, 8, 1, 4, 0, 0)) == "k_split_lines"
    assert bench.kernel_name("pass3", (16, 8, 8, 0, 1, 0, 0)) == "k_pass23"
    assert bench.kernel_name("pass1", (8, 16, 1, 1, 4, 2, 16)) == "k_pass1t"
    assert bench.kernel_name("pass1", (16, 8, 1, 1, 4, 3, 0)) == "k_pass1t"
    assert bench.kernel_name("pass2", (16, 8, 1, 15, 15, 3, 0)) == "k_lines_t"
    assert bench.kernel_name("pass3", (16, 8, 1, 15, 15, 3, 0)) == "k_lines_t"


def test_recorded_traffic_is_keyed_by_sources_and_launch_shape():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    shapes = d["workloads"]["config2-fp32"]["tiles"]
    tile = sorted(shapes)[0]
    assert bench.recorded_traffic("pass1", "config2-fp32", 1000, "1,2,3,4,5,6,7") is None
    assert bench.recorded_traffic("pass1", "no-such-workload", 1000, tile) is None
    for kind, rec in shapes[tile]["kernels"].items():
        got = bench.recorded_traffic(kind, "config2-fp32", 1000, tile)
        if rec["source_digest"] == bench.source_digest(rec["kernel"]):
            assert got == rec["dram_bytes_per_point"] * 1000
        else:  # counters taken on other sources of that kernel are not reported
            assert got is None


def test_kernel_digests_cover_their_sources():
    # every recorded kernel's digest reads files that exist, and a kernel's
    # digest does not depend on another kernel's translation unit
    for k, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_1108_1688_gb300", "csrc", f)), (k, f)
        assert len(bench.source_digest(k)) == 16
    assert "hjm_pass1.cu" not in bench.KERNEL_SOURCES["k_pass1t"]
    assert "hjm_march.cu" not in bench.KERNEL_SOURCES["k_lines_t"]


def test_pass1_fp64_operation_count():
    # 16 lanes of 8 nodes: 15 + 19 + 13 per point and, per lane,
    # 8 + 54 + 25 + 9 + 14 + 4 * 14 + 4 + 24 = 194 for the solve, 24.25 a point
    assert bench.pass1_flops_per_point(16, 8) == 71.25
    # two-node chunks: no backward elimination, no first-row reduction
    assert bench.pass1_flops_per_point(1, 2) == 47 + (8 + 14 + 4) / 2
    # more lanes per line add parallel-cyclic-reduction levels, longer
    # chunks amortise them
    assert bench.pass1_flops_per_point(32, 8) > bench.pass1_flops_per_point(16, 8)
    assert bench.pass1_flops_per_point(16, 16) < bench.pass1_flops_per_point(16, 8)
    assert abs(bench.FP64_PEAK_TFLOPS - 1.259) < 1e-3
