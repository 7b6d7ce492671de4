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
