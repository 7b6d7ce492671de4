"""hjm_price_static: the allocation-free entry point, for callers that cannot
allocate device memory (device memory owned by another allocator or a fixed
pool, latency-critical loops that cannot take cudaMalloc's implicit
synchronisation). Checked through the C ABI against
hjm_price, the allocating entry point, on two calls in a row (the second
reuses the static scratch array left by the first). This file is collected
last so that a run stopping at its first failure has run everything else."""
import pytest

from paper_1108_1688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1688_gb300 import _build
    _build.build()
    from paper_1108_1688_gb300 import hjm
    return torch, hjm


def _cases():
    cap = W.config2_draws(1, seed=W.SEED_BASE + 77, n_r=48, n_y=16, n_v=16, n_steps=40)[0]
    return [("bond_fp64", W.config1(), "fp64"), ("bond_fp32", W.config1(), "fp32"),
            ("caplet_fp64", cap, "fp64"), ("caplet_fp32", cap, "fp32"),
            ("bond_gamma09_fp64", W.paper_2007_set(n_r=20, n_y=8, n_v=9, n_steps=30), "fp64")]


def _close(got, want, prec):
    if prec == "fp64":
        return abs(got - want) <= 1e-10 * max(abs(want), 1e-3)
    return abs(got - want) <= max(1e-4 * abs(want), 1e-6)


@pytest.mark.parametrize("name,item,prec", _cases(), ids=[c[0] for c in _cases()])
def test_static_price_matches_allocating_entry_point(env, name, item, prec):
    torch, H = env
    with H.Grid(item) as g:
        want = g.price(prec)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out.fill_(float("nan"))
        H.hjm_price_static(item, prec, out, stream)
        torch.cuda.synchronize()
        got = out.item()
        assert _close(got, want, prec), (got, want)


def test_static_rejects_items_beyond_the_array(env):
    torch, H = env
    big = W.config2_draws(1, n_r=128, n_y=64, n_v=64, n_steps=8)[0]  # 2 x 4 MiB FP64 fields
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HJMError) as ei:
        H.hjm_price_static(big, "fp64", out)
    assert ei.value.status == H.HJM_ERANGE and "static array" in str(ei.value)
    with pytest.raises(H.HJMError) as ei:
        H.hjm_price_static(W.config1(), "fp64", __import__("numpy").zeros(1))
    assert ei.value.status == H.HJM_EINVAL
