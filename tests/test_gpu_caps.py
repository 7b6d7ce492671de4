"""Floorlets, caps and floors through the C ABI against the CPU FP64 oracle:
the floorlet's terminal field (the Section 7.2 cell average of
max(Delta_M p(T,T_M) - 1, 0)) element by element, whole marches in FP64
(within 1e-10) and FP32 (within max(1e-4 |p|, 1e-6)), the put-call parity of
the discrete march (caplet - floorlet against P(0,T) - Delta_M P(0,T_M), the
GPU's gap equal to the oracle's), and strips (hjm_price_strip: a cap or
floor is the sum of its periods; malformed strips are refused)."""
import numpy as np
import pytest

from paper_1108_1688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1688_gb300 import _build
    _build.build()
    from paper_1108_1688_gb300 import hjm
    return hjm


def _pair(seed, n_r=48, n_y=24, n_v=24, n_steps=48, K=0.003):
    d = W.config2_draws(1, seed=W.SEED_BASE + 900 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    c, m, g = d["curve"], d["model"], dict(d["grid"], explicit_midpoint=1)
    T, TM = d["inst"]["T"], d["inst"]["TM"]
    return W.item(c, m, g, W.caplet(T, TM, K)), W.item(c, m, g, W.floorlet(T, TM, K))


def test_floorlet_terminal_field(H, orc):
    import torch
    _, flo = _pair(0)
    g = flo["grid"]
    with orc.Ctx(flo) as X, H.Grid(flo) as gr:
        want = X.terminal()
        out = torch.empty(gr.shape, dtype=torch.float64, device="cuda")
        gr.field("fp64", 0, out)
        got = out.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.abs(want).max())
    assert np.any(want > 0) and np.any(want == 0) and g["n_r"] == want.shape[2]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_floorlet_prices_match_oracle(H, orc, seed):
    cap, flo = _pair(seed, K=0.002 * (seed - 2))
    want = orc.price(flo)
    p64 = H.hjm_price_batch([flo], "fp64")[0]
    assert abs(p64 - want) <= 1e-10 * max(abs(want), 1e-3), (p64, want)
    p32 = H.hjm_price_batch([flo], "fp32")[0]
    assert abs(p32 - want) <= max(1e-4 * abs(want), 1e-6), (p32, want)


def test_discrete_put_call_parity(H, orc):
    # caplet - floorlet on the same grid: the GPU's gap to the forward contract
    # equals the oracle's (they march the same discrete scheme); the gap
    # itself is discretisation error (its convergence is pinned in the oracle
    # tests), here a coarse-grid sanity bound (measured 1.4e-3 of the price
    # with F at t^{n+1/2})
    cap, flo = _pair(4, K=0.001)
    c = cap["curve"]
    T, TM = cap["inst"]["T"], cap["inst"]["TM"]
    with orc.Ctx(cap) as X:
        K = X.strike
    fwd = orc.curve_P(c, T) - (1.0 + (TM - T) * K) * orc.curve_P(c, TM)
    pc, pf = H.hjm_price_batch([cap, flo], "fp64")
    oc, of = orc.price(cap), orc.price(flo)
    assert abs((pc - pf) - (oc - of)) <= 1e-10 * abs(fwd) + 1e-14
    assert abs((pc - pf) - fwd) <= 5e-3 * max(pc, pf)


def _strip(kind, count=4, K=0.03):
    c = W.ns_curve(0.03, -0.01, 0.012, 2.0)
    m = W.model(0.1, 0.011, 0.0, 1.0, 0.35, -0.3)
    return W.strip(c, m, 1.0, 0.5, count, K, kind=kind, n_r=48, n_y=24, n_v=24, steps_per_year=16,
                   explicit_midpoint=1)


@pytest.mark.parametrize("kind", [1, 2])
def test_strip_is_the_sum_of_its_periods(H, orc, kind):
    items = _strip(kind)
    total, each = H.hjm_price_strip(items, "fp64")
    assert each == pytest.approx(list(H.hjm_price_batch(items, "fp64")), rel=0, abs=0)
    assert total == pytest.approx(sum(each), rel=1e-15)
    want = [orc.price(x) for x in items]
    assert np.allclose(each, want, rtol=1e-10, atol=1e-14)


def test_cap_minus_floor_is_the_swap(H):
    # Summed over the strip, caplet - floorlet parity gives the payer swap
    # sum_i P(0,T_i) - Delta P(0,T_i + tenor), up to discretisation error
    # (measured 7e-4 of the cap with F at t^{n+1/2}).
    from oracle import curve_P
    caps, floors = _strip(1), _strip(2)
    cap, _ = H.hjm_price_strip(caps, "fp64")
    floor, _ = H.hjm_price_strip(floors, "fp64")
    c = caps[0]["curve"]
    swap = sum(curve_P(c, x["inst"]["T"]) - (1.0 + 0.5 * 0.03) * curve_P(c, x["inst"]["TM"]) for x in caps)
    assert abs((cap - floor) - swap) <= 5e-3 * max(cap, floor)


def test_malformed_strips_are_refused(H):
    items = _strip(1)
    bad = [items[0], items[2]]  # a gap between the periods
    with pytest.raises(H.HJMError):
        H.hjm_price_strip(bad, "fp32")
    mixed = [items[0]] + _strip(2)[1:2]  # a caplet and a floorlet
    with pytest.raises(H.HJMError):
        H.hjm_price_strip(mixed, "fp32")
    k2 = [dict(x) for x in items]
    k2[1] = dict(k2[1], inst=dict(k2[1]["inst"], K=0.031))  # two strikes
    with pytest.raises(H.HJMError):
        H.hjm_price_strip(k2, "fp32")
