"""Precision control through the C ABI: the FP32 march's a-posteriori
rounding indicator bounds its measured error against the FP64 oracle, and
MIXED re-runs in FP64 exactly the instruments whose indicator misses the
tolerance max(tol_rel |p|, 1e-6)."""
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


def _instruments():
    items = [W.config1(), W.paper_2007_set(n_r=24, n_y=10, n_v=10, n_steps=60)]
    items += W.config2_draws(6, seed=W.SEED_BASE + 40, n_r=64, n_y=24, n_v=24, n_steps=120)
    items += W.config3_batch(6, sizes=(64, 96))
    for x in items[-6:]:
        x["grid"]["n_steps"] = 96
    b = W.config1()
    b["grid"].update(n_steps=600)  # many steps: rounding of U accumulates
    items.append(b)
    return items


def test_indicator_bounds_fp32_error(H, orc):
    items = _instruments()
    want = np.array([orc.price(x) for x in items])
    p32, inf = H.hjm_price_batch(items, "fp32", infos=True)
    err = np.abs(p32 - want)
    ind = np.array([inf[i].err_estimate for i in range(len(items))])
    assert np.all(ind > 0)
    assert np.all(err <= ind), list(zip(err, ind))
    # FP64 indicators are at FP64 roundoff scale
    p64, inf64 = H.hjm_price_batch(items, "fp64", infos=True)
    ind64 = np.array([inf64[i].err_estimate for i in range(len(items))])
    assert np.all(ind64 < 1e-9 * np.maximum(np.abs(p64), 1.0))
    assert np.all(np.abs(p64 - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3))


def test_indicator_bounds_fp32_error_at_benchmark_size(H, orc):
    # The safety factor C = 8 of the indicator was fitted on small grids;
    # here three caplets of the 100-caplet benchmark batch at its full size
    # (128 x 64 x 64, 400 steps) against the oracle (its OpenMP build, same
    # results as the serial one): the indicator must still bound the FP32
    # march's error, and MIXED at the stated 1e-4 keeps every FP32 price.
    items = [W.config2_draws(100)[i] for i in (0, 50, 99)]
    want = np.array([orc.price(x, omp=True) for x in items])
    p32, inf = H.hjm_price_batch(items, "fp32", infos=True)
    err = np.abs(p32 - want)
    ind = np.array([inf[i].err_estimate for i in range(len(items))])
    assert np.all(err <= ind), list(zip(err, ind))
    assert np.all(ind <= 1e-4 * np.abs(p32)), list(zip(ind, p32))
    pm, infm = H.hjm_price_batch(items, "mixed", tol_rel=1e-4, infos=True)
    assert np.array_equal(pm, p32) and not any(infm[i].escalated for i in range(len(items)))


def test_mixed_keeps_fp32_when_within_tolerance(H):
    items = W.config2_draws(4, seed=W.SEED_BASE + 41, n_r=48, n_y=16, n_v=16, n_steps=60)
    p32 = H.hjm_price_batch(items, "fp32")
    pm, inf = H.hjm_price_batch(items, "mixed", tol_rel=1e-4, infos=True)
    assert np.array_equal(pm, p32)
    assert all(inf[i].escalated == 0 and inf[i].precision_used == H.HJM_FP32 for i in range(4))


def test_mixed_escalates_exactly_the_flagged_items(H, torch_dev):
    torch = torch_dev
    long_bond = W.config1()
    long_bond["grid"].update(n_steps=600)
    items = W.config2_draws(3, seed=W.SEED_BASE + 42, n_r=48, n_y=16, n_v=16, n_steps=60)
    items.insert(1, long_bond)
    p32, i32 = H.hjm_price_batch(items, "fp32", infos=True)
    p64 = H.hjm_price_batch(items, "fp64")
    tol = 1e-7
    flagged = [i32[i].err_estimate > max(tol * abs(p32[i]), 1e-6) for i in range(len(items))]
    assert flagged[1] and not any(flagged[:1] + flagged[2:])
    out = torch.empty(len(items), dtype=torch.float64, device="cuda")
    _, inf = H.hjm_price_batch(items, "mixed", tol_rel=tol, out=out, infos=True)
    got = out.cpu().numpy()
    for i in range(len(items)):
        if flagged[i]:
            # the escalation march (FP32 increments on an FP64 state), or FP64
            # where its bound still misses
            assert inf[i].escalated == 1 and inf[i].precision_used in (H.HJM_MIXED, H.HJM_FP64)
            if inf[i].precision_used == H.HJM_FP64:
                assert got[i] == p64[i]
            else:
                assert abs(got[i] - p64[i]) <= inf[i].err_estimate
                assert inf[i].err_estimate <= max(tol * abs(got[i]), 1e-6)
        else:
            assert got[i] == p32[i] and inf[i].escalated == 0 and inf[i].precision_used == H.HJM_FP32


def test_escalation_march_against_the_oracle(H, orc):
    # tol_rel = 0 sends every instrument through the escalation: the Douglas
    # ones through the march of FP32 increments on an FP64 state, whose
    # indicator must bound its error against the oracle and whose error must
    # be well below the FP32 march's; a Craig-Sneyd item goes to FP64.
    items = _instruments()
    cs = W.with_grid(W.config2_draws(1, seed=W.SEED_BASE + 43, n_r=48, n_y=16, n_v=16, n_steps=40)[0],
                     scheme=1, theta_adi=0.5)
    items.append(cs)
    want = np.array([orc.price(x) for x in items])
    p32 = H.hjm_price_batch(items, "fp32")
    pm, inf = H.hjm_price_batch(items, "mixed", tol_rel=0.0, infos=True)
    err32, errm = np.abs(p32 - want), np.abs(pm - want)
    ind = np.array([i.err_estimate for i in inf])
    used = [i.precision_used for i in inf]
    assert all(i.escalated == 1 for i in inf)
    assert used[-1] == H.HJM_FP64 and pm[-1] == H.hjm_price_batch([cs], "fp64")[0]
    assert all(u == H.HJM_MIXED for u in used[:-1]), used
    assert np.all(errm[:-1] <= ind[:-1]), list(zip(errm, ind))
    # the state no longer carries an FP32 rounding per step
    assert errm[:-1].sum() <= 0.25 * err32[:-1].sum(), (errm.sum(), err32.sum())


def test_single_price_mixed(H):
    long_bond = W.config1()
    long_bond["grid"].update(n_steps=600)
    with H.Grid(long_bond) as g:
        p64 = g.price("fp64")
        pm, info = H.hjm_price(g.h, long_bond["inst"], "mixed", tol_rel=1e-9, with_info=True)
        assert info.escalated == 1
        if info.precision_used == H.HJM_FP64:
            assert pm == p64
        else:  # the escalation march, within its bound of the FP64 march
            assert info.precision_used == H.HJM_MIXED and abs(pm - p64) <= info.err_estimate <= 1e-6


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    return torch


def test_non_finite_price_is_reported(H, orc):
    # A valid but absurd input (lambda = 30: the domain reaches |r| ~ 1000
    # and the Dirichlet bond prices overflow) gives a non-finite price, as in
    # the oracle; every precision reports HJM_ENUMERIC for that item instead
    # of returning it (MIXED after its FP64 re-run). No device fault: IEEE
    # infinities and NaNs only.
    c = W.flat_curve(0.03)
    m = W.model(0.1, 30.0, 0.0, 1.0, 0.3, -0.3)
    bad = W.item(c, m, W.default_grid(c, m, 5.0, 16, 8, 8, 4), W.bond(5.0))
    assert not np.isfinite(orc.price(bad))
    items = [W.config1(), bad]
    for prec in ("fp32", "fp64", "mixed"):
        with pytest.raises(H.HJMError) as ei:
            H.hjm_price_batch(items, prec)
        assert ei.value.status == H.HJM_ENUMERIC and "item 1" in str(ei.value), prec
    # the library stays usable
    assert abs(H.hjm_price_batch([W.config1()], "fp64")[0] - orc.price(W.config1())) < 1e-12
