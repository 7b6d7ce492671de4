"""The discrete initial curve (Section 6.1: discount factors at knots,
smoothed by the natural cubic spline of ln P that the set-up kernel builds)
on the GPU against the CPU FP64 oracle, through the C ABI: axis tables
(the r metric is centred at f(0,0) for a bond), terminal field, whole
marches (field and price) for bonds and caplets in FP64 and FP32, with the
Douglas and the Hundsdorfer-Verwer schemes, batches mixing curve kinds, and
the validation of bad knots. Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

from paper_1108_1688_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "fp32"]


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1688_gb300 import _build
    _build.build()
    from paper_1108_1688_gb300 import hjm
    return hjm


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _item(seed, inst, n_r, n_y, n_v, n_steps, times=W.MARKET_KNOT_TIMES, **grid_kw):
    c = W.synthetic_knot_curve(seed, times=times)
    m = W.model(0.1, 0.01, 0.0, 1.0, 0.4, -0.5)
    T = inst["T"]
    g = W.default_grid(c, m, T, n_r, n_y, n_v, n_steps, **grid_kw)
    return W.item(c, m, g, inst)


CASES = {
    "bond_5y_40x20x20": lambda: _item(1, W.bond(5.0), 40, 20, 20, 30),
    "caplet_5y_37x11x13": lambda: _item(2, W.caplet(5.0, 5.5), 37, 11, 13, 12),
    "caplet_12y_100x9x10_midpoint": lambda: _item(3, W.caplet(12.0, 12.5), 100, 9, 10, 10, explicit_midpoint=1),
    "caplet_0.4y_before_the_first_knots": lambda: _item(4, W.caplet(0.4, 0.9), 24, 8, 8, 6),
    "caplet_5y_past_the_last_knot_3y": lambda: _item(5, W.caplet(5.0, 6.0), 33, 9, 9, 8,
                                                     times=(0.25, 0.5, 1.0, 2.0, 3.0)),
    "caplet_5y_hv": lambda: _item(6, W.caplet(5.0, 5.5), 37, 11, 13, 12, scheme=3, theta_adi=0.5 + 3 ** 0.5 / 6),
    "bond_one_knot": lambda: _item(9, W.bond(5.0), 24, 8, 8, 10, times=(7.0,)),
}


def _ptype(torch, prec):
    return torch.float64 if prec == "fp64" else torch.float32


@pytest.mark.parametrize("name", list(CASES))
def test_axis_tables(H, orc, name):
    it = CASES[name]()
    with H.Grid(it) as g, orc.Ctx(it) as X:
        for axis in range(3):
            for a, b_ in zip(g.axis(axis), X.axis(axis)):
                assert np.max(np.abs(a - b_)) <= 1e-13 * (np.max(np.abs(b_)) + 1e-300), axis


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_march_field_and_price(H, orc, torch_mod, name, prec):
    torch = torch_mod
    it = CASES[name]()
    ns = it["grid"]["n_steps"]
    stages = 2 if it["grid"].get("scheme", 0) else 1
    with H.Grid(it) as g, orc.Ctx(it) as X:
        out = torch.empty(g.shape, dtype=_ptype(torch, prec), device="cuda")
        g.field(prec, 0, out)
        U0 = X.terminal()
        tol0 = 1e-13 if prec == "fp64" else 2.0 ** -23
        assert np.max(np.abs(out.double().cpu().numpy() - U0)) <= tol0 * np.max(np.abs(U0))
        want = X.march()
        pref = X.readout(want)
        g.field(prec, ns, out)
        got = out.double().cpu().numpy()
        scale = np.max(np.abs(want))
        p = g.price(prec)
        if prec == "fp64":
            assert np.max(np.abs(got - want)) <= 1e-10 * scale
            assert abs(p - pref) <= 1e-10 * max(abs(pref), scale * 1e-3)
        else:
            assert np.max(np.abs(got - want)) <= stages * 16.0 * (ns + 1) * 2.0 ** -24 * scale
            assert abs(p - pref) <= max(1e-4 * abs(pref), 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_mixing_curve_kinds(H, orc, prec):
    items = [_item(7, W.caplet(5.0, 5.5), 40, 10, 12, 8)]
    items += W.config2_draws(2, seed=17, n_r=40, n_y=10, n_v=12, n_steps=8)
    flat = W.config2_draws(1, seed=18, n_r=40, n_y=10, n_v=12, n_steps=8)[0]
    flat["curve"] = W.flat_curve(0.03)
    items.append(flat)
    items.append(_item(8, W.bond(3.0), 24, 8, 8, 10))
    want = np.array([orc.price(x) for x in items])
    got = H.hjm_price_batch(items, prec)
    if prec == "fp64":
        assert np.all(np.abs(got - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3))
    else:
        assert np.all(np.abs(got - want) <= np.maximum(1e-4 * np.abs(want), 1e-6))


def test_bond_reprices_the_discrete_curve(H, orc):
    # Section 6.1: the bond on the smoothed discrete curve reproduces P(0,T)
    # to O(1e-5) on a moderate mesh (FP32 march).
    it = _item(2, W.bond(5.0), 40, 20, 20, 100, explicit_midpoint=1)
    with H.Grid(it) as g:
        assert abs(g.price("fp32") - orc.curve_P(it["curve"], 5.0)) < 1e-5


def test_bad_knots_rejected(H):
    base = _item(1, W.bond(5.0), 24, 8, 8, 4)
    bad = []
    for mutate in (lambda c: c.update(n_knots=0), lambda c: c.update(n_knots=33),
                   lambda c: c["knot_t"].__setitem__(3, c["knot_t"][2]),
                   lambda c: c["knot_P"].__setitem__(1, 0.0), lambda c: c["knot_t"].__setitem__(0, -1.0)):
        it = {k: (dict(v) if isinstance(v, dict) else v) for k, v in base.items()}
        it["curve"] = {k: (list(v) if isinstance(v, list) else v) for k, v in base["curve"].items()}
        mutate(it["curve"])
        bad.append(it)
    for it in bad:
        with pytest.raises(H.HJMError) as ei:
            H.hjm_price_batch([it], "fp32")
        assert ei.value.status == H.HJM_EINVAL
