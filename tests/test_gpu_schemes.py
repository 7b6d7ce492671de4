"""The Craig-Sneyd family on the GPU (CS, modified CS, Hundsdorfer-Verwer;
Section 5.1 and the In 't Hout-Welfert schemes it cites) against the CPU
FP64 oracle, through the C ABI: the correction stage's pass 1 alone, whole
marches (field and price) over pass-1 chunk widths, both r-face kinds and
every strided-pass launch shape (split, fused, staged pass 1), batches that
mix schemes, and the allocation-free entry point. Tolerances as in
test_gpu_parity.py: one pass within 1e-12 (FP64) / 2e-6 (FP32) of the larger
of the input and output scales; a march within 1e-10 (FP64) and within
max(1e-4 |p|, 1e-6) for FP32 prices."""
import math

import numpy as np
import pytest

from paper_1108_1688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCHEMES = {1: 0.5, 2: 1.0 / 3.0, 3: 0.5 + math.sqrt(3.0) / 6.0}  # scheme -> theta
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


def _caplet(n_r, n_y, n_v, n_steps, scheme, seed=0, **kw):
    # strong correlation and vol-of-vol so the mixed term matters
    it = W.config2_draws(1, seed=W.SEED_BASE + 500 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    it["model"].update(rho=-0.8, epsilon=0.8)
    it["grid"] = W.default_grid(it["curve"], it["model"], it["inst"]["T"], n_r, n_y, n_v, n_steps)
    it["grid"].update(scheme=scheme, theta_adi=SCHEMES[scheme], **kw)
    return it


def _bond_gamma(scheme):
    it = W.paper_2007_set(n_r=13, n_y=7, n_v=9, n_steps=12)
    it["grid"].update(scheme=scheme, theta_adi=SCHEMES[scheme])
    return it


CASES = {
    "caplet_37x11x13": lambda s: _caplet(37, 11, 13, 10, s),
    "caplet_100x9x10_F_at_tn": lambda s: _caplet(100, 9, 10, 8, s, seed=1, explicit_midpoint=0),
    "caplet_400x6x7": lambda s: _caplet(400, 6, 7, 4, s, seed=2),
    "bond_gamma09_13x7x9": _bond_gamma,
    "caplet_uniform_5x5x5": lambda s: _caplet(5, 5, 5, 6, s, seed=3, alpha_r=0.0, alpha_v=0.0, alpha_y=0.0),
}


def _ptype(torch, prec):
    return torch.float64 if prec == "fp64" else torch.float32


def _correction_stage(X, n, U, Y, scheme, theta):
    """Z1 - B of the correction stage from U^n and Y3 (the scheme's definition
    with the oracle's operators, every explicit one at t^{n+1/2})."""
    t, dt = X.time(n + 0.5), X.dt
    z = X.explicit(n, U)  # Y0 - U^n
    if scheme in (1, 2):
        c = 0.5 if scheme == 1 else theta
        z = z + c * dt * (X.apply_dir(3, t, Y) - X.apply_dir(3, t, U))
    if scheme in (2, 3):
        c = 0.5 - theta if scheme == 2 else 0.5
        z = z + c * dt * (X.apply_F(t, Y) - X.apply_F(t, U))
    if scheme == 3:
        z = z - (Y - U)
    return X.solve_dir(0, t, z)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("name", list(CASES))
def test_correction_pass(H, orc, torch_mod, name, scheme, prec):
    torch = torch_mod
    it = CASES[name](scheme)
    n = min(2, it["grid"]["n_steps"] - 1)
    with H.Grid(it) as g, orc.Ctx(it) as X:
        U = X.terminal()
        for s in range(n):
            U = X.step(s, U)
        th = X.time(n + 0.5)
        E = X.solve_dir(2, th, X.solve_dir(1, th, X.solve_dir(0, th, X.explicit(n, U))))
        dt = _ptype(torch, prec)
        dev = lambda a: torch.tensor(a, dtype=dt, device="cuda")
        Ud, Yd = dev(U), dev(U + E)
        Ur, Yr = Ud.double().cpu().numpy(), Yd.double().cpu().numpy()
        want = _correction_stage(X, n, Ur, Yr, scheme, SCHEMES[scheme])
        out = torch.empty(g.shape, dtype=dt, device="cuda")
        g.douglas_pass(prec, 4, n, Ud, Yd, out)
        got = out.double().cpu().numpy()
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.max(np.abs(got - want)) <= tol * max(np.max(np.abs(want)), np.max(np.abs(U)))
        # the first stage's pass 3 writes Y3 = U^n + dU3 to a separate buffer
        dU2 = X.solve_dir(1, th, X.solve_dir(0, th, X.explicit(n, U)))
        inp = dev(dU2)
        Y3 = torch.empty(g.shape, dtype=dt, device="cuda")
        g.douglas_pass(prec, 3, n, inp, Ud, Y3)
        want3 = Ur + X.solve_dir(2, th, inp.double().cpu().numpy())
        got3 = Y3.double().cpu().numpy()
        assert np.max(np.abs(got3 - want3)) <= tol * max(np.max(np.abs(want3)), np.max(np.abs(dU2)))
        assert np.array_equal(Ud.double().cpu().numpy(), Ur)  # U^n untouched


def _check_march(H, orc, torch, it, prec):
    ns = it["grid"]["n_steps"]
    with H.Grid(it) as g, orc.Ctx(it) as X:
        want = X.march()
        pref = X.readout(want)
        out = torch.empty(g.shape, dtype=_ptype(torch, prec), device="cuda")
        g.field(prec, ns, out)
        got = out.double().cpu().numpy()
        scale = np.max(np.abs(want))
        p = g.price(prec)
        if prec == "fp64":
            assert np.max(np.abs(got - want)) <= 1e-10 * scale
            assert abs(p - pref) <= 1e-10 * max(abs(pref), scale * 1e-3)
        else:
            assert np.max(np.abs(got - want)) <= 2 * 16.0 * (ns + 1) * 2.0 ** -24 * scale
            assert abs(p - pref) <= max(1e-4 * abs(pref), 1e-6)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("name", list(CASES))
def test_march_field_and_price(H, orc, torch_mod, name, scheme, prec):
    _check_march(H, orc, torch_mod, CASES[name](scheme), prec)


def _tiles(nr, prec):
    # a split of each strided pass, the fused strided passes and the staged
    # pass 1 (which the correction stage replaces by the direct kernel)
    base = (16, 4)
    return [base + (1, 2, 4), base + (2, 4, 2), base + (1, 0, 1), base + (1, 1, 1, 1, 2)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_launch_shapes(H, orc, torch_mod, scheme, prec):
    it = _caplet(64, 16, 12, 6, scheme, seed=4)
    g = it["grid"]
    try:
        for t in _tiles(g["n_r"], prec):
            H.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], prec, t)
            assert H.hjm_tile_get(g["n_r"], g["n_v"], g["n_y"], prec)[:len(t)] == tuple(t)
            _check_march(H, orc, torch_mod, it, prec)
    finally:
        H.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], prec, None)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_mixing_schemes(H, orc, torch_mod, prec):
    # the same grid shape under all four schemes in one call (one group per
    # scheme), plus another shape; caller order kept
    items = []
    for q, s in enumerate((0, 1, 2, 3, 3, 1)):
        x = _caplet(40, 10, 12, 8, s if s else 1, seed=10 + (q >= 4) * q)  # items 0-3: one instrument
        x["grid"].update(scheme=s, theta_adi=SCHEMES.get(s, 0.5))
        items.append(x)
    items.append(_caplet(24, 8, 8, 6, 2, seed=20))
    want = np.array([orc.price(x) for x in items])
    got = H.hjm_price_batch(items, prec)
    if prec == "fp64":
        assert np.all(np.abs(got - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3))
    else:
        assert np.all(np.abs(got - want) <= np.maximum(1e-4 * np.abs(want), 1e-6))
    assert len(set(np.round(got[:4], 12))) == 4  # one instrument, four schemes: they differ


def test_static_entry_point(H, orc, torch_mod):
    torch = torch_mod
    for s in SCHEMES:
        it = _caplet(37, 11, 13, 10, s)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        H.hjm_price_static(it, "fp64", out)
        torch.cuda.synchronize()
        want = orc.price(it)
        assert abs(out.item() - want) <= 1e-10 * max(abs(want), 1e-3)


def test_second_order_in_time_on_the_gpu(H):
    # The property the schemes exist for, on the GPU path (FP64): errors
    # against 256 steps at 8, 16, 32 steps fall by about 4 per halving for
    # HV, about 2 for Douglas (strong mixed term, flat curve).
    c = W.flat_curve(0.03)
    m = W.model(0.1, 0.02, 0.0, 1.0, 1.0, -0.9)
    ratios = {}
    for s, th in ((0, 0.5), (3, SCHEMES[3])):
        mk = lambda ns: W.item(c, m, W.default_grid(c, m, 2.0, 24, 16, 16, ns, theta_adi=th, scheme=s,
                                                    explicit_midpoint=1), W.caplet(2.0, 2.5))
        p = H.hjm_price_batch([mk(ns) for ns in (8, 16, 32, 512)], "fp64")
        e = np.abs(p[:3] - p[3])
        ratios[s] = e[:2] / e[1:]
    assert np.all(ratios[0] < 2.8) and np.all(ratios[3] > 3.0), ratios


def test_unknown_scheme_rejected(H):
    it = _caplet(37, 11, 13, 10, 1)
    it["grid"]["scheme"] = 4
    with pytest.raises(H.HJMError) as ei:
        H.hjm_price_batch([it], "fp32")
    assert ei.value.status == H.HJM_EINVAL


def test_mixed_precision_with_the_schemes(H, orc):
    # MIXED on Craig-Sneyd-family items: FP32 marches, the rounding bound of
    # each (both stages feed the indicator), FP64 re-runs where it misses:
    # every price within the tolerance of the oracle and every reported
    # bound within it; an escalated item carries the FP64 price.
    items = [_caplet(37, 11, 13, 10, s, seed=30 + s) for s in SCHEMES]
    want = np.array([orc.price(x) for x in items])
    p, infos = H.hjm_price_batch(items, "mixed", tol_rel=1e-4, infos=True)
    assert np.all(np.abs(p - want) <= np.maximum(1e-4 * np.abs(want), 1e-6))
    for i, inf in enumerate(infos):
        assert inf.err_estimate <= max(1e-4 * abs(p[i]), 1e-6)
        if inf.escalated:
            assert abs(p[i] - want[i]) <= 1e-10 * max(abs(want[i]), 1e-3)
