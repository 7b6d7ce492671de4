"""GPU path vs the CPU FP64 oracle, element by element, through the C ABI.

Tolerances (from the arithmetic, fixed here):
  FP64 march   fields and prices within 1e-10 relative to the field scale
               (the oracle and the kernels differ only in rounding order)
  FP32 march   prices within max(1e-4 |p|, 1e-6); fields within
               FIELD32 = 16 * (n_steps + 1) * 2^-24 of the field scale (one
               rounding per operation of a contractive step, accumulated over
               the steps), checked together with the price criterion
  one pass     FP64: 1e-12, FP32: 2e-6 of the larger of the input and output
               scales (a single pass has no accumulation; pass 1 forms dt F(U)
               as differences of U, so its rounding scales with |U|)
The cases span every chunk width of the r kernel (2, 4, 8, 16 nodes per
lane), ragged r lengths (not multiples of 32 or of the vector width), both
Dirichlet and degenerate r = 0 faces (gamma = 0 and gamma = 0.9), first- and
second-order y faces, flat and Nelson-Siegel curves, bonds and caplets.
"""
import math

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


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _caplet_case(n_r, n_y, n_v, n_steps, seed=0, **grid_kw):
    it = W.config2_draws(1, seed=W.SEED_BASE + 100 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    it["grid"].update(grid_kw)
    return it


def _bond_gamma(n_r, n_y, n_v, n_steps):
    return W.paper_2007_set(n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)


CASES = {
    "config1_bond_M2": lambda: W.config1(),
    "caplet_ragged_37x11x13": lambda: _caplet_case(37, 11, 13, 12),
    "caplet_M4_midpoint_NS": lambda: _caplet_case(100, 9, 10, 10, seed=1, explicit_midpoint=1),
    "caplet_M8_partial_yorder1": lambda: _caplet_case(200, 8, 7, 6, seed=2, y_boundary_order=1),
    "caplet_M16_partial": lambda: _caplet_case(400, 6, 7, 4, seed=3),
    "caplet_nr512": lambda: _caplet_case(512, 5, 6, 3, seed=4),
    "bond_gamma09_nr13": lambda: _bond_gamma(13, 7, 9, 20),
    "bond_gamma09_nr64": lambda: _bond_gamma(64, 10, 12, 15),
    "caplet_uniform_5x5x5": lambda: _caplet_case(5, 5, 5, 7, seed=5, alpha_r=0.0, alpha_v=0.0, alpha_y=0.0),
    "caplet_kappa0_rho_minus1": lambda: _degenerate(dict(kappa=0.0, rho=-1.0), W.caplet(3.0, 3.5)),
    "bond_eps0_theta0": lambda: _degenerate(dict(epsilon=0.0, theta=0.0), W.bond(4.0)),
}


def _degenerate(model_kw, inst):
    # the model's limiting cases: kappa = 0 (G(s) = s), perfect correlation,
    # a variance that neither diffuses nor reverts (A_v = 0)
    c = W.ns_curve(0.03, -0.01, 0.015, 2.0)
    m = W.model(**dict(W.CONFIG1_MODEL, **model_kw))
    return W.item(c, m, W.default_grid(c, m, inst["T"], 29, 9, 11, 10), inst)
PRECS = ["fp64", "fp32"]


def _ptype(torch, prec):
    return torch.float64 if prec == "fp64" else torch.float32


def field32_tol(n_steps):
    return 16.0 * (n_steps + 1) * 2.0 ** -24


@pytest.mark.parametrize("name", list(CASES))
def test_axis_tables(H, orc, name):
    it = CASES[name]()
    with H.Grid(it) as g, orc.Ctx(it) as X:
        for axis in range(3):
            z, J, J2 = g.axis(axis)
            zo, Jo, J2o = X.axis(axis)
            for a, b_ in ((z, zo), (J, Jo), (J2, J2o)):
                scale = np.max(np.abs(b_)) + 1e-300
                assert np.max(np.abs(a - b_)) <= 1e-13 * scale, axis


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_terminal_field(H, orc, torch_mod, name, prec):
    torch = torch_mod
    it = CASES[name]()
    with H.Grid(it) as g, orc.Ctx(it) as X:
        out = torch.empty(g.shape, dtype=_ptype(torch, prec), device="cuda")
        g.field(prec, 0, out)
        got = out.double().cpu().numpy()
        want = X.terminal()
        tol = 1e-13 if prec == "fp64" else 2.0 ** -23
        assert np.max(np.abs(got - want)) <= tol * max(np.max(np.abs(want)), 1e-300)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_douglas_passes(H, orc, torch_mod, name, prec):
    # Each kernel pass against the oracle's corresponding stage, from the same
    # (oracle-made) input state.
    torch = torch_mod
    it = CASES[name]()
    ns = it["grid"]["n_steps"]
    n = min(2, ns - 1)
    with H.Grid(it) as g, orc.Ctx(it) as X:
        U = X.terminal()
        for s in range(n):
            U = X.step(s, U)
        th = X.time(n + 0.5)
        dU0 = X.explicit(n, U)
        dU1 = X.solve_dir(0, th, dU0)
        dU2 = X.solve_dir(1, th, dU1)
        U1 = U + X.solve_dir(2, th, dU2)
        dt = _ptype(torch, prec)
        tol = 1e-12 if prec == "fp64" else 2e-6
        dev = lambda a: torch.tensor(a, dtype=dt, device="cuda")
        out = torch.empty(g.shape, dtype=dt, device="cuda")
        # pass 1 uses U in the march type: compare against the oracle fed the
        # same rounded input, so the check isolates the pass itself.
        Ur = dev(U).double().cpu().numpy()
        want1 = X.solve_dir(0, th, X.explicit(n, Ur))
        g.douglas_pass(prec, 1, n, dev(U), None, out)
        got = out.double().cpu().numpy()
        assert np.max(np.abs(got - want1)) <= tol * max(np.max(np.abs(want1)), np.max(np.abs(U))), "pass 1"
        inp = dev(dU1)
        want2 = X.solve_dir(1, th, inp.double().cpu().numpy())
        g.douglas_pass(prec, 2, n, inp, None, inp)  # in place, as in the march
        got = inp.double().cpu().numpy()
        assert np.max(np.abs(got - want2)) <= tol * max(np.max(np.abs(want2)), np.max(np.abs(dU1))), "pass 2"
        inp = dev(dU2)
        Ud = dev(U)
        want3 = Ud.double().cpu().numpy() + X.solve_dir(2, th, inp.double().cpu().numpy())
        g.douglas_pass(prec, 3, n, inp, Ud, Ud)  # U updated in place
        got = Ud.double().cpu().numpy()
        assert np.max(np.abs(got - want3)) <= tol * max(np.max(np.abs(want3)), np.max(np.abs(dU2))), "pass 3"
        del U1


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_march_field_and_price(H, orc, torch_mod, name, prec):
    torch = torch_mod
    it = CASES[name]()
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
            assert np.max(np.abs(got - want)) <= field32_tol(ns) * scale
            assert abs(p - pref) <= max(1e-4 * abs(pref), 1e-6)


def test_config1_price_matches_curve(H):
    # 5y bond, 40 x 20 x 20, 100 steps: price = exp(-0.15) within the paper's
    # 1e-5 (the oracle's own discretisation error is ~1e-6).
    with H.Grid(W.config1()) as g:
        for prec in PRECS:
            assert abs(g.price(prec) - math.exp(-0.15)) < 1e-5


def _mixed_batch():
    items = []
    items += W.config2_draws(5, seed=11, n_r=48, n_y=12, n_v=10, n_steps=20)
    items += W.config2_draws(4, seed=12, n_r=33, n_y=9, n_v=11, n_steps=15)
    b = W.config1()
    b["grid"].update(n_steps=30)
    items.insert(3, b)
    items += [_bond_gamma(24, 8, 8, 12)]
    items += W.config3_batch(4, sizes=(64,))
    for x in items[-4:]:
        x["grid"].update(n_steps=16)
    return items


@pytest.mark.parametrize("prec", PRECS)
def test_batch_of_mixed_shapes(H, orc, torch_mod, prec):
    torch = torch_mod
    items = _mixed_batch()
    want = np.array([orc.price(x) for x in items])
    host = H.hjm_price_batch(items, prec)
    dev = torch.full((len(items),), float("nan"), dtype=torch.float64, device="cuda")
    H.hjm_price_batch(items, prec, out=dev, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)  # same kernels, same order
    if prec == "fp64":
        assert np.all(np.abs(host - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3))
    else:
        assert np.all(np.abs(host - want) <= np.maximum(1e-4 * np.abs(want), 1e-6))
    # batch result equals the single-instrument path
    with H.Grid(items[3]) as g:
        assert g.price(prec) == host[3]


def test_batch_repeat_is_bitwise_stable(H):
    # First call: launches straight to the stream; second: the batch graph
    # is captured and launched; third: replayed. Same kernels per group, so
    # the same bits (the groups' concurrency in the graph changes nothing).
    items = _mixed_batch()
    a = H.hjm_price_batch(items, "fp32")
    b = H.hjm_price_batch(items, "fp32")
    c = H.hjm_price_batch(items, "fp32")
    assert np.array_equal(a, b) and np.array_equal(b, c)


def _oracle_prices_parallel(orc, items, workers=4):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, len(items))) as pool:
        return np.array(pool.map(orc.price, items))


def test_full_size_config2_bench_batch(H, orc, torch_mod):
    # The bench workload: 100 seeded caplets on 128 x 64 x 64 with 400 steps,
    # FP32, one batch call. Sampled against the oracle (4 draws, full size)
    # and, for all 100, against the FP64 GPU path (itself checked above).
    torch = torch_mod
    items = W.config2_draws(100)
    sample = [0, 37, 64, 99]
    want = _oracle_prices_parallel(orc, [items[i] for i in sample])
    p32 = torch.empty(100, dtype=torch.float64, device="cuda")
    H.hjm_price_batch(items, "fp32", out=p32, stream=torch.cuda.current_stream())
    p64 = H.hjm_price_batch(items, "fp64")
    torch.cuda.synchronize()
    p32 = p32.cpu().numpy()
    assert np.all(np.abs(p32[sample] - want) <= np.maximum(1e-4 * np.abs(want), 1e-6)), (p32[sample], want)
    assert np.all(np.abs(p64[sample] - want) <= 1e-10 * np.abs(want)), (p64[sample], want)
    assert np.all(np.abs(p32 - p64) <= np.maximum(1e-4 * np.abs(p64), 1e-6))
    assert np.all(p64 > 0.0)


def test_full_size_config4_first_step_and_march(H, orc, torch_mod):
    # The 512 x 256 x 256 caplet of the benchmark, in the launch shape the
    # autotuner picks for it (32,16,8,8,8): the whole field after the first
    # step against the oracle element by element (FP32 and FP64), then the
    # full 1000-step FP32 price against the FP64 GPU march (the oracle cannot
    # run 3.4e10 point-steps; the FP64 path is pinned to it above).
    torch = torch_mod
    it = W.config4()
    g = it["grid"]
    H.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], "fp32", (32, 16, 8, 8, 8, 0, 0))
    try:
        with orc.Ctx(it) as X:
            want = X.step(0, X.terminal())
        scale = np.max(np.abs(want))
        with H.Grid(it) as gr:
            for prec, tol in (("fp32", field32_tol(1)), ("fp64", 1e-10)):
                out = torch.empty(gr.shape, dtype=_ptype(torch, prec), device="cuda")
                gr.field(prec, 1, out)
                got = out.double().cpu().numpy()
                assert np.max(np.abs(got - want)) <= tol * scale, prec
                del out
            p32, p64 = gr.price("fp32"), gr.price("fp64")
        assert abs(p32 - p64) <= max(1e-4 * abs(p64), 1e-6), (p32, p64)
    finally:
        H.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], "fp32", None)


def test_full_size_config3_batch(H, orc):
    # The 256 uneven caplets of the benchmark in one call after the
    # benchmark's autotuning: FP32 against the FP64 GPU march for all, and
    # both against the oracle on the caplets of the smallest grid (64 x 32 x
    # 32, 128 steps).
    items = W.config3_batch()
    H.hjm_autotune(items, "fp32", steps=4)
    p32 = H.hjm_price_batch(items, "fp32")
    p64 = H.hjm_price_batch(items, "fp64")
    assert np.all(np.abs(p32 - p64) <= np.maximum(1e-4 * np.abs(p64), 1e-6))
    small = [i for i, x in enumerate(items) if x["grid"]["n_r"] == 64][:3]
    want = _oracle_prices_parallel(orc, [items[i] for i in small], workers=3)
    assert np.all(np.abs(p64[small] - want) <= 1e-10 * np.abs(want)), (p64[small], want)
    assert np.all(np.abs(p32[small] - want) <= np.maximum(1e-4 * np.abs(want), 1e-6))
    for x in items:
        H.hjm_tile_set(x["grid"]["n_r"], x["grid"]["n_v"], x["grid"]["n_y"], "fp32", None)


@pytest.mark.parametrize("prec,lim", [("fp32", 908), ("fp64", 454)])
def test_strided_line_length_limits(H, orc, prec, lim):
    # The longest v and y lines the one-lane-per-line kernels hold in shared
    # memory (two columns of 32 lines for pass 3), priced against the
    # oracle; one node more is refused.
    tol = (lambda p, w: abs(p - w) <= 1e-10 * max(abs(w), 1e-3)) if prec == "fp64" else \
          (lambda p, w: abs(p - w) <= max(1e-4 * abs(w), 1e-6))
    for nv, ny in ((lim, 6), (6, lim)):
        it = _caplet_case(6, ny, nv, 3, seed=7)
        assert tol(H.hjm_price_batch([it], prec)[0], orc.price(it)), (nv, ny)
    for nv, ny in ((lim + 1, 6), (6, lim + 1)):
        with pytest.raises(H.HJMError) as ei:
            H.hjm_price_batch([_caplet_case(6, ny, nv, 3, seed=7)], prec)
        assert ei.value.status == H.HJM_ERANGE


def test_size_limits(H):
    it = _caplet_case(512, 5, 5, 2)
    with H.Grid(it) as g:
        assert g.price("fp32") > 0.0
    bad = _caplet_case(513, 5, 5, 2)
    with pytest.raises(H.HJMError) as ei:
        H.hjm_grid_create(bad["curve"], bad["model"], bad["grid"])
    assert ei.value.status == H.HJM_ERANGE


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["config1_bond_M2", "caplet_ragged_37x11x13", "caplet_M4_midpoint_NS",
                                  "bond_gamma09_nr13"])
def test_greeks_match_oracle(H, orc, name, prec):
    # dC/dr and dC/dv at the read-out point (derivatives of the FP64 read-out
    # interpolant of the final field) against the oracle's on its own march.
    it = CASES[name]()
    with orc.Ctx(it) as X:
        U = X.march()
        want_r, want_v = X.readout_greeks(U)
        _, Jr, _ = X.axis(0)
        _, Jv, _ = X.axis(1)
    p, infos = H.hjm_price_batch([it], prec, infos=True)
    got_r, got_v = infos[0].d_dr, infos[0].d_dv
    g = it["grid"]
    # scale of a derivative of the interpolant: field size x nodes per unit
    sr = np.max(np.abs(U)) * (g["n_r"] - 1) / np.min(Jr)
    sv = np.max(np.abs(U)) * (g["n_v"] - 1) / np.min(Jv)
    rel = 1e-9 if prec == "fp64" else 2e-4
    assert abs(got_r - want_r) <= rel * sr, (got_r, want_r, sr)
    assert abs(got_v - want_v) <= rel * sv, (got_v, want_v, sv)


def test_concurrent_callers_on_their_own_streams(H, torch_mod):
    # Two host threads price different batches on their own CUDA streams at
    # the same time (the library serialises its host state, each stream has
    # its own workspace); every result equals the single-threaded one.
    import threading
    torch = torch_mod
    batches = [W.config2_draws(6, seed=41, n_r=48, n_y=12, n_v=10, n_steps=20),
               W.config2_draws(5, seed=42, n_r=33, n_y=9, n_v=11, n_steps=15) + [W.config1()]]
    want = [H.hjm_price_batch(b, "fp32") for b in batches]
    got = [[None] * 3 for _ in batches]
    errors = []

    def worker(q):
        try:
            s = torch.cuda.Stream()
            out = torch.empty(len(batches[q]), dtype=torch.float64, device="cuda")
            for r in range(3):
                with torch.cuda.stream(s):
                    H.hjm_price_batch(batches[q], "fp32", out=out, stream=s)
                s.synchronize()
                got[q][r] = out.cpu().numpy().copy()
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(q,)) for q in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for q in range(2):
        for r in range(3):
            assert np.array_equal(got[q][r], want[q]), (q, r)
