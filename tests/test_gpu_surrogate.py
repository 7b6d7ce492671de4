"""The pricing surrogate through the C ABI: its tensor-core GEMM against an
exact product, its loss gradient against the CPU FP64 reference network
(oracle/mlp_oracle.py, itself pinned by finite differences), training,
gating with the march as fallback, checkpointing, the PDE-judged error of a
trained network and what it gains over pricing with the march alone."""
import math
import os
import time

import numpy as np
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


def _cfg(H, n_train=256, epochs=2, batch=64, lr=1e-3, seed=7, label=None, ckpt=None):
    return H.surrogate_cfg(n_train, epochs, batch, lr, seed, W.SURROGATE_BOX_LO, W.SURROGATE_BOX_HI,
                           label or W.surrogate_label_grid(24, 10, 10, 24), ckpt)


def _bf16_tensor(torch, a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_tensor_core_gemm(env, ta, tb):
    torch, H = env
    rng = np.random.default_rng(ta * 2 + tb)
    M, N, K = 100, 70, 48
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    Ad, Bd = _bf16_tensor(torch, A), _bf16_tensor(torch, B)
    Ar = Ad.float().cpu().numpy().astype(np.float64)
    Br = Bd.float().cpu().numpy().astype(np.float64)
    want = (Ar.T if ta else Ar) @ (Br.T if tb else Br)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    H.hjm_mlp_gemm(M, N, K, Ad, A.shape[1], ta, Bd, B.shape[1], tb, C, N)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())


def _features(x):
    f = x.astype(np.float64).copy()
    f[:, 7] = f[:, 7] - f[:, 8]
    return f


def test_loss_gradient_matches_fp64_reference(env):
    # Element by element against the CPU FP64 reference with the kernels'
    # bfloat16 roundings replayed (bf16_round=True); the per-element tolerance
    # is one bfloat16 unit of each element's magnitude scale (tests/mlp_bounds.py:
    # the rounding decisions that FP32 arithmetic may take the other way).
    # The relative norm of each block is kept only as a summary.
    torch, H = env
    from oracle import mlp_oracle as M
    from tests import mlp_bounds as B
    h = H.hjm_surrogate_create(_cfg(H))
    try:
        p = H.hjm_surrogate_get_params(h).astype(np.float64)
        rng = np.random.default_rng(11)
        x = W.surrogate_draws(192, seed=5)
        t = rng.standard_normal(192).astype(np.float32)
        g = torch.empty(H.HJM_SURROGATE_PARAMS, dtype=torch.float32, device="cuda")
        loss = H.hjm_surrogate_loss_grad(h, torch.tensor(x).cuda(), torch.tensor(t).cuda(), g)
        torch.cuda.synchronize()
        lo, hi = np.array(W.SURROGATE_BOX_LO), np.array(W.SURROGATE_BOX_HI)
        f, t64 = _features(x), t.astype(np.float64)
        lref, gref = M.loss_and_grad(p, f, t64, lo, hi, bf16_round=True)
        assert abs(loss - lref) <= 1e-4 * abs(lref)
        gg = g.cpu().numpy().astype(np.float64)
        scale = B.grad_scale(p, f, t64, lo, hi)
        for name, shape, off in M.LAYOUT:
            n = int(np.prod(shape))
            sl = slice(off, off + n)
            excess, i = B.elementwise_excess(gg[sl], gref[sl], scale[sl])
            assert excess <= 1.0, (name, i, gg[off + i], gref[off + i], scale[off + i])
            rel = np.linalg.norm(gg[sl] - gref[sl]) / max(np.linalg.norm(gref[sl]), 1e-30)
            assert rel < 5e-3, (name, rel)  # summary
        # forward pass, row by row
        y = torch.empty(192, dtype=torch.float32, device="cuda")
        H.hjm_surrogate_forward(h, torch.tensor(x).cuda(), y)
        torch.cuda.synchronize()
        yref = M.forward(p, f, lo, hi, bf16_round=True)
        excess, i = B.elementwise_excess(y.cpu().numpy(), yref, B.forward_scale(p, f, lo, hi))
        assert excess <= 1.0, (i, excess)
    finally:
        H.hjm_surrogate_destroy(h)


def test_fit_reduces_loss(env):
    torch, H = env
    h = H.hjm_surrogate_create(_cfg(H, batch=256, lr=2e-3))
    try:
        x = W.surrogate_draws(4096, seed=6)
        f = _features(x)
        lo, hi = np.array(W.SURROGATE_BOX_LO), np.array(W.SURROGATE_BOX_HI)
        z = 2 * (f - lo) / (hi - lo) - 1
        t = (np.sin(2 * z[:, 5]) + 0.5 * z[:, 7] ** 2 - 0.3 * z[:, 3] * z[:, 4]).astype(np.float32)
        xd, td = torch.tensor(x).cuda(), torch.tensor(t).cuda()
        g = torch.empty(H.HJM_SURROGATE_PARAMS, dtype=torch.float32, device="cuda")
        l0 = H.hjm_surrogate_loss_grad(h, xd, td, g)
        H.hjm_surrogate_fit(h, xd, td, 20)
        l1 = H.hjm_surrogate_loss_grad(h, xd, td, g)
        assert l1 < 0.05 * l0, (l0, l1)
    finally:
        H.hjm_surrogate_destroy(h)


def _pde_forward_premium(H, x, label, prec="fp32"):
    items = [W.surrogate_item(r, label) for r in x]
    C = H.hjm_price_batch(items, prec)
    out = []
    for r, c in zip(x, C):
        T, dl, F = float(r[5]), float(r[6]), float(r[8])
        out.append(c * math.exp(math.log1p(F * dl) / dl * T))
    return np.array(out)


def test_forward_premium_depends_on_the_curve_only_through_the_forward(env):
    # The reduction behind the surrogate's ninth input: with gamma = 0 the
    # forward premium C / P(0,T) of a caplet depends on the initial curve only
    # through the simple forward F over [T, T_M] (the bond formula of Section
    # 3.2 gives p(T,T_M) through P(0,T_M)/P(0,T); the law of (x, y, v) does
    # not involve the curve). The FP64 march on a Nelson-Siegel curve and on
    # the flat curve with the same F must agree up to the discretisation
    # error, which shrinks under refinement (F at t^{n+1/2}, so the time error
    # of the curve-dependent drift is second order).
    torch, H = env
    from oracle import curve_P
    gaps = []
    for n in ((48, 24, 24, 96), (96, 48, 48, 192), (192, 96, 96, 384)):
        worst = 0.0
        for x in W.config2_draws(3, n_r=n[0], n_y=n[1], n_v=n[2], n_steps=n[3]):
            x["grid"]["explicit_midpoint"] = 1
            c, m, inst = x["curve"], x["model"], x["inst"]
            T, TM = inst["T"], inst["TM"]
            dl = TM - T
            P0 = curve_P(c, T)
            F = (P0 / curve_P(c, TM) - 1.0) / dl
            fc = W.flat_curve(math.log1p(F * dl) / dl)
            y = W.item(fc, m, W.default_grid(fc, m, T, *n, explicit_midpoint=1),
                       W.caplet(T, TM, F, atm_relative=False))
            C_ns, C_flat = H.hjm_price_batch([x, y], "fp64")
            worst = max(worst, abs(C_ns / P0 - C_flat / curve_P(fc, T)))
        gaps.append(worst)
    assert gaps[2] < gaps[0] and gaps[2] < 5e-6, gaps


def test_gaussian_part_matches_the_oracle_closed_form(env):
    # The closed-form base the network corrects: the Gaussian-HJM caplet
    # (epsilon = 0) as forward premium, on the device, against the oracle's
    # own closed form (itself pinned by quadrature and by the PDE's Gaussian
    # limit) on a flat curve with the row's forward.
    torch, H = env
    from oracle import curve_P, gauss_caplet
    x = W.surrogate_draws(256, seed=12)
    out = torch.empty(256, dtype=torch.float64, device="cuda")
    H.hjm_surrogate_gauss_premium(torch.tensor(x).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for r, g in zip(x, got):
        kap, lam, th, eps, rho, T, dl, K, F = [float(v) for v in r]
        c = W.flat_curve(math.log1p(F * dl) / dl)
        m = W.model(kap, lam, 0.0, th, 0.0, 0.0)
        want = gauss_caplet(c, m, T, T + dl, K) / curve_P(c, T)
        assert abs(g - want) <= 1e-12 * max(abs(want), 1e-6), (r, g, want)


def test_untrained_surrogate_falls_back_everywhere(env):
    torch, H = env
    label = W.surrogate_label_grid(24, 10, 10, 24)
    h = H.hjm_surrogate_create(_cfg(H, label=label))
    try:
        x = W.surrogate_draws(40, seed=8, out_of_box=0.25)
        out = torch.empty(40, dtype=torch.float64, device="cuda")
        used = torch.zeros(40, dtype=torch.uint8, device="cuda")
        H.hjm_surrogate_infer(h, torch.tensor(x).cuda(), out, used)
        torch.cuda.synchronize()
        assert bool(used.all())
        want = _pde_forward_premium(H, x, label)
        assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=1e-15)
    finally:
        H.hjm_surrogate_destroy(h)


def test_train_gate_checkpoint_and_resume(env, tmp_path):
    torch, H = env
    label = W.surrogate_label_grid(24, 10, 10, 24)
    path = str(tmp_path / "s.ckpt")
    h = H.hjm_surrogate_train(_cfg(H, n_train=1024, epochs=2, batch=128, label=label, ckpt=path))
    try:
        assert os.path.exists(path)
        table = H.hjm_surrogate_error_table(h)
        assert table.shape == (72,) and np.all(table >= 0)
        # out-of-box rows always fall back; in-box rows follow their bin
        x = W.surrogate_draws(64, seed=9, out_of_box=0.25)
        out = torch.empty(64, dtype=torch.float64, device="cuda")
        used = torch.zeros(64, dtype=torch.uint8, device="cuda")
        H.hjm_surrogate_infer(h, torch.tensor(x).cuda(), out, used)
        torch.cuda.synchronize()
        u = used.cpu().numpy().astype(bool)
        assert u[:16].all()
        want = _pde_forward_premium(H, x[u], label)
        assert np.allclose(out.cpu().numpy()[u], want, rtol=1e-12, atol=1e-15)
        # save / load round trip gives the same network
        p1 = H.hjm_surrogate_get_params(h)
        h2 = H.hjm_surrogate_load(path)
        try:
            assert np.array_equal(H.hjm_surrogate_get_params(h2), p1)
            assert np.array_equal(H.hjm_surrogate_error_table(h2), table)
        finally:
            H.hjm_surrogate_destroy(h2)
        # resuming with more epochs continues from the checkpoint
        h3 = H.hjm_surrogate_train(_cfg(H, n_train=1024, epochs=3, batch=128, label=label, ckpt=path))
        try:
            assert not np.array_equal(H.hjm_surrogate_get_params(h3), p1)
        finally:
            H.hjm_surrogate_destroy(h3)
    finally:
        H.hjm_surrogate_destroy(h)


TRAINED_LABEL = dict(n_r=64, n_y=32, n_v=32, n_steps=128)


@pytest.fixture(scope="module")
def trained(env):
    # A network trained on 2^16 PDE labels (64 x 32 x 32, 128 steps), shared
    # by the tests below.
    torch, H = env
    label = W.surrogate_label_grid(**TRAINED_LABEL)
    t0 = time.time()
    h = H.hjm_surrogate_train(H.surrogate_cfg(1 << 16, 120, 1024, 3e-3, 2024, W.SURROGATE_BOX_LO,
                                              W.SURROGATE_BOX_HI, label, None))
    yield h, label, time.time() - t0
    H.hjm_surrogate_destroy(h)


def test_trained_surrogate_error_coverage_and_gain(env, trained):
    # The trained network judged by the PDE on fresh draws (5% out of the
    # box): every answered row within 1e-4 of the PDE forward premium, the
    # rest priced by the PDE; then the speed-up of surrogate pricing over the
    # march alone on 65,536 rows.
    torch, H = env
    h, label, train_s = trained
    table = H.hjm_surrogate_error_table(h)
    print("surrogate: held-out bin errors min %.2e median %.2e max %.2e, bins under 5e-5: %d/72"
          % (table.min(), np.median(table), table.max(), int((table <= 5e-5).sum())))
    x = W.surrogate_draws(2048, seed=31, out_of_box=0.05)
    out = torch.empty(2048, dtype=torch.float64, device="cuda")
    used = torch.zeros(2048, dtype=torch.uint8, device="cuda")
    H.hjm_surrogate_infer(h, torch.tensor(x).cuda(), out, used)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    u = used.cpu().numpy().astype(bool)
    want = _pde_forward_premium(H, x, label)
    err = np.abs(got - want)
    coverage = 1.0 - u.mean()
    print("surrogate: train %.1fs coverage %.3f max err answered %.2e median %.2e"
          % (train_s, coverage, err[~u].max() if (~u).any() else 0, np.median(err[~u]) if (~u).any() else 0))
    assert np.all(err[u] <= 1e-12 + 1e-12 * np.abs(want[u]))  # fallback rows are the PDE
    assert np.all(err[~u] <= 1e-4)
    assert coverage > 0.9
    # gain: 65,536 rows through the network vs the march on a 256-row sample
    xb = torch.tensor(W.surrogate_draws(65536, seed=32)).cuda()
    yb = torch.empty(65536, dtype=torch.float32, device="cuda")
    H.hjm_surrogate_forward(h, xb, yb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        H.hjm_surrogate_forward(h, xb, yb)
    torch.cuda.synchronize()
    net_per_row = (time.perf_counter() - t0) / 5 / 65536
    xs = W.surrogate_draws(256, seed=33)
    items = [W.surrogate_item(r, label) for r in xs]
    H.hjm_price_batch(items, "fp32")
    t0 = time.perf_counter()
    H.hjm_price_batch(items, "fp32")
    pde_per_row = (time.perf_counter() - t0) / 256
    print("surrogate: %.3g s/row vs march %.3g s/row: %.0fx" % (net_per_row, pde_per_row, pde_per_row / net_per_row))
    assert pde_per_row / net_per_row > 100


def test_calibration_with_the_surrogate(env, trained):
    # The use the surrogate is built for (cap and floor calibration, Section
    # 1): fit (lambda, epsilon, rho) to a strip of caps made by the PDE (caps
    # of 6-month caplets from 1y to 2y, 3y, 4y and 5y at 5 strikes, flat
    # curve: 20 quotes, each the sum of its discounted caplets) with one
    # least-squares solver and start, four ways: the march in the loop; the
    # network in the loop (hjm_surrogate_premium: the Gaussian-HJM closed form
    # plus the learned stochastic-volatility correction); the gated network
    # (hjm_surrogate_infer, untrusted rows priced by the march); then the
    # march again, started from the network's answer (the final PDE
    # confirmation). The march arms and the target use the FP64 march: the
    # solver's finite differences in epsilon and rho move prices by ~1e-7,
    # below the FP32 march's rounding, which is not smooth in the parameters.
    scipy_opt = pytest.importorskip("scipy.optimize")
    torch, H = env
    h, label, _ = trained
    F, dl = 0.04, 0.5
    kap, th = 0.1, 1.0
    c = math.log1p(F * dl) / dl  # flat curve with simple forward F on every period
    true = np.array([0.011, 0.35, -0.3])
    expiries = [1.0 + dl * i for i in range(8)]
    strikes = [F + dk for dk in (-0.015, -0.0075, 0.0, 0.0075, 0.015)]
    rows = np.array([[kap, 0.0, th, 0.0, 0.0, T, dl, K, F] for T in expiries for K in strikes], dtype=np.float32)
    disc = np.array([math.exp(-c * T) for T in expiries for K in strikes])
    # cap (maturity m, strike k) = sum of the caplets with T + dl <= m
    A = np.array([[1.0 if (abs(r[7] - K) < 1e-9 and r[5] + dl <= mat + 1e-9) else 0.0 for r in rows]
                  for mat in (2.0, 3.0, 4.0, 5.0) for K in np.array(strikes, dtype=np.float32)])
    assert A.shape == (20, 40) and np.all(A.sum(axis=1) >= 2)

    def caps(premia):
        return A @ (disc * premia)

    def with_params(p):
        x = rows.copy()
        x[:, 1], x[:, 3], x[:, 4] = p[0], p[1], p[2]
        return x

    target = caps(_pde_forward_premium(H, with_params(true), label, "fp64"))
    n = len(rows)
    xd = torch.empty((n, 9), dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    used = torch.zeros(n, dtype=torch.uint8, device="cuda")
    fallback = []
    # unknowns q = (lambda / 0.01, epsilon, rho + 1): all of order one and
    # none near zero, because the solver's finite-difference step is relative
    # to the unknown (5 %: above the bf16 network's activation quantization;
    # an unknown starting at 0 would get a step of 1e-8, which the network
    # cannot resolve)
    S, O = np.array([0.01, 1.0, 1.0]), np.array([0.0, 0.0, 1.0])
    to_p = lambda q: q * S - O
    to_q = lambda p: (p + O) / S

    def resid_net(q):
        xd.copy_(torch.from_numpy(with_params(to_p(q))))
        H.hjm_surrogate_premium(h, xd, out)
        return (caps(out.cpu().numpy()) - target) / 1e-4

    def resid_gated(q):
        xd.copy_(torch.from_numpy(with_params(to_p(q))))
        H.hjm_surrogate_infer(h, xd, out, used)
        fallback.append(int(used.sum().item()))
        return (caps(out.cpu().numpy()) - target) / 1e-4

    def resid_pde(q):
        return (caps(_pde_forward_premium(H, with_params(to_p(q)), label, "fp64")) - target) / 1e-4

    kw = dict(bounds=(to_q(np.array([0.005, 0.1, -0.7])), to_q(np.array([0.015, 0.6, 0.3]))), diff_step=5e-2,
              xtol=1e-10, ftol=1e-10, max_nfev=100)
    start = to_q(np.array([0.008, 0.2, 0.0]))
    res = {}
    for name, fun in (("pde", resid_pde), ("net", resid_net), ("gated", resid_gated), ("confirm", resid_pde)):
        x0 = to_q(res["net"][0]) if name == "confirm" else start
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = scipy_opt.least_squares(fun, x0, **kw)
        res[name] = (to_p(r.x), time.perf_counter() - t0, r.nfev)
    for name, (x, secs, nfev) in res.items():
        print("calibration %s: lambda %.5f eps %.4f rho %.4f (true %s) in %.3f s, %d evaluations"
              % (name, x[0], x[1], x[2], true, secs, nfev))
    print("calibration gated: %d of %d rows priced by the march over %d evaluations"
          % (sum(fallback), n * len(fallback), len(fallback)))
    # every arm recovers the parameters the caps were made with: the march
    # from the plain start and from the network's answer, and the network
    # (which carries epsilon and rho through its learned correction), far
    # faster than the march
    for name in ("pde", "confirm", "net", "gated"):
        x = res[name][0]
        assert abs(x[0] / true[0] - 1) < 1e-3 and abs(x[1] - true[1]) < 0.02 and abs(x[2] - true[2]) < 0.05, name
    assert res["pde"][1] > 5 * res["net"][1]
