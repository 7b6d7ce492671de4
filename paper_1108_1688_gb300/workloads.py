"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws and lays out parameters (curves, model constants, grid
specifications, instruments). It contains none of the pricing arithmetic, so
both the GPU library and the CPU oracle can be fed from it.

Every item is a plain dict with four parts, mirroring the paper's statement of
the problem:
  curve : initial forward curve f(0,t) (Section 2). kind 0 = flat,
          kind 1 = Nelson-Siegel forward form
          f(0,t) = beta0 + beta1 e^{-t/tau} + beta2 (t/tau) e^{-t/tau}.
  model : kappa, lambda, gamma, theta, epsilon, rho, v0 (Section 3.1).
  grid  : node counts n_r x n_y x n_v, steps, physical domain, sinh metric
          (Section 4.3 / 7.1) and scheme options (Section 5).
  inst  : kind 0 = zero-coupon bond, kind 1 = caplet (Section 3.2). For a
          caplet, strike_atm_relative = 1 means K is an offset from the ATM
          forward rate, which each side computes from the curve itself.

Domain recipe (the paper's rescaled values in Section 7.1 disagree with its
figure captions, so the domain is set from the model's scales instead):
  r in [min(0, -fb - W_r), fb + W_r], W_r = 7 lambda sqrt(v_max T), fb a
      bound on |f(0,t)| (gamma = 0); r in [0, fb + W_r] when gamma > 0, with
      lambda replaced by lambda (2 fb)^gamma here and in y;
  v in [0, max(5, 1 + 10 epsilon / sqrt(2 theta))];
  y in [0, 4 lambda^2 v_max (1 - e^{-2 kappa T}) / (2 kappa)] (T lambda^2 v_max
      times 4 when kappa = 0);
  sinh metric: centre in r at the strike (bond: at f(0,0)), in v at 1, in y at
      0; width alpha = a fraction of each axis length.
"""
from __future__ import annotations

import copy
import math

import numpy as np

SEED_BASE = 1108000

CONFIG1_MODEL = dict(kappa=0.1, lambda_=0.01, gamma=0.0, theta=1.0, epsilon=0.3,
                     rho=-0.3, v0=1.0)

# Metric widths as fractions of the axis length.
ALPHA_FRAC_R = 0.25
ALPHA_FRAC_V = 0.25
ALPHA_FRAC_Y = 0.25


def flat_curve(rate):
    return dict(kind=0, flat_rate=float(rate), beta0=0.0, beta1=0.0, beta2=0.0, tau=1.0)


def ns_curve(beta0, beta1, beta2, tau):
    return dict(kind=1, flat_rate=0.0, beta0=float(beta0), beta1=float(beta1),
                beta2=float(beta2), tau=float(tau))


MAX_KNOTS = 32


def knot_curve(knot_t, knot_P):
    """Discrete initial curve (Section 6.1): discount factors knot_P at
    maturities knot_t (increasing, > 0, at most MAX_KNOTS)."""
    knot_t, knot_P = [float(v) for v in knot_t], [float(v) for v in knot_P]
    return dict(kind=2, flat_rate=0.0, beta0=0.0, beta1=0.0, beta2=0.0, tau=1.0,
                n_knots=len(knot_t), knot_t=knot_t, knot_P=knot_P)


# Maturities of a typical market discount curve: 3 and 6 months, 1 to 10
# years yearly, then 12, 15, 20, 25 and 30 years.
MARKET_KNOT_TIMES = (0.25, 0.5) + tuple(float(y) for y in range(1, 11)) + (12.0, 15.0, 20.0, 25.0, 30.0)


def synthetic_knot_curve(seed, times=MARKET_KNOT_TIMES, bump_bp=5.0):
    """A seeded discrete curve: continuously compounded zero rates at market
    maturities, z(t) = z0 + s (1 - e^{-t/5}) with z0 U[0.01, 0.035] and s
    U[-0.01, 0.025] (upward or inverted curves), each moved by up to bump_bp
    basis points of quote noise so the knots are not a smooth family;
    P = e^{-z t}."""
    rng = np.random.default_rng(seed)
    z0, sl = rng.uniform(0.01, 0.035), rng.uniform(-0.01, 0.025)
    Ps = [math.exp(-(z0 + sl * -math.expm1(-t / 5.0) + rng.uniform(-1.0, 1.0) * bump_bp * 1e-4) * t)
          for t in times]
    return knot_curve(times, Ps)


def model(kappa, lambda_, gamma, theta, epsilon, rho, v0=1.0):
    return dict(kappa=float(kappa), lambda_=float(lambda_), gamma=float(gamma),
                theta=float(theta), epsilon=float(epsilon), rho=float(rho), v0=float(v0))


def bond(T):
    return dict(kind=0, T=float(T), TM=float(T), K=0.0, strike_atm_relative=0)


def caplet(T, TM, K=0.0, atm_relative=True):
    return dict(kind=1, T=float(T), TM=float(TM), K=float(K),
                strike_atm_relative=1 if atm_relative else 0)


def floorlet(T, TM, K=0.0, atm_relative=True):
    """Floorlet on [T, TM]: pays max(Delta_M p(T,TM) - 1, 0) at T (the other
    side of the caplet; caplet - floorlet is the forward contract)."""
    return dict(kind=2, T=float(T), TM=float(TM), K=float(K),
                strike_atm_relative=1 if atm_relative else 0)


def strip(curve, mdl, T0, tenor, count, K, kind=1, n_r=64, n_y=32, n_v=32, steps_per_year=24, **grid_kw):
    """A cap (kind 1) or floor (kind 2) as its strip of caplets / floorlets on
    the periods [T0 + i tenor, T0 + (i + 1) tenor], i < count, each with
    absolute strike K on its own grid (the domain recipe of default_grid for
    its expiry, steps_per_year time steps a year). The strip's price is the
    sum of the items' prices."""
    out = []
    for i in range(count):
        T = T0 + i * tenor
        inst = (caplet if kind == 1 else floorlet)(T, T + tenor, K, atm_relative=False)
        ns = max(8, int(round(steps_per_year * T)))
        out.append(item(curve, mdl, default_grid(curve, mdl, T, n_r, n_y, n_v, ns, **grid_kw), inst))
    return out


def curve_level_bound(curve):
    """An upper bound on |f(0,t)| read off the parameters (x e^{-x} <= 1/e);
    for a discrete curve a rough scale: twice the largest zero rate or
    forward between knots (the spline's forward can overshoot them)."""
    if curve["kind"] == 0:
        return abs(curve["flat_rate"])
    if curve["kind"] == 2:
        ts = [0.0] + list(curve["knot_t"][:curve["n_knots"]])
        ls = [0.0] + [math.log(p) for p in curve["knot_P"][:curve["n_knots"]]]
        fwd = [abs((ls[i] - ls[i + 1]) / (ts[i + 1] - ts[i])) for i in range(len(ts) - 1)]
        return 2.0 * max(fwd)
    return abs(curve["beta0"]) + abs(curve["beta1"]) + abs(curve["beta2"]) / math.e


def default_grid(curve, mdl, T, n_r, n_y, n_v, n_steps, *, r_width_sd=7.0,
                 alpha_frac=(ALPHA_FRAC_R, ALPHA_FRAC_V, ALPHA_FRAC_Y),
                 theta_adi=0.5, y_boundary_order=2, explicit_midpoint=0, scheme=0, r_inf=None):
    """Grid specification following the domain recipe in the module docstring."""
    kap = mdl["kappa"]
    v_max = max(5.0, 1.0 + 10.0 * mdl["epsilon"] / math.sqrt(2.0 * max(mdl["theta"], 1e-12)))
    fb = curve_level_bound(curve)
    # Normal volatility scale: lambda r^gamma taken at r = 2 fb when gamma > 0.
    lam = mdl["lambda_"] * ((2.0 * fb) ** mdl["gamma"] if mdl["gamma"] > 0.0 else 1.0)
    w_r = r_width_sd * lam * math.sqrt(v_max * T)
    if mdl["gamma"] == 0.0:
        r_min, r_max = min(0.0, -fb - w_r), fb + w_r
    else:
        r_min, r_max = 0.0, (r_inf if r_inf is not None else fb + w_r)
    if kap > 0.0:
        y_max = 4.0 * lam * lam * v_max * (-math.expm1(-2.0 * kap * T)) / (2.0 * kap)
    else:
        y_max = 4.0 * lam * lam * v_max * T
    y_max = max(y_max, 1e-12)
    return dict(n_r=int(n_r), n_y=int(n_y), n_v=int(n_v), n_steps=int(n_steps),
                r_min=r_min, r_max=r_max, y_max=y_max, v_max=v_max,
                alpha_r=alpha_frac[0] * (r_max - r_min),
                alpha_v=alpha_frac[1] * v_max,
                alpha_y=alpha_frac[2] * y_max,
                k_r=0.0, k_v=1.0, center_r_on_strike=1,
                theta_adi=float(theta_adi), y_boundary_order=int(y_boundary_order),
                explicit_midpoint=int(explicit_midpoint), scheme=int(scheme))


def item(curve, mdl, grid, inst):
    return dict(curve=curve, model=mdl, grid=grid, inst=inst)


def config1():
    """5y zero-coupon bond, 40 x 20 x 20 (r x y x v), 100 steps, flat 3% forward,
    kappa 0.1, lambda 0.01, theta 1, epsilon 0.3, rho -0.3, gamma 0. The exact
    price is exp(-0.15)."""
    c = flat_curve(0.03)
    m = model(**CONFIG1_MODEL)
    g = default_grid(c, m, 5.0, 40, 20, 20, 100)
    return item(c, m, g, bond(5.0))


def _ns_draw(rng):
    return ns_curve(rng.uniform(0.02, 0.05), rng.uniform(-0.02, 0.02),
                    rng.uniform(-0.02, 0.02), rng.uniform(1.0, 5.0))


def config2_draws(n=100, seed=SEED_BASE + 2, n_r=128, n_y=64, n_v=64, n_steps=400):
    """Seeded 5y-into-6m ATM caplets on 128 x 64 x 64 with 400 steps: Nelson-Siegel
    curve (beta0 U[0.02,0.05], beta1, beta2 U[-0.02,0.02], tau U[1,5]),
    epsilon U[0.1,0.6], rho U[-0.7,0.3]; kappa, lambda, theta as in config1."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        c = _ns_draw(rng)
        eps = rng.uniform(0.1, 0.6)
        rho = rng.uniform(-0.7, 0.3)
        m = model(CONFIG1_MODEL["kappa"], CONFIG1_MODEL["lambda_"], 0.0,
                  CONFIG1_MODEL["theta"], eps, rho, 1.0)
        g = default_grid(c, m, 5.0, n_r, n_y, n_v, n_steps)
        out.append(item(c, m, g, caplet(5.0, 5.5, 0.0, True)))
    return out


def config3_batch(n=256, seed=SEED_BASE + 3, sizes=(64, 96, 128, 160, 192, 224, 256)):
    """256 caplets with expiry U{1..10}, T_M = T + 0.5, strike ATM + U[-0.02, 0.02],
    per-caplet curve and epsilon, rho as in config2, grids n_r in `sizes`,
    n_y = n_v = n_r / 2, steps = 2 n_r."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        c = _ns_draw(rng)
        eps = rng.uniform(0.1, 0.6)
        rho = rng.uniform(-0.7, 0.3)
        T = float(rng.integers(1, 11))
        dk = rng.uniform(-0.02, 0.02)
        nr = int(sizes[rng.integers(0, len(sizes))])
        m = model(CONFIG1_MODEL["kappa"], CONFIG1_MODEL["lambda_"], 0.0,
                  CONFIG1_MODEL["theta"], eps, rho, 1.0)
        g = default_grid(c, m, T, nr, nr // 2, nr // 2, 2 * nr)
        out.append(item(c, m, g, caplet(T, T + 0.5, dk, True)))
    return out


def config4(n_r=512, n_y=256, n_v=256, n_steps=1000):
    """10y-into-6m ATM caplet on 512 x 256 x 256 with 1000 steps, flat 3%, config1
    model parameters."""
    c = flat_curve(0.03)
    m = model(**CONFIG1_MODEL)
    g = default_grid(c, m, 10.0, n_r, n_y, n_v, n_steps)
    return item(c, m, g, caplet(10.0, 10.5, 0.0, True))


def paper_2007_set(n_r=40, n_y=20, n_v=20, n_steps=100, T=5.0):
    """The paper's 2007 market set (Section 3.3): p(0,T) = 1.04^{-T},
    kappa 0.001, lambda 0.15, gamma 0.9, epsilon 1.5, theta 0.25, rho -0.75."""
    c = flat_curve(math.log(1.04))
    m = model(0.001, 0.15, 0.9, 0.25, 1.5, -0.75, 1.0)
    # First-order y faces: with lambda = 0.15 the Courant number on the y = 0
    # face exceeds the bound under which second-order faces are stable.
    g = default_grid(c, m, T, n_r, n_y, n_v, n_steps, y_boundary_order=1)
    return item(c, m, g, bond(T))


def paper_timing_set():
    """The caplets of the paper's computation-time table (Section 6.3): expiry
    Tc = 1, 10, 19 years into a one-year period (TMc = Tc + 1), ATM, on a
    100 x 50 x 50 (r x y x v) mesh with 12 steps per year; the model is the
    2007 market set of Section 3.3 (the table does not name one)."""
    out = []
    for Tc in (1, 10, 19):
        x = paper_2007_set(n_r=100, n_y=50, n_v=50, n_steps=12 * Tc, T=float(Tc))
        x["inst"] = caplet(float(Tc), float(Tc + 1))
        x["grid"] = default_grid(x["curve"], x["model"], float(Tc), 100, 50, 50, 12 * Tc, y_boundary_order=1)
        out.append(x)
    return out


def with_grid(it, **kw):
    """Copy of an item with some grid fields replaced."""
    out = copy.deepcopy(it)
    out["grid"].update(kw)
    return out


def point_steps(it):
    g = it["grid"]
    return g["n_r"] * g["n_y"] * g["n_v"] * g["n_steps"]


# Surrogate input box (features kappa, lambda, theta, epsilon, rho, T, delta,
# K - F, F): epsilon and rho as in config2/3, kappa, lambda, theta 50-100%
# around config1, expiries 1..10y, accruals 3m..1y, strikes ATM +- 200bp.
SURROGATE_BOX_LO = (0.05, 0.005, 0.5, 0.1, -0.7, 1.0, 0.25, -0.02, 0.01)
SURROGATE_BOX_HI = (0.2, 0.015, 2.0, 0.6, 0.3, 10.0, 1.0, 0.02, 0.07)


def surrogate_label_grid(n_r=96, n_y=48, n_v=48, n_steps=192):
    """Counts and scheme of the surrogate's label march (the library sets the
    domain of each label from its draw)."""
    return dict(n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps, r_min=0.0, r_max=0.0, y_max=0.0, v_max=0.0,
                alpha_r=0.0, alpha_y=0.0, alpha_v=0.0, k_r=0.0, k_v=1.0, center_r_on_strike=1,
                theta_adi=0.5, y_boundary_order=2, explicit_midpoint=0, scheme=0)


def surrogate_draws(n, seed, box_lo=SURROGATE_BOX_LO, box_hi=SURROGATE_BOX_HI, out_of_box=0.0):
    """Raw surrogate inputs (kappa, lambda, theta, epsilon, rho, T, delta, K, F)
    uniform over the box; a fraction out_of_box has one feature pushed 20%
    of its range outside the box."""
    rng = np.random.default_rng(seed)
    lo, hi = np.array(box_lo), np.array(box_hi)
    f = lo + (hi - lo) * rng.random((n, 9))
    m = int(round(out_of_box * n))
    for r in range(m):
        k = int(rng.integers(0, 9))
        f[r, k] = hi[k] + 0.2 * (hi[k] - lo[k]) if k != 4 else hi[k] + 0.1
    x = f.copy()
    x[:, 7] = f[:, 7] + f[:, 8]
    return x.astype(np.float32)


def surrogate_item(x, label_grid):
    """The march's item for one raw surrogate input row (flat curve with the
    row's forward F over [T, T + delta]: continuous rate ln(1 + F delta)/delta)."""
    kap, lam, th, eps, rho, T, dl, K, F = [float(v) for v in x]
    c = math.log1p(F * dl) / dl
    curve = flat_curve(c)
    m = model(kap, lam, 0.0, th, eps, rho, 1.0)
    g = default_grid(curve, m, T, label_grid["n_r"], label_grid["n_y"], label_grid["n_v"], label_grid["n_steps"])
    return item(curve, m, g, caplet(T, T + dl, K, atm_relative=False))
