"""Every launch shape of the march kernels against the CPU FP64 oracle: the
pass-1 shapes (lanes per r line, nodes per lane, lines per segment) and the
split line solves of passes 2 and 3 (warps per v / y line), one Douglas pass
at a time and over a whole march, plus the shape-selection calls
(hjm_tile_get / hjm_tile_set / hjm_autotune). Tolerances as in
test_gpu_parity.py: a single pass within 1e-12 (FP64) / 2e-6 (FP32) of the
larger of the input and output scales, a march within 1e-10 (FP64)."""
import itertools

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


def _caplet(n_r, n_y, n_v, n_steps, seed=0, **kw):
    it = W.config2_draws(1, seed=W.SEED_BASE + 300 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    it["grid"].update(kw)
    return it


CASES = {
    "config1_bond": lambda: W.config1(),
    "caplet_37x11x13": lambda: _caplet(37, 11, 13, 8),
    "caplet_64x40x70_NS": lambda: _caplet(64, 40, 70, 6, seed=1),
    "caplet_130x17x33_yorder1": lambda: _caplet(130, 17, 33, 5, seed=2, y_boundary_order=1),
    "bond_gamma09_13x7x9": lambda: W.paper_2007_set(n_r=13, n_y=7, n_v=9, n_steps=12),
}

P1_SHAPES = {"fp32": [(8, 8), (8, 16), (16, 4), (16, 8), (16, 16), (32, 2), (32, 4), (32, 8), (32, 16)],
             "fp64": [(16, 2), (16, 4), (16, 8), (32, 2), (32, 4), (32, 8), (32, 16)]}


def split_ok(n, P):
    return P == 1 or (n >= 2 * P and -(-n // P) <= 32)


def tiles_for(it, prec):
    g = it["grid"]
    nr, nv, ny = g["n_r"], g["n_v"], g["n_y"]
    out = []
    cover = min(S * M for S, M in P1_SHAPES[prec] if S * M >= nr)
    for (S, M), R in itertools.product(P1_SHAPES[prec], (1, 3)):
        if S * M >= nr and S * M <= max(2 * nr + 32, cover):
            out.append((S, M, R, 1, 1))
    for P in (2, 4, 8):
        out.append((out[0][0], out[0][1], 2, P if split_ok(nv, P) else 1, P if split_ok(ny, P) else 1))
    # passes 2 and 3 fused over slabs of 8 r nodes
    if nr * (8 if prec == "fp64" else 4) % 16 == 0:
        out.append((out[0][0], out[0][1], 2, 0, 1))
    # staged y planes (rows copied in 16-byte pieces): every shape, with
    # strips of 1 or 2 lines per segment and runs of 1 or 3 planes
    if nr * (8 if prec == "fp64" else 4) % 16 == 0:
        for (S, M), R, J in itertools.product(P1_SHAPES[prec], (1, 2), (1, 3)):
            if S * M >= nr and S * M <= max(2 * nr + 32, cover):
                out.append((S, M, R, 1, 1, 1, J))
    return out


def _shape(it):
    g = it["grid"]
    return g["n_r"], g["n_v"], g["n_y"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_every_tile_matches_oracle_pass_by_pass(H, orc, name, prec):
    import torch
    it = CASES[name]()
    nr, nv, ny = _shape(it)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 2e-6
    dev = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    with orc.Ctx(it) as X:
        U = X.step(0, X.terminal())
        n = 1
        th = X.time(n + 0.5)
        Ur = dev(U).double().cpu().numpy()
        want1 = X.solve_dir(0, th, X.explicit(n, Ur))
        dU1 = dev(want1)
        want2 = X.solve_dir(1, th, dU1.double().cpu().numpy())
        dU2 = dev(want2)
        want3 = Ur + X.solve_dir(2, th, dU2.double().cpu().numpy())
        try:
            for tile in tiles_for(it, prec):
                H.hjm_tile_set(nr, nv, ny, prec, tile)
                assert H.hjm_tile_get(nr, nv, ny, prec) == tuple(tile) + (0,) * (7 - len(tile))
                with H.Grid(it) as g:
                    out = torch.empty(g.shape, dtype=dt, device="cuda")
                    g.douglas_pass(prec, 1, n, dev(U), None, out)
                    got = out.double().cpu().numpy()
                    assert np.max(np.abs(got - want1)) <= tol * max(np.abs(want1).max(), np.abs(U).max()), \
                        ("pass 1", tile)
                    inp = dU1.clone()
                    g.douglas_pass(prec, 2, n, inp, None, inp)
                    got = inp.double().cpu().numpy()
                    assert np.max(np.abs(got - want2)) <= tol * max(np.abs(want2).max(), np.abs(want1).max()), \
                        ("pass 2", tile)
                    Ud = dev(U)
                    g.douglas_pass(prec, 3, n, dU2.clone(), Ud, Ud)
                    got = Ud.double().cpu().numpy()
                    assert np.max(np.abs(got - want3)) <= tol * max(np.abs(want3).max(), np.abs(want2).max()), \
                        ("pass 3", tile)
        finally:
            H.hjm_tile_set(nr, nv, ny, prec, None)


@pytest.mark.parametrize("name", list(CASES))
def test_split_tiles_march_matches_oracle(H, orc, name):
    it = CASES[name]()
    nr, nv, ny = _shape(it)
    pref = orc.price(it)
    try:
        for tile in tiles_for(it, "fp64")[-3:]:
            H.hjm_tile_set(nr, nv, ny, "fp64", tile)
            p = H.hjm_price_batch([it], "fp64")[0]
            assert abs(p - pref) <= 1e-10 * max(abs(pref), 1e-3), (tile, p, pref)
    finally:
        H.hjm_tile_set(nr, nv, ny, "fp64", None)


def test_tile_calls_validate_and_restore(H):
    default = H.hjm_tile_get(128, 64, 64, "fp32")
    default64 = H.hjm_tile_get(128, 64, 64, "fp64")
    for bad in [(16, 4, 4, 1, 1),      # 64 nodes do not cover n_r = 128
                (12, 16, 4, 1, 1),     # 12 lanes per line is not compiled
                (16, 8, 0, 1, 1),      # no lines
                (16, 8, 4, 3, 1),      # 3 warps per line
                (16, 8, 4, 1, 64),     # more warps than the y line allows
                (16, 8, 4, -1, 1)]:    # no such pass-2 mapping
        with pytest.raises(H.HJMError):
            H.hjm_tile_set(128, 64, 64, "fp32", bad)
    H.hjm_tile_set(128, 64, 64, "fp32", (32, 4, 2, 8, 4))
    assert H.hjm_tile_get(128, 64, 64, "fp32") == (32, 4, 2, 8, 4, 0, 0)
    H.hjm_tile_set(128, 64, 64, "fp32", (16, 8, 2, 1, 1, 1, 16))
    assert H.hjm_tile_get(128, 64, 64, "fp32") == (16, 8, 2, 1, 1, 1, 16)
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(130, 64, 64, "fp32", (16, 16, 1, 1, 1, 1, 8))  # 130 * 4 bytes: not 16-byte rows
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(128, 64, 64, "fp32", (16, 8, 1, 1, 1, 0, 8))   # planes only when staged
    assert H.hjm_tile_get(128, 64, 64, "fp64") == default64  # precisions are separate entries
    H.hjm_tile_set(128, 64, 64, "fp32", None)
    assert H.hjm_tile_get(128, 64, 64, "fp32") == default


def test_autotune_keeps_results(H):
    items = W.config2_draws(6, n_r=64, n_y=32, n_v=32, n_steps=40)
    before = H.hjm_price_batch(items, "fp64")
    H.hjm_autotune(items, "fp64", steps=4)
    tile = H.hjm_tile_get(64, 32, 32, "fp64")
    after = H.hjm_price_batch(items, "fp64")
    H.hjm_tile_set(64, 32, 32, "fp64", None)
    assert np.allclose(after, before, rtol=1e-11, atol=1e-15), tile
