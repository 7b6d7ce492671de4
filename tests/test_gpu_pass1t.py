"""The TMA-fed pass 1 (launch shapes with p1_staged = 2, and 3 persistent)
against the CPU FP64 oracle: one Douglas pass 1 (Section 5.1: dt F(U^n) with the r-v mixed term,
then the r-line solve) for every compiled (lanes, nodes) shape, strips of one
or two lines per segment, runs of 1, 3 and 8 y planes (so runs start and end
on both y faces, and a run may hold the last plane alone) and the persistent
grid's balanced shares (runs that cross strips and instruments), v strips that
leave a ragged last strip, first- and second-order y faces, Nelson-Siegel
drift (a(t) at t^n and t^{n+1/2} differ) and flat curves; whole marches of
FP32 prices; the shapes the kernel does not cover falling back to the
default pass 1 (gamma > 0, the Craig-Sneyd correction stage); and a bounded
wait made to run out (a plane copy that is never started), which must come
back as HJM_ETIMEOUT and leave the device usable. Tolerances as in
test_gpu_tiles.py: one FP32 pass within 2e-6 of the larger of its input and
output scales; FP32 prices within max(1e-4 |p|, 1e-6)."""
import numpy as np
import pytest

from paper_1108_1688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(4, 16), (8, 8), (8, 12), (8, 16), (16, 8), (16, 12), (16, 16), (32, 8), (32, 16)]


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
    it = W.config2_draws(1, seed=W.SEED_BASE + 700 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    it["grid"].update(kw)
    return it


CASES = {
    # n_r = 64: strips of 16 (S = 8) or 32 (S = 4) lines; n_v = 35 leaves 3
    "64x10x35_NS": lambda: _caplet(64, 10, 35, 6, seed=1),
    "96x12x19_yorder1": lambda: _caplet(96, 12, 19, 5, seed=2, y_boundary_order=1),
    "128x9x16": lambda: _caplet(128, 9, 16, 4, seed=3),
    # padded lines: 160 nodes on 16 x 12, 224 on 16 x 16
    "160x7x20": lambda: _caplet(160, 7, 20, 4, seed=4),
    "224x6x16_flat": lambda: W.with_grid(_caplet(224, 6, 16, 4, seed=5), explicit_midpoint=1),
    "256x5x8": lambda: _caplet(256, 5, 8, 3, seed=6),
}


def tma_tiles(nr, nv):
    out = []
    for S, M in SHAPES:
        if S * M < nr or S * M > 2 * nr + 64:
            continue
        for R in (1, 2):
            KB = 4 * (32 // S) * R
            if nv % KB != 0 and nv % KB < 3:
                continue
            for J in (1, 3, 8):
                out.append((S, M, R, 1, 1, 2, J))
            out.append((S, M, R, 1, 1, 3, 0))  # persistent, balanced shares
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_tma_pass1_matches_oracle(H, orc, name):
    import torch
    it = CASES[name]()
    g = it["grid"]
    nr, nv, ny = g["n_r"], g["n_v"], g["n_y"]
    tiles = tma_tiles(nr, nv)
    assert tiles, name
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    with orc.Ctx(it) as X:
        U = X.step(0, X.terminal())
        for n in (1, g["n_steps"] - 1):
            Ur = dev(U).double().cpu().numpy()
            want = X.solve_dir(0, X.time(n + 0.5), X.explicit(n, Ur))
            scale = max(np.abs(want).max(), np.abs(Ur).max())
            try:
                for tile in tiles:
                    H.hjm_tile_set(nr, nv, ny, "fp32", tile)
                    assert H.hjm_tile_get(nr, nv, ny, "fp32") == tile
                    with H.Grid(it) as gr:
                        out = torch.full(gr.shape, float("nan"), dtype=torch.float32, device="cuda")
                        gr.douglas_pass("fp32", 1, n, dev(Ur), None, out)
                        got = out.double().cpu().numpy()
                    err = np.max(np.abs(got - want))
                    assert err <= 2e-6 * scale, (name, n, tile, err / scale)
            finally:
                H.hjm_tile_set(nr, nv, ny, "fp32", None)
    H.hjm_wait_status()


@pytest.mark.parametrize("name", ["64x10x35_NS", "160x7x20", "256x5x8"])
def test_tma_march_prices_match_oracle(H, orc, name):
    it = CASES[name]()
    g = it["grid"]
    nr, nv, ny = g["n_r"], g["n_v"], g["n_y"]
    items = [it, _caplet(nr, ny, nv, g["n_steps"], seed=40)]
    want = [orc.price(x) for x in items]
    try:
        for tile in tma_tiles(nr, nv)[:4]:
            H.hjm_tile_set(nr, nv, ny, "fp32", tile)
            got = H.hjm_price_batch(items, "fp32")
            for p, q in zip(got, want):
                assert abs(p - q) <= max(1e-4 * abs(q), 1e-6), (tile, p, q)
    finally:
        H.hjm_tile_set(nr, nv, ny, "fp32", None)


def test_uncovered_groups_fall_back(H, orc):
    # gamma > 0 (the r = 0 face is not Dirichlet) and the correction stage of
    # the Craig-Sneyd family are not covered by the TMA-fed kernel: with a
    # stage-2 shape set they run the default pass 1 and still match the oracle.
    gam = W.paper_2007_set(n_r=64, n_y=8, n_v=12, n_steps=12)
    cs = W.with_grid(_caplet(64, 8, 12, 6, seed=7), scheme=3, theta_adi=0.5 + 3 ** 0.5 / 6)
    try:
        for it in (gam, cs):
            g = it["grid"]
            H.hjm_tile_set(64, g["n_v"], g["n_y"], "fp32", (8, 8, 1, 1, 1, 2, 3))
            p = H.hjm_price_batch([it], "fp32")[0]
            q = orc.price(it)
            assert abs(p - q) <= max(1e-4 * abs(q), 1e-6), (p, q)
    finally:
        H.hjm_tile_set(64, 12, 8, "fp32", None)


def test_tma_shapes_are_validated(H):
    for bad in [(8, 16, 1, 1, 1, 2, 8),    # n_r = 130 is not a multiple of 32
                (8, 12, 1, 1, 1, 2, 8)]:   # 96 nodes do not cover 130
        with pytest.raises(H.HJMError):
            H.hjm_tile_set(130, 64, 64, "fp32", bad)
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(128, 64, 64, "fp64", (8, 16, 1, 1, 1, 2, 8))   # FP32 only
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(128, 17, 64, "fp32", (8, 16, 1, 1, 1, 2, 8))   # last v strip of one line
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(128, 64, 64, "fp32", (12, 16, 1, 1, 1, 2, 8))  # 12 lanes: not compiled


@pytest.mark.parametrize("tile", [(8, 8, 1, 1, 1, 2, 3), (8, 8, 1, 1, 1, 3, 0)])
def test_bounded_wait_runs_out_and_reports(H, tile):
    # A plane copy that is never started: every CTA whose run needs plane 2
    # gives up after a short bounded wait, leaves without writing, and the
    # host reads HJM_ETIMEOUT; afterwards the device prices normally again.
    items = [_caplet(64, 10, 16, 6, seed=8), _caplet(64, 10, 16, 6, seed=9)]
    H.hjm_tile_set(64, 16, 10, "fp32", tile)
    try:
        ref = H.hjm_price_batch(items, "fp32")[0]
        H.hjm_wait_status(reset=True)
        H.hjm_test_drop_plane(2, 2000)
        with pytest.raises(H.HJMError) as e:
            H.hjm_price_batch(items, "fp32")
        assert e.value.status == H.HJM_ETIMEOUT
    finally:
        H.hjm_test_drop_plane(-1, 0)
        H.hjm_tile_set(64, 16, 10, "fp32", None)
    H.hjm_wait_status(reset=True)
    H.hjm_tile_set(64, 16, 10, "fp32", tile)
    try:
        again = H.hjm_price_batch(items, "fp32")[0]
    finally:
        H.hjm_tile_set(64, 16, 10, "fp32", None)
    H.hjm_wait_status()
    assert again == ref
