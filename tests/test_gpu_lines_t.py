"""The TMA-fed strided passes (launch shape p2_warps = p3_warps =
HJM_LINES_TMA) against the CPU FP64 oracle and against the lane-per-line
kernels they replace: pass 2 (the v-line solve of Section 5.1) and pass 3
(the y-line solve fused with U^{n+1} = U^n + dU3) one at a time on ragged
r lengths (the last tile of 32 r nodes partly outside the field), both r
faces (Dirichlet r_min with gamma = 0; gamma > 0, where pass 3 falls back to
one lane per line), short and 256-node lines; whole FP32 marches of batches
large enough that every warp of the persistent grid marches several tiles
through its ring of slots (the refills), bit for bit equal to the
lane-per-line shape and within the FP32 price tolerance of the oracle; the
shapes the kernel refuses; and a bounded wait made to run out (a tile copy
that never starts), which must come back as HJM_ETIMEOUT and leave the
device usable. Tolerances as in test_gpu_tiles.py: one FP32 pass within
2e-6 of the larger of its input and output scales; FP32 prices within
max(1e-4 |p|, 1e-6)."""
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
    it = W.config2_draws(1, seed=W.SEED_BASE + 1100 + seed, n_r=n_r, n_y=n_y, n_v=n_v, n_steps=n_steps)[0]
    it["grid"].update(kw)
    return it


CASES = {
    "36x9x11_ragged": lambda: _caplet(36, 9, 11, 5),
    "100x12x20_NS": lambda: _caplet(100, 12, 20, 4, seed=1),
    "64x5x5_short_yorder1": lambda: _caplet(64, 5, 5, 4, seed=2, y_boundary_order=1),
    "32x256x6_long_y": lambda: _caplet(32, 256, 6, 3, seed=3),
    "32x6x256_long_v": lambda: _caplet(32, 6, 256, 3, seed=4),
    "gamma09_44x7x9": lambda: W.paper_2007_set(n_r=44, n_y=7, n_v=9, n_steps=12),
}


def _tma(H, it, p=None):
    g = it["grid"]
    H.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], "fp32", None)
    d = H.hjm_tile_get(g["n_r"], g["n_v"], g["n_y"], "fp32")
    p = H.HJM_LINES_TMA if p is None else p
    return d[:3] + (p, p) + d[5:]


@pytest.mark.parametrize("name", list(CASES))
def test_tma_strided_passes_match_oracle(H, orc, name):
    import torch
    it = CASES[name]()
    g = it["grid"]
    nr, nv, ny = g["n_r"], g["n_v"], g["n_y"]
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    with orc.Ctx(it) as X:
        U = X.step(0, X.terminal())
        n = 1
        th = X.time(n + 0.5)
        Ur = dev(U).double().cpu().numpy()
        dU1 = dev(X.solve_dir(0, th, X.explicit(n, Ur)))
        a1 = dU1.double().cpu().numpy()
        want2 = X.solve_dir(1, th, a1)
        dU2 = dev(want2)
        a2 = dU2.double().cpu().numpy()
        want3 = Ur + X.solve_dir(2, th, a2)
        got = {}
        try:
            for lane_per_line, tile in ((False, _tma(H, it)), (True, _tma(H, it, 1))):
                H.hjm_tile_set(nr, nv, ny, "fp32", tile)
                with H.Grid(it) as gr:
                    x = dU1.clone()
                    gr.douglas_pass("fp32", 2, n, x, None, x)
                    Ud = dev(Ur)
                    gr.douglas_pass("fp32", 3, n, dU2.clone(), Ud, Ud)
                    got[lane_per_line] = (x.cpu().numpy(), Ud.cpu().numpy())
        finally:
            H.hjm_tile_set(nr, nv, ny, "fp32", None)
    p2, p3 = got[False]
    assert np.max(np.abs(p2 - want2)) <= 2e-6 * max(np.abs(want2).max(), np.abs(a1).max()), name
    assert np.max(np.abs(p3 - want3)) <= 2e-6 * max(np.abs(want3).max(), np.abs(a2).max()), name
    # the same arithmetic as one lane per line
    assert np.array_equal(p2, got[True][0]) and np.array_equal(p3, got[True][1]), name
    H.hjm_wait_status()


@pytest.mark.parametrize("shape", [(64, 32, 32, 160), (96, 48, 48, 12), (128, 64, 64, 8), (96, 200, 16, 64)])
def test_tma_strided_march_batches(H, orc, shape):
    # B n_y ceil(n_r / 32) tiles per pass: several per warp of the persistent
    # grid, so every warp refills its slots; the last shape has y lines of
    # 200 nodes (few warps per SM) and a ragged last tile (n_r = 96)
    nr, ny, nv, B = shape
    items = W.config2_draws(B, seed=W.SEED_BASE + 1200 + nr, n_r=nr, n_y=ny, n_v=nv, n_steps=6)
    try:
        one, tma = _tma(H, items[0], 1), _tma(H, items[0])
        H.hjm_tile_set(nr, nv, ny, "fp32", one)
        ref = H.hjm_price_batch(items, "fp32")
        H.hjm_tile_set(nr, nv, ny, "fp32", tma)
        got = H.hjm_price_batch(items, "fp32")
    finally:
        H.hjm_tile_set(nr, nv, ny, "fp32", None)
    assert np.array_equal(np.asarray(got), np.asarray(ref))
    for i in (0, B - 1):
        q = orc.price(items[i])
        assert abs(got[i] - q) <= max(1e-4 * abs(q), 1e-6), (i, got[i], q)
    H.hjm_wait_status()


def test_tma_strided_with_tma_pass1(H, orc):
    # every pass of the Douglas step fed by TMA (pass 1 persistent, stage 3)
    items = W.config2_draws(8, seed=W.SEED_BASE + 1300, n_r=64, n_y=32, n_v=32, n_steps=10)
    try:
        H.hjm_tile_set(64, 32, 32, "fp32", (8, 8, 1, H.HJM_LINES_TMA, H.HJM_LINES_TMA, 3, 0))
        got = H.hjm_price_batch(items, "fp32")
    finally:
        H.hjm_tile_set(64, 32, 32, "fp32", None)
    for p, it in zip(got, items):
        q = orc.price(it)
        assert abs(p - q) <= max(1e-4 * abs(q), 1e-6), (p, q)


def test_tma_strided_shapes_are_validated(H):
    T = H.HJM_LINES_TMA
    base = H.hjm_tile_get(64, 32, 32, "fp32")[:3]
    with pytest.raises(H.HJMError):
        H.hjm_tile_set(64, 32, 32, "fp64", base + (T, T))        # FP32 only
    for nr, nv, ny in [(66, 32, 32),    # n_r not a multiple of 4 (16-byte rows)
                       (64, 257, 32),   # a v line of more than 256 nodes
                       (64, 32, 257)]:  # a y line of more than 256 nodes
        b = H.hjm_tile_get(nr, nv, ny, "fp32")[:3]
        with pytest.raises(H.HJMError):
            H.hjm_tile_set(nr, nv, ny, "fp32", b + (T, T))
    H.hjm_tile_set(64, 32, 32, "fp32", base + (1, 1))
    assert H.hjm_tile_get(64, 32, 32, "fp32")[3:5] == (1, 1)
    H.hjm_tile_set(64, 32, 32, "fp32", base + (T, T))
    assert H.hjm_tile_get(64, 32, 32, "fp32")[3:5] == (T, T)
    H.hjm_tile_set(64, 32, 32, "fp32", None)
    assert H.hjm_tile_get(64, 32, 32, "fp32")[3:5] == (T, T)  # the FP32 default


def test_tma_strided_bounded_wait_runs_out_and_reports(H):
    # Tile 3 of each pass-2 and pass-3 launch is never copied: the warp that
    # owns it gives up after a short bounded wait, leaves without writing its
    # remaining tiles, and the host reads HJM_ETIMEOUT; afterwards the
    # device prices normally again. Pass 1 reads its rows from global memory
    # (no TMA copy of its own is dropped).
    items = W.config2_draws(2, seed=W.SEED_BASE + 1400, n_r=64, n_y=10, n_v=16, n_steps=6)
    tile = (16, 4, 4, H.HJM_LINES_TMA, H.HJM_LINES_TMA, 0, 0)
    H.hjm_tile_set(64, 16, 10, "fp32", tile)
    try:
        ref = H.hjm_price_batch(items, "fp32")
        H.hjm_wait_status(reset=True)
        H.hjm_test_drop_plane(3, 2000)
        with pytest.raises(H.HJMError) as e:
            H.hjm_price_batch(items, "fp32")
        assert e.value.status == H.HJM_ETIMEOUT
    finally:
        H.hjm_test_drop_plane(-1, 0)
        H.hjm_tile_set(64, 16, 10, "fp32", None)
    H.hjm_wait_status(reset=True)
    H.hjm_tile_set(64, 16, 10, "fp32", tile)
    try:
        again = H.hjm_price_batch(items, "fp32")
    finally:
        H.hjm_tile_set(64, 16, 10, "fp32", None)
    H.hjm_wait_status()
    assert list(again) == list(ref)
