"""The element-wise tolerance used to compare the surrogate network's GPU
forward pass and gradient with the CPU reference (tests/mlp_bounds.py),
checked on the CPU: it passes the rounding noise the GPU adds (every value
rounded to bfloat16 first perturbed at FP32 level, so that rounding decisions
near a bfloat16 boundary go the other way as they do on the GPU), and it
fails on mistakes planted in the reference's gradient and forward pass: a
wrong sign confined to a few rows, two swapped rows, a transposed block, a
dropped bias term."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from tests import mlp_bounds as B

N = 192


def _net(seed=21):
    # Glorot-uniform weights as the library initialises them, biases small.
    rng = np.random.default_rng(seed)
    p = np.zeros(M.N_PARAMS)
    for name, shape, off in M.LAYOUT:
        n = int(np.prod(shape))
        if name.startswith("W"):
            fi = shape[1] if len(shape) == 2 else shape[0]
            fo = shape[0] if len(shape) == 2 else 1
            a = np.sqrt(6.0 / (fi + fo))
            p[off:off + n] = rng.uniform(-a, a, n)
        else:
            p[off:off + n] = 0.01 * rng.standard_normal(n)
    lo = np.array([0.05, 0.005, 0.5, 0.1, -0.7, 1.0, 0.25, -0.02, 0.01])
    hi = np.array([0.2, 0.015, 2.0, 0.6, 0.3, 10.0, 1.0, 0.02, 0.07])
    x = lo + (hi - lo) * rng.random((N, 9))
    t = rng.standard_normal(N)
    return p, x, t, lo, hi


def _noisy_bf16(seed):
    """bfloat16 rounding of a value first moved by a relative FP32-level
    amount (a few units of 2^-24), as the GPU's FP32 arithmetic moves it."""
    rng = np.random.default_rng(seed)
    exact = M.bf16

    def r(a):
        a = np.asarray(a, np.float64)
        return exact(a * (1.0 + 4.0 * 2.0 ** -24 * rng.standard_normal(a.shape)))
    return r


def test_rounding_noise_passes(monkeypatch):
    p, x, t, lo, hi = _net()
    _, g = M.loss_and_grad(p, x, t, lo, hi, bf16_round=True)
    y = M.forward(p, x, lo, hi, bf16_round=True)
    gs, ys = B.grad_scale(p, x, t, lo, hi), B.forward_scale(p, x, lo, hi)
    monkeypatch.setattr(M, "bf16", _noisy_bf16(5))
    _, gn = M.loss_and_grad(p, x, t, lo, hi, bf16_round=True)
    yn = M.forward(p, x, lo, hi, bf16_round=True)
    assert np.any(gn != g)  # some rounding decisions did change
    eg, _ = B.elementwise_excess(gn, g, gs)
    ey, _ = B.elementwise_excess(yn, y, ys)
    assert eg < 0.2 and ey < 0.2, (eg, ey)


def _block(g, name):
    for n, shape, off in M.LAYOUT:
        if n == name:
            return g[off:off + int(np.prod(shape))].reshape(shape)
    raise KeyError(name)


@pytest.mark.parametrize("mistake", ["sign_3_rows_W2", "swap_rows_W1", "transpose_W3", "drop_b0",
                                     "sign_1_row_W0", "drop_b2", "sign_1_column_W1"])
def test_planted_gradient_mistakes_fail(mistake):
    p, x, t, lo, hi = _net()
    _, g = M.loss_and_grad(p, x, t, lo, hi, bf16_round=True)
    gs = B.grad_scale(p, x, t, lo, hi)
    bad = g.copy()
    if mistake == "sign_3_rows_W2":
        _block(bad, "W2")[[5, 77, 200]] *= -1.0
    elif mistake == "swap_rows_W1":
        w = _block(bad, "W1")
        w[[10, 11]] = w[[11, 10]]
    elif mistake == "transpose_W3":
        w = _block(bad, "W3")
        w[:] = w.T.copy()
    elif mistake == "drop_b0":
        _block(bad, "b0")[:] = 0.0
    elif mistake == "drop_b2":
        _block(bad, "b2")[:] = 0.0
    elif mistake == "sign_1_column_W1":
        _block(bad, "W1")[:, 40] *= -1.0
    else:
        _block(bad, "W0")[3] *= -1.0
    e, _ = B.elementwise_excess(bad, g, gs)
    assert e > 1.0, (mistake, e)


def test_planted_forward_mistakes_fail(monkeypatch):
    p, x, t, lo, hi = _net()
    y = M.forward(p, x, lo, hi, bf16_round=True)
    ys = B.forward_scale(p, x, lo, hi)
    P = M.unpack(p)
    # output bias dropped / output weights of one unit with the wrong sign
    _, (_, _, h) = M.forward(p, x, lo, hi, bf16_round=True, keep=True)
    for bad in (h[3] @ P["W4"], y - 2.0 * h[3][:, 7] * P["W4"][7]):
        assert B.elementwise_excess(bad, y, ys)[0] > 1.0
