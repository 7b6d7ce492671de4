"""Pins of the CPU FP64 surrogate-network reference (oracle/mlp_oracle.py):
its gradient against central finite differences of its own loss (exact FP64
network), and its bfloat16 rounding against the definition of the format."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _setup(n=7, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(M.N_PARAMS) * 0.05
    lo = np.array([0.05, 0.005, 0.5, 0.1, -0.7, 1.0, 0.25, -0.02, 0.01])
    hi = np.array([0.2, 0.015, 2.0, 0.6, 0.3, 10.0, 1.0, 0.02, 0.07])
    x = lo + (hi - lo) * rng.random((n, 9))
    t = rng.standard_normal(n)
    return p, x, t, lo, hi


def test_parameter_count():
    assert M.N_PARAMS == 9 * 256 + 256 + 3 * (256 * 256 + 256) + 256 + 1 == 200193


def test_gradient_matches_central_differences():
    p, x, t, lo, hi = _setup()
    _, g = M.loss_and_grad(p, x, t, lo, hi, bf16_round=False)
    rng = np.random.default_rng(9)
    # sample coordinates from every block
    idx = []
    for name, shape, off in M.LAYOUT:
        n = int(np.prod(shape))
        idx += list(off + rng.choice(n, size=min(6, n), replace=False))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = M.loss_and_grad(p + e, x, t, lo, hi, bf16_round=False)
        lm, _ = M.loss_and_grad(p - e, x, t, lo, hi, bf16_round=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_rounding_definition():
    # bfloat16 keeps 8 significant bits: 1 + 2^-7 is representable, 1 + 2^-8
    # is a tie (rounds to even: 1), 1 + 3 * 2^-8 rounds up to 1 + 2^-6.
    vals = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.0e-3])
    r = M.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1 + 2 ** -7 and r[2] == 1.0 and r[3] == 1 + 2 ** -6
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 2 ** -8 * 3.0e-3
    assert np.all(M.bf16(r) == r)


def test_silu_gradient():
    u = np.linspace(-6, 6, 25)
    fd = (M.silu(u + 1e-6) - M.silu(u - 1e-6)) / 2e-6
    assert np.allclose(M.silu_grad(u), fd, atol=1e-8)


def test_rounded_network_close_to_exact():
    p, x, t, lo, hi = _setup()
    y1 = M.forward(p, x, lo, hi, bf16_round=True)
    y0 = M.forward(p, x, lo, hi, bf16_round=False)
    assert np.max(np.abs(y1 - y0)) < 1e-2 * max(1.0, np.max(np.abs(y0)))


def _fd_mismatch(loss_and_grad, p, x, t, lo, hi):
    """Largest gap between a gradient routine and central differences of the
    (unmutated) loss on a sample of coordinates from every block."""
    _, g = loss_and_grad(p, x, t, lo, hi, bf16_round=False)
    rng = np.random.default_rng(19)
    worst = 0.0
    for name, shape, off in M.LAYOUT:
        n = int(np.prod(shape))
        fd, gi = [], []
        for i in off + rng.choice(n, size=min(4, n), replace=False):
            e = np.zeros_like(p)
            e[i] = 1e-6
            lp = float(np.mean((M.forward(p + e, x, lo, hi, False) - t) ** 2))
            lm = float(np.mean((M.forward(p - e, x, lo, hi, False) - t) ** 2))
            fd.append((lp - lm) / 2e-6)
            gi.append(g[i])
        fd, gi = np.array(fd), np.array(gi)
        worst = max(worst, np.max(np.abs(fd - gi)) / max(np.max(np.abs(fd)), 1e-12))
    return worst


@pytest.mark.parametrize("mutation", ["silu_grad_sign", "transposed_weight", "bias_grad_dropped"])
def test_planted_backward_mistakes_fail_the_pin(monkeypatch, mutation):
    # Each plausible mistake in the backward pass, planted in the reference,
    # must break the finite-difference pin above.
    p, x, t, lo, hi = _setup()
    assert _fd_mismatch(M.loss_and_grad, p, x, t, lo, hi) < 1e-5
    if mutation == "silu_grad_sign":
        monkeypatch.setattr(M, "silu_grad", lambda u: M.sigmoid(u) * (1.0 - u * (1.0 - M.sigmoid(u))))
    elif mutation == "transposed_weight":
        orig = M.unpack

        def unpack_t(q):
            P = orig(q)
            if unpack_t.calls == 1:  # the backward pass's own unpack
                for l in (1, 2, 3):
                    P["W%d" % l] = P["W%d" % l].T
            unpack_t.calls += 1
            return P
        unpack_t.calls = 0
        monkeypatch.setattr(M, "unpack", unpack_t)
    else:
        orig_lg = M.loss_and_grad

        def lg(q, *a, **k):
            l, g = orig_lg(q, *a, **k)
            g = g.copy()
            for name, shape, off in M.LAYOUT:
                if name.startswith("b"):
                    g[off:off + int(np.prod(shape))] = 0.0
            return l, g
        monkeypatch.setattr(M, "loss_and_grad", lg)
    assert _fd_mismatch(M.loss_and_grad, p, x, t, lo, hi) > 1e-2, mutation
