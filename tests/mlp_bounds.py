"""Element-wise tolerances for comparing the surrogate network's GPU forward
pass and loss gradient with the CPU FP64 reference (oracle/mlp_oracle.py).

Both sides round the same quantities to bfloat16 (the weights and input
activations of the three 256 x 256 layers, and the back-propagated signal that
enters their transposed products), but the GPU forms the values it rounds in
FP32 and the reference in FP64. Where such a value lies within FP32 rounding
of a bfloat16 rounding boundary, the two sides round it to neighbouring
bfloat16 numbers, one unit in the last place apart: at most 2^-7 of its
magnitude. A factor is that close to a boundary with probability of order
2^8 times its FP32 relative error, i.e. rarely.

Each output element is a sum of products. Its magnitude scale is the sum of
the absolute values of those products plus, for a gradient element, one level
up: the sum of the absolute values of the products that form its
back-propagated factor, all taken with the reference's own values.
If every rounding among those products went the other way, the element would
move by about one bfloat16 unit of that scale; the tolerance is that unit,
2^-7 of the scale. FP32 accumulation (about 2^-24 per term) and flips further
upstream (damped by the cancellation of the sums they pass through) stay far
below it: with the GPU's FP32 rounding simulated, the largest difference is
about 5 % of the tolerance. A wrong sign, a wrong index or a dropped term
moves an element by more than twice it (tests/test_mlp_bounds.py).
"""
from __future__ import annotations

import numpy as np

from oracle import mlp_oracle as M

# One bfloat16 unit in the last place, relative to the magnitude scale.
REL = 2.0 ** -7

_A = np.abs


def forward_scale(p, x, lo, hi):
    """Magnitude scale of each forward output: |h3| . |W4| + |b4| (the output
    layer's products; its FP32 input h3 is not rounded, and a flipped h2
    moves h3 by one 2^-7 part of one of its 256 terms)."""
    P = M.unpack(p)
    _, (_, _, h) = M.forward(p, x, lo, hi, bf16_round=True, keep=True)
    return _A(h[3]) @ _A(P["W4"]) + abs(P["b4"][0])


def grad_scale(p, x, t, lo, hi):
    """Magnitude scale of each gradient element (flattened like the parameter
    vector): |bf16(dz_l)|^T |h_{l-1}| for W_l and sum_n |dz_l| for b_l (W0,
    b0 alike with the normalised inputs z, W4 and b4 with dL/dy), where each
    |dz_l| also carries the products that form it from the layer above,
    (|bf16(dz_{l+1})| |bf16(W_{l+1})|) * |silu'(pre_l)|."""
    P = M.unpack(p)
    _, _, (z, pre, h), sig = M.loss_and_grad(p, x, t, lo, hi, bf16_round=True, keep=True)
    dyA = _A(sig["dy"])
    g = {"W4": _A(h[3]).T @ dyA, "b4": np.array([dyA.sum()])}
    dz_up = np.outer(dyA, _A(P["W4"])) * _A(M.silu_grad(pre[3]))
    for l in (3, 2, 1, 0):
        own = _A(M.bf16(sig["dz%d" % l])) if l > 0 else _A(sig["dz0"])
        dzA = own + dz_up
        prev = _A(h[l - 1]) if l > 0 else _A(z)
        g["W%d" % l] = dzA.T @ prev
        g["b%d" % l] = dzA.sum(axis=0)
        if l > 0:
            dz_up = (_A(M.bf16(sig["dz%d" % l])) @ _A(M.bf16(P["W%d" % l]))) * _A(M.silu_grad(pre[l - 1]))
    return np.concatenate([g[name].reshape(-1) for name, _, _ in M.LAYOUT])


def elementwise_excess(got, want, scale, rel=REL):
    """Largest |got - want| / (rel * scale) over the elements (<= 1 passes),
    with the index of that element."""
    d = _A(np.asarray(got, np.float64) - np.asarray(want, np.float64))
    q = d / (rel * np.maximum(scale, 1e-300))
    i = int(np.argmax(q))
    return float(q[i]), i
