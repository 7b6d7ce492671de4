"""CPU FP64 reference of the pricing surrogate's network (test infrastructure).

TEST INFRASTRUCTURE ONLY: the GPU surrogate kernels are checked against this
module; the product path never imports it. It shares no code with them.

The network (the surrogate of the method's caplet price, not a part of the
paper's method): inputs x (9 raw features) are mapped to [-1, 1] by the
training box, z = 2 (x - lo) / (hi - lo) - 1; four hidden layers of width 256
with SiLU(u) = u / (1 + e^{-u}); a linear output. Layer 0 (9 -> 256) and the
output layer (256 -> 1) are evaluated in floating point without rounding; the
three 256 x 256 layers take their weights and their input activations
rounded to bfloat16 (round to nearest even), as the tensor-core kernels do,
and accumulate exactly (here in FP64). With bf16=False every rounding is
skipped and the function is the plain FP64 network, whose gradient is pinned
by central finite differences in the tests.

Parameter vector layout (float, flattened, this order):
  W0 [256 x 9], b0 [256], W1 [256 x 256], b1 [256], W2, b2, W3, b3,
  W4 [256], b4 [1]                                  (200,193 values)
Loss: mean over the batch of (y - t)^2.
"""
from __future__ import annotations

import numpy as np

WIDTH = 256
N_IN = 9


def layout():
    """(name, shape, offset) of every parameter block."""
    blocks = [("W0", (WIDTH, N_IN)), ("b0", (WIDTH,))]
    for l in (1, 2, 3):
        blocks += [("W%d" % l, (WIDTH, WIDTH)), ("b%d" % l, (WIDTH,))]
    blocks += [("W4", (WIDTH,)), ("b4", (1,))]
    out, off = [], 0
    for name, shape in blocks:
        n = int(np.prod(shape))
        out.append((name, shape, off))
        off += n
    return out, off


LAYOUT, N_PARAMS = layout()


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return {name: p[off:off + int(np.prod(shape))].reshape(shape) for name, shape, off in LAYOUT}


def bf16(a):
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sigmoid(u):
    return 1.0 / (1.0 + np.exp(-u))


def silu(u):
    return u * sigmoid(u)


def silu_grad(u):
    s = sigmoid(u)
    return s * (1.0 + u * (1.0 - s))


def normalise(x, lo, hi):
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * (x - lo) / (hi - lo) - 1.0


def forward(p, x, lo, hi, bf16_round=True, keep=False):
    P = unpack(p)
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    z = normalise(x, lo, hi)
    pre = [z @ P["W0"].T + P["b0"]]
    h = [r(silu(pre[0]))]
    for l in (1, 2, 3):
        pre.append(h[-1] @ r(P["W%d" % l]).T + P["b%d" % l])
        h.append(r(silu(pre[-1])))
    y = h[-1] @ P["W4"] + P["b4"][0]
    if keep:
        return y, (z, pre, h)
    return y


def loss_and_grad(p, x, t, lo, hi, bf16_round=True, keep=False):
    """Mean squared error and its gradient with respect to p (flattened).
    With bf16_round the backward pass rounds the back-propagated signal of
    the 256 x 256 layers to bfloat16 where the kernels do. With keep, also
    the forward intermediates (z, pre, h) and the back-propagated signals
    {"dy": dL/dy, "dz0".."dz3": dL/dpre of each hidden layer}."""
    P = unpack(p)
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    y, (z, pre, h) = forward(p, x, lo, hi, bf16_round, keep=True)
    n = len(y)
    dy = 2.0 * (y - t) / n
    g = {}
    g["W4"] = h[3].T @ dy
    g["b4"] = np.array([dy.sum()])
    dz = np.outer(dy, P["W4"]) * silu_grad(pre[3])
    sig = {"dy": dy, "dz3": dz}
    for l in (3, 2, 1):
        g["W%d" % l] = r(dz).T @ h[l - 1]
        g["b%d" % l] = dz.sum(axis=0)
        dh = r(dz) @ r(P["W%d" % l])
        dz = dh * silu_grad(pre[l - 1])
        sig["dz%d" % (l - 1)] = dz
    g["W0"] = dz.T @ z
    g["b0"] = dz.sum(axis=0)
    grad = np.concatenate([g[name].reshape(-1) for name, _, _ in LAYOUT])
    if keep:
        return float(np.mean((y - t) ** 2)), grad, (z, pre, h), sig
    return float(np.mean((y - t) ** 2)), grad
