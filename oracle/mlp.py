"""CPU oracle of the learned cardinality estimator — TEST INFRASTRUCTURE ONLY.

A 3-layer perceptron 64 -> 128 -> 128 -> 1 with ReLU, predicting log(1 + |R(q')|) for a
sub-query q' (the cardinality Alg. 1 needs for each sub-query and in its join costs). The
network is defined with bf16 weights and fp32 accumulation, and every operand of its matrix
products is a bf16 value; this oracle computes in float64 and rounds to bf16 exactly at those
operands (the standardised input, both hidden layers' weights, the first hidden layer and,
backward, the layer errors that feed gradient products):

  x_s = bf16((x - mu) / sd)                        standardised input
  z1  = x_s @ bf16(W1).T + b1 ;  h1 = bf16(relu(z1))
  z2  = h1 @ bf16(W2).T + b2  ;  h2 = relu(z2)       (feeds only a dot product: fp32)
  y   = h2 @ w3 + b3

Loss: mean squared error 0.5 * mean((y - t)^2) over the rows. Backward (same rounding points):
  dy = (y - t) / B ; dz2 = (dy w3) * [z2 > 0] ; dz2_b = bf16(dz2)
  dh1 = dz2_b @ bf16(W2) ; dz1 = dh1 * [z1 > 0] ; dz1_b = bf16(dz1)
  dW2 = dz2_b.T @ h1 ; dW1 = dz1_b.T @ x_s ; db2 = sum dz2 ; db1 = sum dz1
  dw3 = h2.T @ dy ; db3 = sum dy

With bf16=False every rounding is skipped, which is the plain real-valued network; that form is
what the pins in tests/test_mlp_oracle.py check against finite differences.

Parameter vector layout (float32, 24961 entries): W1[128,64], b1[128], W2[128,128], b2[128],
w3[128], b3[1] (row-major, rows = output units).
"""
from __future__ import annotations

import numpy as np

D_IN, D_H = 64, 128
SIZES = [("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)), ("w3", (D_H,)),
         ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via the float32 value as the GPU does."""
    x32 = np.asarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, x, mu, sd, rounded=True):
    P = unpack(p)
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    xs = r((np.asarray(x, np.float64) - mu) / sd)
    z1 = xs @ r(P["W1"]).T + P["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(P["W2"]).T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, dict(xs=xs, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_and_grad(p, x, t, mu, sd, rounded=True):
    P = unpack(p)
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, x, mu, sd, rounded)
    B = len(y)
    diff = y - np.asarray(t, np.float64)
    loss = 0.5 * np.mean(diff ** 2)
    dy = diff / B
    dz2 = np.outer(dy, P["w3"]) * (c["z2"] > 0)
    dz2b = r(dz2)
    dh1 = dz2b @ r(P["W2"])
    dz1 = dh1 * (c["z1"] > 0)
    dz1b = r(dz1)
    g = {"W1": dz1b.T @ c["xs"], "b1": dz1.sum(0), "W2": dz2b.T @ c["h1"], "b2": dz2.sum(0),
         "w3": c["h2"].T @ dy, "b3": np.array([dy.sum()])}
    return loss, pack(g)


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation from a seeded generator."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        fan_in = {"W1": D_IN, "b1": D_IN, "W2": D_H, "b2": D_H, "w3": D_H, "b3": D_H}[name]
        bound = 1.0 / np.sqrt(fan_in)
        d[name] = rng.uniform(-bound, bound, size=shape)
    return pack(d).astype(np.float32)
