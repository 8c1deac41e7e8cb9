"""Pins of the MLP oracle against facts independent of its code: central finite differences of
the real-valued network, closed forms, and the bf16 rounding rule on exact cases."""
import numpy as np

from oracle import mlp


def _data(seed, B=37):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, mlp.D_IN)) * 3 + 1
    t = rng.normal(size=B)
    mu, sd = x.mean(0), x.std(0) + 0.5
    return x, t, mu, sd


def test_gradient_matches_finite_differences():
    x, t, mu, sd = _data(1)
    p = mlp.init_params(7).astype(np.float64)
    loss, g = mlp.loss_and_grad(p, x, t, mu, sd, rounded=False)
    rng = np.random.default_rng(3)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 0, 8192 + 5, 8192 + 128 + 16384 + 128 + 3]])
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp = mlp.loss_and_grad(pp, x, t, mu, sd, rounded=False)[0]
        lm = mlp.loss_and_grad(pm, x, t, mu, sd, rounded=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])


def test_zero_network_outputs_bias_and_gradient_closed_form():
    x, t, mu, sd = _data(2, B=11)
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 0.75  # b3
    y, _ = mlp.forward(p, x, mu, sd)
    assert np.all(y == 0.75)
    loss, g = mlp.loss_and_grad(p, x, t, mu, sd)
    assert np.isclose(loss, 0.5 * np.mean((0.75 - t) ** 2))
    assert np.isclose(g[-1], np.mean(0.75 - t))  # d loss / d b3
    assert np.all(g[:-1] == 0.0)  # every ReLU is off


def test_single_path_closed_form():
    """One active unit per layer: y = w3_0 * relu(W2_00 * relu(W1_0 . xs + b1_0) + b2_0) + b3."""
    x, t, mu, sd = _data(4, B=5)
    P = {k: np.zeros(s) for k, s in mlp.SIZES}
    P["W1"][0, 3] = 0.5
    P["b1"][0] = 2.0
    P["W2"][0, 0] = 1.5
    P["b2"][0] = 0.25
    P["w3"][0] = -2.0
    P["b3"][0] = 0.125
    p = mlp.pack(P)
    xs = (x - mu) / sd
    h1 = np.maximum(0.5 * xs[:, 3] + 2.0, 0)
    expect = -2.0 * np.maximum(1.5 * h1 + 0.25, 0) + 0.125
    y, _ = mlp.forward(p, x, mu, sd, rounded=False)
    assert np.allclose(y, expect, rtol=0, atol=1e-12)


def test_bf16_rounding_rule():
    # exact bf16 values are fixed points; halfway cases round to even
    assert mlp.bf16(1.0) == 1.0 and mlp.bf16(-3.5) == -3.5
    one_ulp = 2.0 ** -7  # bf16 has 8 significant bits: ulp(1) = 2^-7
    assert mlp.bf16(1.0 + one_ulp / 2) == 1.0           # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * one_ulp / 2) == 1.0 + 2 * one_ulp  # tie -> even
    assert mlp.bf16(1.0 + one_ulp * 0.75) == 1.0 + one_ulp
    x = np.random.default_rng(5).normal(size=1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2.0 ** -8 * 1.0000001)


def test_rounded_forward_close_to_real_valued():
    x, t, mu, sd = _data(6)
    p = mlp.init_params(9).astype(np.float64)
    y1, _ = mlp.forward(p, x, mu, sd, rounded=True)
    y0, _ = mlp.forward(p, x, mu, sd, rounded=False)
    assert np.max(np.abs(y1 - y0)) < 0.05 * (1 + np.max(np.abs(y0)))
