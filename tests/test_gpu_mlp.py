"""The tensor-core MLP (forward, gradient, Adam training) against the CPU oracle oracle/mlp.py.

Tolerances: both sides round to bf16 at the same points (every operand of a tensor-core
product is bf16: the standardised input, the weights, h1 and the layer-2 error dz2, dz1); the
GPU accumulates in fp32 (tensor cores, then atomics across 128-row tiles) where the oracle uses
float64, so outputs agree to ~1e-6 relative, except where an fp32 value sits within its rounding
error of a bf16 rounding boundary (rare: ~1e-7 / 2^-8 per element) and flips one bf16 ulp (2^-8
relative) of a single hidden activation. In a gradient entry summed over B rows that flip moves
one of B terms by 2^-8 of its size. The bounds below (1e-3 relative per entry, plus an absolute
1e-4 of the parameter block's largest entry for entries that cancel to near zero) leave an
order of magnitude above that.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _setup(seed, rows):
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(rows, 64)) * rng.uniform(0.5, 4, size=64) + rng.normal(size=64)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.1 * x[:, 1] - 0.05 * x[:, 2] ** 2).astype(np.float32)
    mu = x.mean(0).astype(np.float32)
    sd = (x.std(0) + 0.1).astype(np.float32)
    return x, t, mu, sd


@pytest.mark.parametrize("rows", [1, 128, 300])
def test_forward_matches_oracle(gpu_lib, rows):
    import torch

    huge = gpu_lib
    x, t, mu, sd = _setup(rows, rows)
    p = omlp.init_params(11)
    m = huge.MLP(0)
    m.set_params(p, mu, sd)
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros(rows, dtype=torch.float32, device="cuda")
    m.forward(dx, dy)
    y = dy.cpu().numpy().astype(np.float64)
    ye, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64), mu.astype(np.float64),
                         sd.astype(np.float64))
    assert np.allclose(y, ye, rtol=1e-3, atol=1e-3), np.max(np.abs(y - ye))


def test_gradient_matches_oracle(gpu_lib):
    import torch

    huge = gpu_lib
    rows = 300
    x, t, mu, sd = _setup(5, rows)
    p = omlp.init_params(13)
    m = huge.MLP(0)
    m.set_params(p, mu, sd)
    g = torch.zeros(m.n_params, dtype=torch.float32, device="cuda")
    loss = m.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), g)
    le, ge = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64),
                                mu.astype(np.float64), sd.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss - le) <= 1e-3 * (1 + abs(le))
    o = 0
    for name, shape in omlp.SIZES:
        n = int(np.prod(shape))
        a, b = gg[o:o + n], ge[o:o + n]
        atol = 1e-4 * float(np.max(np.abs(b))) + 1e-9
        bad = ~np.isclose(a, b, rtol=1e-3, atol=atol)
        assert not bad.any(), (name, int(bad.sum()), n, np.flatnonzero(bad)[:5], a[bad][:5], b[bad][:5])
        o += n


def test_training_reduces_loss(gpu_lib):
    import torch

    huge = gpu_lib
    rows = 4096
    x, t, mu, sd = _setup(7, rows)
    m = huge.MLP(3)
    m.set_params(None, mu, sd)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    g = torch.zeros(m.n_params, dtype=torch.float32, device="cuda")
    l0 = m.loss_grad(dx, dt, g)
    l1 = m.train(dx, dt, epochs=200, batch_rows=1024, lr=2e-3)
    l2 = m.loss_grad(dx, dt, g)
    assert l2 < 0.2 * l0, (l0, l1, l2)
