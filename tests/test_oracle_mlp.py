"""Pins of the oracle's tile-error MLP: bfloat16 rounding against torch's
conversion, finite differences of the double-precision network, the bf16
mode equal to the plain network when every value is exactly representable,
and ReLU gating."""
import math

import numpy as np
import pytest
import torch


def _net(rng, scale=0.3):
    return dict(W1=rng.normal(0, scale, (128, 16)), b1=rng.normal(0, 0.1, 128), W2=rng.normal(0, scale / 4, (128, 128)),
                b2=rng.normal(0, 0.1, 128), W3=rng.normal(0, scale / 4, 128), b3=rng.normal(0, 0.1, 1))


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.normal(0, 10, 3000), rng.uniform(-1, 1, 3000),
                         (1 + np.arange(256) / 256.0 + 1 / 512.0),          # ties
                         [0.0, -0.0, 1e-40, 3.4e38, -2.5]])
    want = torch.tensor(xs, dtype=torch.float64).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.round_bf16(float(v)) for v in xs])
    np.testing.assert_array_equal(got, want)


def test_mlp_finite_differences(orc):
    rng = np.random.default_rng(1)
    w = _net(rng)
    x = np.zeros((40, 16))
    x[:, :5] = rng.normal(size=(40, 5))
    t = rng.normal(size=40)
    loss, g = orc.mlp_backward(x, t, w, bf16=False)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = w[name].reshape(-1)
        idx = rng.choice(flat.size, min(12, flat.size), replace=False)
        for i in idx:
            wp = {k: v.copy() for k, v in w.items()}
            wm = {k: v.copy() for k, v in w.items()}
            wp[name].reshape(-1)[i] += h
            wm[name].reshape(-1)[i] -= h
            fd = (orc.mlp_backward(x, t, wp, bf16=False)[0] - orc.mlp_backward(x, t, wm, bf16=False)[0]) / (2 * h)
            assert fd == pytest.approx(g[name].reshape(-1)[i], rel=1e-5, abs=1e-9), (name, i)
    y, _, _ = orc.mlp_forward(x, w, bf16=False)
    assert loss == pytest.approx(0.5 * np.mean((y - t) ** 2), rel=1e-12)


def test_bf16_mode_is_exact_on_representable_values(orc):
    """Small integer weights and inputs keep every product, sum and
    activation an integer below 256, exact in bfloat16: both modes agree."""
    rng = np.random.default_rng(2)
    w = dict(W1=rng.integers(-1, 2, (128, 16)).astype(float), b1=rng.integers(-1, 2, 128).astype(float),
             W2=np.zeros((128, 128)), b2=rng.integers(0, 3, 128).astype(float),
             W3=rng.integers(-1, 2, 128).astype(float), b3=np.array([1.0]))
    w["W2"][np.arange(128), rng.integers(0, 128, 128)] = 1.0        # one input per unit
    x = np.zeros((20, 16))
    x[:, :5] = rng.integers(0, 4, (20, 5))
    ya, _, _ = orc.mlp_forward(x, w, bf16=True)
    yb, _, _ = orc.mlp_forward(x, w, bf16=False)
    np.testing.assert_array_equal(ya, yb)
    t = rng.integers(-5, 5, 20).astype(float)
    la, ga = orc.mlp_backward(x, t, w, bf16=True)
    lb, gb = orc.mlp_backward(x, t, w, bf16=False)
    # adjoints are multiples of 1/R with small numerators: exact in bf16 for R = 20? not always,
    # so compare within bf16 rounding of the hidden adjoints
    for k in ga:
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-2, atol=1e-2 * np.abs(gb[k]).max() + 1e-12)


def test_relu_gating(orc):
    rng = np.random.default_rng(3)
    w = _net(rng)
    w["b1"][:] = -100.0                         # every first-layer unit inactive
    x = np.zeros((10, 16))
    x[:, :5] = rng.normal(size=(10, 5))
    y, h1, h2 = orc.mlp_forward(x, w, bf16=False)
    assert np.all(h1 == 0)
    np.testing.assert_allclose(h2, np.maximum(w["b2"], 0)[None, :].repeat(10, 0))
    _, g = orc.mlp_backward(x, rng.normal(size=10), w, bf16=False)
    assert np.all(g["W1"] == 0) and np.all(g["b1"] == 0) and np.all(g["W2"] == 0)


def test_bf16_rounding_ties_to_even(orc):
    """Values exactly half way between two bfloat16 neighbours round to the
    one with an even last bit (1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6 ...),
    as torch's conversion does."""
    import torch
    for base in (1.0, -3.0, 0.75, 1024.0):
        ulp = 2.0 ** (math.floor(math.log2(abs(base))) - 7)     # bf16 spacing in base's binade
        for k in range(-6, 7):
            x = base + (k + 0.5) * ulp * (1 if base > 0 else -1)
            want = float(torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float())
            assert orc.round_bf16(x) == want, (x, orc.round_bf16(x), want)
