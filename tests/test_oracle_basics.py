"""Pins of the oracle's building blocks against things other than itself:
scipy's spherical harmonics, numpy's fp16 rounding, SplitMix64's published
outputs, the exact binary logarithm, and Table 6 of the paper."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase from scipy's complex Y_l^m."""
    from scipy.special import sph_harm_y
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return float(np.real(sph_harm_y(l, 0, theta, phi)))
    Y = sph_harm_y(l, abs(m), theta, phi)
    return float(math.sqrt(2.0) * (np.real(Y) if m > 0 else np.imag(Y)))


def test_sh_basis_matches_scipy(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = orc.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, d), abs=1e-12)


def test_sh_basis_gradient_finite_difference(orc):
    rng = np.random.default_rng(6)
    for _ in range(10):
        d = rng.normal(size=3)
        _, G = orc.sh_basis(d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            Yp, _ = orc.sh_basis(d + e)
            Ym, _ = orc.sh_basis(d - e)
            np.testing.assert_allclose((Yp - Ym) / (2 * h), G[:, a], atol=1e-7)


def test_sh_known_values(orc):
    # Y_0^0 = 1/(2 sqrt(pi)), Y_1^1 = -sqrt(3/(4 pi)) x on the unit sphere
    Y, _ = orc.sh_basis(np.array([1.0, 0.0, 0.0]))
    assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
    assert Y[3] == pytest.approx(-math.sqrt(3.0 / (4.0 * math.pi)), abs=1e-15)


def test_fp16_rounding_matches_numpy(orc):
    rng = np.random.default_rng(7)
    xs = np.concatenate([
        rng.uniform(0, 2, 3000), rng.uniform(0, 1e-4, 2000), rng.uniform(60000, 70000, 200),
        np.ldexp(rng.integers(0, 2048, 500).astype(np.float64) + 0.5, -24),   # ties in subnormals
        np.ldexp(1024 + rng.integers(0, 1024, 500) + 0.5, -10),                 # ties in [1, 2)
        -rng.uniform(0, 2, 200), [0.0, 65504.0, 65519.99, 65520.0, 1e9],
    ])
    for x in xs:
        with np.errstate(over="ignore"):          # values past 65520 round to infinity, as intended
            want = int(np.array(x, dtype=np.float64).astype(np.float16).view(np.uint16))
        assert orc.double_to_half(float(x)) == want, x
    for h in range(0, 65536, 7):
        f = np.array(h, dtype=np.uint16).view(np.float16).astype(np.float64)
        got = orc.half_to_double(h)
        assert (math.isnan(got) and math.isnan(f)) or got == f


def test_splitmix64_published_outputs(orc):
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    gamma = int(g["gamma"], 16)
    for k, want in enumerate(g["outputs_from_state_0"], start=1):
        assert orc.mix64((k * gamma) % 2**64) == int(want, 16)


def test_neglog2_fixed_point(orc):
    rng = np.random.default_rng(8)
    hs = [int(x) for x in rng.integers(0, 2**63, 2000, dtype=np.int64)] + [0, 1, 2**63, 2**64 - 1, 12345]
    hs += [int(x) * 2 + 1 for x in rng.integers(0, 2**62, 500, dtype=np.int64)]
    for h in hs:
        u = h | 1
        exact = 64.0 - math.log2(u)
        got = orc.neglog2_q32(h) / 2**32
        assert abs(got - exact) < 2e-9 * max(1.0, exact), (h, got, exact)


def test_error_weight_is_exact(orc):
    for h in range(0, 65536, 3):
        f = np.array(h, dtype=np.uint16).view(np.float16).astype(np.float64)
        w = orc.err_weight(h)
        if not np.isfinite(f) or f < 0 or (f == 0 and h & 0x8000):
            assert w == 0
        else:
            assert w == int(f * 2**24) and float(w) == f * 2**24


def test_table6_defaults():
    from paper_2606_15924_gb300 import config as cfg
    import oracle
    t6 = json.load(open(os.path.join(GOLDEN, "hyperparams_tab6.json")))
    c = cfg.Config()
    assert c.sampling.r_hard == t6["r_hard"] and c.sampling.r_stable == t6["r_stable"]
    assert round(1 - c.sampling.r_hard - c.sampling.r_stable, 6) == t6["r_mixed_remainder"]
    assert c.loss.beta_ema == t6["beta_ema"] == oracle.BETA_EMA
    s = c.schedule
    assert (s.T, s.tau_until, s.tau_from, s.K_max, s.K_min, s.alpha, s.lambda_base) == (
        t6["T_fast"], t6["tau_until_fast"], t6["tau_from"], t6["K_max"], t6["K_min"],
        t6["alpha_view_schedule"], t6["lambda_base"])
    assert cfg.TILE == t6["tile_size"]
    lo, hi = t6["lambda_tile_scale_range"]
    assert lo < s.lam <= hi
