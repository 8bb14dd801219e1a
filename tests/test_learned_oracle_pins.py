"""Pins of the learned-halo oracle pieces (CPU only): the numpy FP64 backprop against finite
differences, the C forward against numpy, and the BF16 rounding against its definition."""
import numpy as np

from oracle import mlp
from oracle import oracle as orc


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(5).astype(np.float64)
    X = rng.standard_normal((7, mlp.NIN))
    T = rng.standard_normal((7, mlp.NOUT))
    loss, g = mlp.loss_and_grad(p, X, T)
    idx = rng.choice(mlp.NPARAM, size=40, replace=False)
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T)[0] - mlp.loss_and_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_gelu_derivative_matches_finite_differences():
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_c_forward_matches_numpy():
    rng = np.random.default_rng(4)
    p = mlp.init_params(2)
    for _ in range(5):
        x = np.array([orc.bf16(v) for v in rng.standard_normal(mlp.NIN)])
        np.testing.assert_allclose(orc.mlp_forward_c(p, x), mlp.forward(p, x[None])[0][0], rtol=1e-13, atol=1e-13)


def test_bf16_rounding_is_round_to_nearest_even():
    assert orc.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even
    assert orc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (upwards)
    assert orc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert orc.bf16(-3.0) == -3.0
    assert orc.bf16(1e-30) > 0
    x = np.random.default_rng(1).standard_normal(1000)
    for v in x:
        b = orc.bf16(v)
        assert abs(b - v) <= 2.0 ** -8 * abs(v)                  # within half a BF16 ulp
