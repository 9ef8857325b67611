"""Pins of the float64 perceptron reference: its gradient equals central
finite differences of its loss, and the bf16 rounding matches the format's
definition on hand-checked values."""
import numpy as np

import mlp_ref as R


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = R.random_params(rng)
    x = rng.normal(0, 1, (40, R.IN))
    y = rng.normal(0, 1, 40)
    _, g = R.loss_grad(p, x, y)
    idx = np.concatenate([rng.choice(R.NPARAM, 60, replace=False), [R.B3, R.B1, R.W3]])
    h = 1e-6
    for i in idx:
        e = np.zeros(R.NPARAM)
        e[i] = h
        fd = (R.loss_grad(p + e, x, y)[0] - R.loss_grad(p - e, x, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_rounding():
    # float32 bit pattern -> the bf16 it rounds to (top 16 bits), worked by hand:
    # below half / above half / exact ties to even (down and up) / negative /
    # large / denormal
    cases = {0x3F800000: 0x3F80, 0x3F807FFF: 0x3F80, 0x3F808001: 0x3F81,
             0x3F808000: 0x3F80, 0x3F818000: 0x3F82, 0xC0200000: 0xC020,
             0x7F61B1E6: 0x7F62, 0x000116C2: 0x0001}
    for bits, want in cases.items():
        f = np.array([bits], np.uint32).view(np.float32)
        got = R.bf16_round(f).astype(np.float32).view(np.uint32)[0]
        assert got == (want << 16), (hex(bits), hex(got))


def test_adam_reference_first_step():
    # first bias-corrected step moves every parameter by lr * sign(g)
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = R.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01, 0.9, 0.999, 1e-12)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-6)
