"""Pins of the CNN prox oracle (no GPU): bf16 rounding against torch's
conversion, the 3x3 convolution against scipy's correlation, an identity
network in closed form, the receptive field, the chain-rule gradient against
finite differences, and Adam's first step in closed form."""
import numpy as np
import pytest
import scipy.signal
import torch

from oracle import cnn
from synth.cnn_init import init_params


def test_bf16_round_matches_torch_conversion():
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(10000) * 10.0 ** g.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, -1.5, 65504.0, 3.0e38, 1.0e-39]]).astype(np.float32)
    # exact ties: 1 + 2^-8 (rounds down to even) and 1 + 3 * 2^-8 (rounds up)
    x = np.concatenate([x, np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16_round(x), ref)
    assert cnn.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert cnn.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_conv3x3_is_scipy_correlation_with_zero_fill():
    g = np.random.default_rng(1)
    a = g.standard_normal((3, 9, 7))
    W = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    out = cnn.conv3x3(a, W, b)
    for o in range(4):
        ref = sum(scipy.signal.correlate2d(a[c], W[o, c], mode="same", boundary="fill") for c in range(3)) + b[o]
        np.testing.assert_allclose(out[o], ref, atol=1e-12)


def _identity_params(scale_last=1.0):
    """Layers 1..7 copy channel 0 (centre tap 1), the last layer reads
    channel 0 with weight scale_last; all biases zero."""
    parts = []
    for l in range(1, cnn.N_LAYERS + 1):
        cin, cout = cnn.CHANNELS[l - 1], cnn.CHANNELS[l]
        W = np.zeros((cout, cin, 3, 3))
        W[0, 0, 1, 1] = scale_last if l == cnn.N_LAYERS else 1.0
        parts += [W.ravel(), np.zeros(cout)]
    return np.concatenate(parts)


def test_identity_network_doubles_a_nonnegative_input():
    """With copying layers and z >= 0 the ReLUs pass z through, so
    out = z + z exactly without rounding, and z + bf16(z) with it."""
    z = np.random.default_rng(2).uniform(0, 1, (12, 10)).astype(np.float32).astype(np.float64)
    p = _identity_params()
    out, _, _ = cnn.forward(p, z, rounding=False)
    np.testing.assert_array_equal(out, 2 * z)
    out, _, _ = cnn.forward(p, z, rounding=True)
    np.testing.assert_array_equal(out, cnn.f32_round(z + cnn.bf16_round(z)))
    # a negative input is cut by the first ReLU: out = z
    out, _, _ = cnn.forward(p, -z, rounding=False)
    np.testing.assert_array_equal(out, -z)


def test_receptive_field_is_eight_pixels():
    p = init_params(3).astype(np.float64)
    z = np.random.default_rng(3).uniform(0, 1, (24, 24))
    o0, _, _ = cnn.forward(p, z, rounding=False)
    z1 = z.copy()
    z1[11, 12] += 0.5
    o1, _, _ = cnn.forward(p, z1, rounding=False)
    changed = np.argwhere(np.abs(o1 - o0) > 0)
    assert np.abs(changed[:, 0] - 11).max() == 8 and np.abs(changed[:, 1] - 12).max() == 8


def test_gradient_matches_finite_differences():
    """Exact arithmetic (no rounding): the chain-rule gradient of the mean
    squared error equals central differences along random directions."""
    chans = (1, 4, 5, 1)
    g = np.random.default_rng(4)
    p = init_params(4, chans).astype(np.float64)
    p[-1] = 0.03                                            # a non-zero last bias
    z = g.uniform(0, 1, (9, 8))
    t = g.uniform(0, 1, (9, 8))
    loss, grad = cnn.loss_and_grad(p, z, t, rounding=False, channels=chans)
    for _ in range(5):
        v = g.standard_normal(p.size)
        h = 1e-5
        lp, _ = cnn.loss_and_grad(p + h * v, z, t, rounding=False, channels=chans)
        lm, _ = cnn.loss_and_grad(p - h * v, z, t, rounding=False, channels=chans)
        assert np.vdot(grad, v) == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    # the full-width network: a few single coordinates, one per layer
    p = init_params(5).astype(np.float64)
    z = g.uniform(0, 1, (10, 10))
    t = z + 0.1 * g.standard_normal((10, 10))
    loss, grad = cnn.loss_and_grad(p, z, t, rounding=False)
    k = 0
    for ws, bs in cnn.param_shapes():
        for idx in (k + 3, k + int(np.prod(ws)) + bs[0] - 1):
            e = np.zeros(p.size)
            e[idx] = 1e-5
            lp, _ = cnn.loss_and_grad(p + e, z, t, rounding=False)
            lm, _ = cnn.loss_and_grad(p - e, z, t, rounding=False)
            assert grad[idx] == pytest.approx((lp - lm) / 2e-5, rel=1e-5, abs=1e-10)
        k += int(np.prod(ws)) + bs[0]


def test_adam_first_step_closed_form():
    """At step 1 the bias corrections give m_hat = g and v_hat = g^2, so the
    update is lr g / (|g| + eps)."""
    g = np.random.default_rng(5)
    p = g.standard_normal(100)
    grad = g.standard_normal(100)
    p1, m, v = cnn.adam_step(p, grad, np.zeros(100), np.zeros(100), 1, 1e-3)
    np.testing.assert_allclose(p1, p - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * grad, atol=1e-16)
    np.testing.assert_allclose(v, 0.001 * grad ** 2, atol=1e-16)


def test_param_count():
    assert cnn.n_params() == 9 * 32 + 32 + 6 * (9 * 32 * 32 + 32) + 9 * 32 + 1 == init_params(0).size


def test_pnp_with_identity_network_is_fista_without_penalty():
    """A network whose residual branch is zero returns float32(z): the
    plug-and-play loop is then FISTA on Eq. 3 with beta = 0 (whose prox is
    the identity), up to that float32 rounding."""
    import math
    import oracle as orc
    n, na, nb = 12, 9, 16
    geo = orc.Geometry(np.arange(na) * math.pi / na, (nb - 1) / 2, nb, n, n, 0.5)
    g = np.random.default_rng(6)
    sino = geo.P(g.uniform(0, 1, (n, n))) + 0.01 * g.standard_normal((na, nb))
    L = 1.01 * orc.power_iteration(geo, np.ones((n, n)), 50)[0]
    p = np.zeros(cnn.n_params())
    for use_fista in (True, False):
        x, e = cnn.pnp_fista(geo, sino, p, L, 6, use_fista=use_fista)
        xr, er = orc.fista(geo, sino, 0.0, L, 6, n_inner=1, use_fista=use_fista)
        np.testing.assert_allclose(x, xr, rtol=1e-6, atol=1e-6 * np.abs(xr).max())
        np.testing.assert_allclose(e, er, rtol=1e-5)


def test_fista_returns_the_last_prox_input():
    """beta = 0: the prox is the identity, so the last z is the iterate;
    beta > 0: the iterate is the TV prox of the returned z."""
    import math
    import oracle as orc
    n, na, nb = 10, 7, 14
    geo = orc.Geometry(np.arange(na) * math.pi / na + 0.1, (nb - 1) / 2, nb, n, n, 0.5)
    sino = geo.P(np.random.default_rng(7).uniform(0, 1, (n, n)))
    L = 1.01 * orc.power_iteration(geo, np.ones((n, n)), 50)[0]
    x, _, z = orc.fista(geo, sino, 0.0, L, 4, n_inner=1, return_z=True)
    np.testing.assert_array_equal(x, z)
    x, _, z = orc.fista(geo, sino, 0.02, L, 4, n_inner=15, return_z=True)
    xp, _, _ = orc.tv_prox(z, 0.02 / L, 15)
    np.testing.assert_array_equal(x, xp)
