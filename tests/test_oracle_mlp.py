"""Pins of the FP64 surrogate-network oracle: GELU special values, the
composition of the layers in the affine limit, backpropagation against
central finite differences, and AdamW's bias correction.  No GPU."""
import math

import numpy as np

from oracle import mlp_oracle as M
from paper_2408_15115_gb300 import inputs as I


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, M.N_IN)), rng.standard_normal((n, M.N_OUT))


def test_layout_size():
    assert M.N_PARAM == 34 * 128 + 128 + 2 * (128 * 128 + 128) + 6 * 128 + 6 == 38278
    p = I.mlp_init_params(0)
    assert p.shape == (M.N_PARAM,)
    assert np.array_equal(M.pack(M.unpack(p)), p)


def test_gelu_special_values():
    # gelu(x) = x Phi(x): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (standard normal table)
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    x = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)  # Phi(x) + Phi(-x) = 1
    assert abs(M.gelu_prime(np.array(0.0)) - 0.5) < 1e-16
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.abs(fd - M.gelu_prime(x)).max() < 1e-9


def test_forward_is_the_affine_composition_when_gelu_is_the_identity():
    # with hidden pre-activations far above zero gelu(z) = z to rounding, so the
    # network is W4 (W3 (W2 (W1 x + b1) + b2) + b3) + b4, written column-wise
    rng = np.random.default_rng(3)
    P = M.unpack(I.mlp_init_params(1) * 0.05)
    for k in ("b1", "b2", "b3"):
        P[k] = 60.0 + rng.random(P[k].shape)
    P["b4"] = rng.standard_normal(6)
    p = M.pack(P)
    x, _ = _batch(4, 7)
    y, _ = M.forward(p, x)
    for i in range(4):
        h = x[i][:, None]
        for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4")):
            h = P[W] @ h + P[b][:, None]
        assert np.allclose(y[i], h[:, 0], rtol=1e-12, atol=1e-12)


def test_backprop_matches_central_differences():
    p = I.mlp_init_params(2)
    x, t = _batch(5, 11)
    _, g = M.loss_and_grad(p, x, t)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(M.N_PARAM, 300, replace=False),
                          np.arange(M.OFFSETS["b4"][0], M.N_PARAM),        # output biases
                          M.OFFSETS["b1"][0] + np.arange(0, 128, 17)])     # first-layer biases
    h = 1e-5
    for i in idx:
        e = np.zeros(M.N_PARAM)
        e[i] = h
        fd = (M.loss(p + e, x, t) - M.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_gradient_step_descends():
    p = I.mlp_init_params(4)
    x, t = _batch(16, 12)
    L0, g = M.loss_and_grad(p, x, t)
    assert M.loss(p - 1e-3 * g, x, t) < L0


def test_adamw_bias_correction_with_a_constant_gradient():
    # a constant gradient makes the corrected moments exactly g and g^2, so
    # every step moves each parameter by -lr (g / (|g| + eps) + wd p [weights])
    rng = np.random.default_rng(9)
    p = rng.standard_normal(M.N_PARAM)
    g = rng.standard_normal(M.N_PARAM)
    m = np.zeros(M.N_PARAM)
    v = np.zeros(M.N_PARAM)
    lr, wd, eps = 1e-3, 0.01, 1e-8
    mask = M.weight_mask()
    assert mask.sum() == 34 * 128 + 2 * 128 * 128 + 6 * 128
    for step in range(1, 6):
        q = p.copy()
        p, m, v = M.adamw(p, g, m, v, step, lr, eps=eps, wd=wd)
        want = q - lr * (g / (np.abs(g) + eps) + wd * mask * q)
        assert np.allclose(p, want, rtol=0, atol=1e-15)
