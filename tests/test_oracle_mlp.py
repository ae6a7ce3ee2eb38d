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


def _rot(axis, deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return {"x": np.array([[1, 0, 0], [0, c, -s], [0, s, c]]),
            "y": np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]]),
            "z": np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])}[axis]


def _matrix_of(q):
    # rotation matrix of a unit quaternion (w, x, y, z) (textbook form)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_quaternion_special_rotations():
    assert np.allclose(M.quaternion(np.eye(3)), [1, 0, 0, 0], atol=1e-15)
    for deg in (10.0, 75.0, 170.0):
        h = math.radians(deg) / 2
        assert np.allclose(M.quaternion(_rot("z", deg)), [math.cos(h), 0, 0, math.sin(h)], atol=1e-14)
        assert np.allclose(M.quaternion(_rot("x", deg)), [math.cos(h), math.sin(h), 0, 0], atol=1e-14)
    # half turns: w = 0, the axis carries the sign convention's remaining freedom
    for axis, e in (("x", 1), ("y", 2), ("z", 3)):
        q = M.quaternion(_rot(axis, 180.0))
        assert abs(q[0]) < 1e-12 and abs(abs(q[e]) - 1.0) < 1e-12


def test_quaternion_reconstructs_random_rotations():
    rng = np.random.default_rng(1)
    for _ in range(200):
        A = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        if np.linalg.det(A) < 0:
            A[:, 0] = -A[:, 0]
        q = M.quaternion(A)
        assert abs(np.linalg.norm(q) - 1) < 1e-13 and q[0] >= 0
        assert np.allclose(_matrix_of(q), A, atol=1e-12)


def test_features_are_frame_invariant():
    # rotating the lab frame rotates M's columns and every lab vector alike:
    # body-frame features are unchanged
    rng = np.random.default_rng(2)
    M0 = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    M0 *= np.sign(np.linalg.det(M0))
    v, w = rng.standard_normal(3), rng.standard_normal(3)
    Fh, Th = rng.standard_normal((4, 3)), rng.standard_normal((4, 3))
    Rl = _rot("y", 33.0) @ _rot("z", -71.0)
    a = M.features(M0, v, w, Fh, Th)
    b = M.features(M0 @ Rl.T, Rl @ v, Rl @ w, Fh @ Rl.T, Th @ Rl.T)
    assert np.allclose(a[4:], b[4:], atol=1e-12)
    assert a.shape == (34,)


def test_features_and_target_of_a_hand_worked_history():
    # Five consecutive trajectory records (t-3 .. t+1) of a body turned by
    # -90 degrees about z: its axes in the lab frame are d0 = (0, 1, 0),
    # d1 = (-1, 0, 0), d2 = (0, 0, 1), so M (rows d_i) takes lab (a, b, c) to
    # body (b, -a, c), and its quaternion is (cos 45, 0, 0, -sin 45).
    # Forces newest first F(t) = (0,0,4), F(t-1) = (0,0,2), F(t-2) = (3,0,0),
    # F(t-3) = (0,1,0): s_F = 4; torques T(t) = (1,0,0), T(t-1) = (0,2,0),
    # T(t-2) = 0, T(t-3) = (0,0,-1): s_T = 2.  v = (1,2,3), w = (0,0,0.5).
    # Next level F(t+1) = (1,0,7), T(t+1) = (2,-2,0): departures from linear
    # extrapolation (0,0,6) and (2,-2,0) are (1,0,1) and 0.  Every number
    # below is worked out by hand from these.
    d = np.array([0.0, 1.0, 0.0, -1.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    F = [(0, 1, 0), (3, 0, 0), (0, 0, 2), (0, 0, 4), (1, 0, 7)]   # t-3 .. t+1
    T = [(0, 0, -1), (0, 0, 0), (0, 2, 0), (1, 0, 0), (2, -2, 0)]
    log = np.zeros((5, M.LOG_REC))
    for j in range(5):
        log[j, 0:9] = d
        log[j, 9:12] = (1, 2, 3)
        log[j, 12:15] = (0, 0, 0.5)
        log[j, 15:18] = F[j]
        log[j, 18:21] = T[j]
        log[j, 21] = 100 + j
    x, y = M.samples(log)
    assert x.shape == (1, 34) and y.shape == (1, 6)
    r = math.sqrt(0.5)
    want_x = np.array([r, 0, 0, -r,                  # quaternion, w >= 0
                       2, -1, 3,                      # M v
                       0, 0, 0.5,                     # M w
                       0, 0, 1, 0, -0.5, 0,           # h = 0: M F(t) / 4, M T(t) / 2
                       0, 0, 0.5, 1, 0, 0,            # h = 1
                       0, -0.75, 0, 0, 0, 0,          # h = 2
                       0.25, 0, 0, 0, 0, -0.5])       # h = 3
    want_y = np.array([0, -0.25, 0.25, 0, 0, 0])
    assert np.abs(x[0] - want_x).max() < 1e-15, x[0] - want_x
    assert np.abs(y[0] - want_y).max() < 1e-15, y[0] - want_y
    # the network's output y turned back into a lab-frame prediction
    Fh = [np.array(F[3 - h], float) for h in range(4)]
    Th = [np.array(T[3 - h], float) for h in range(4)]
    Fp, Tp = M.prediction(d.reshape(3, 3), Fh, Th, want_y)
    assert np.abs(Fp - np.array([1, 0, 7])).max() < 1e-15
    assert np.abs(Tp - np.array([2, -2, 0])).max() < 1e-15
