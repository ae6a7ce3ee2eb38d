"""Plain FP64 reference of the force/torque surrogate network (TEST
INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's CPU leg
may use it; it shares no code with the CUDA path).

The surrogate is not part of the paper: the paper's only predictor is the
orientation predictor-corrector of the rigid-body update (Sec. 2.3).  The
network maps the particle's recent state to its next hydrodynamic force and
torque, so that the marker velocities of the immersed-boundary step (Sec. 2.2)
can be predicted at t + 1 instead of t + 1/2.

Network: 34 inputs -> three hidden layers of 128 GELU units -> 6 outputs,
    z_1 = W_1 x + b_1,  a_l = gelu(z_l),  z_{l+1} = W_{l+1} a_l + b_{l+1},
    y = W_4 a_3 + b_4,
with GELU in its exact form gelu(x) = x Phi(x), Phi the standard normal CDF,
on standardised inputs and outputs; loss = mean over samples and outputs of
(y - t)^2.  Backpropagation is the chain rule written out layer by layer.
AdamW is Loshchilov & Hutter, "Decoupled weight decay regularization" (2019):
moments with bias correction, weight decay applied to the weight matrices
directly (not through the gradient).

Flat parameter layout (float, shared with the C ABI):
    W1 [128][34], b1 [128], W2 [128][128], b2 [128], W3 [128][128], b3 [128],
    W4 [6][128], b4 [6]   -> 38278 values.
"""
import math

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 34, 128, 6
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]


def _offsets():
    off, out = 0, {}
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


OFFSETS, N_PARAM = _offsets()


def unpack(p):
    """Views of the flat parameter vector as the named matrices."""
    p = np.asarray(p, dtype=np.float64)
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFFSETS.items()}


def pack(d):
    out = np.zeros(N_PARAM)
    for k, (o, s) in OFFSETS.items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], dtype=np.float64).reshape(-1)
    return out


def weight_mask():
    """1 for weight-matrix entries (decayed by AdamW), 0 for biases."""
    m = np.zeros(N_PARAM)
    for k, (o, s) in OFFSETS.items():
        if k.startswith("W"):
            m[o:o + int(np.prod(s))] = 1.0
    return m


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_prime(x):
    # d/dx [x Phi(x)] = Phi(x) + x phi(x)
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p, x):
    """x: standardised inputs [n][34] -> (y [n][6], cache)."""
    P = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ P["W1"].T + P["b1"]
    a1 = gelu(z1)
    z2 = a1 @ P["W2"].T + P["b2"]
    a2 = gelu(z2)
    z3 = a2 @ P["W3"].T + P["b3"]
    a3 = gelu(z3)
    y = a3 @ P["W4"].T + P["b4"]
    return y, (x, z1, a1, z2, a2, z3, a3)


def loss(p, x, t):
    y, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grad(p, x, t):
    """Mean squared error and its gradient with respect to the flat parameters."""
    P = unpack(p)
    y, (x, z1, a1, z2, a2, z3, a3) = forward(p, x)
    t = np.asarray(t, dtype=np.float64)
    n = x.shape[0]
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (n * N_OUT)
    g = {"W4": dy.T @ a3, "b4": dy.sum(0)}
    dz3 = (dy @ P["W4"]) * gelu_prime(z3)
    g["W3"], g["b3"] = dz3.T @ a2, dz3.sum(0)
    dz2 = (dz3 @ P["W3"]) * gelu_prime(z2)
    g["W2"], g["b2"] = dz2.T @ a1, dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * gelu_prime(z1)
    g["W1"], g["b1"] = dz1.T @ x, dz1.sum(0)
    return L, pack(g)


def adamw(p, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    p = p - lr * (mhat / (np.sqrt(vhat) + eps) + wd * weight_mask() * p)
    return p, m, v


def standardisation(data):
    """Per-column mean and standard deviation (population), zero std -> 1."""
    data = np.asarray(data, dtype=np.float64)
    mu = data.mean(0)
    sd = data.std(0)
    sd[sd == 0.0] = 1.0
    return mu, sd


# --------------------------------------------------------------------------
# Predictor features (the network's inputs), from the particle state at time
# level t with orientation matrix M (rows d_0, d_1, d_2: the body axes):
#   quaternion (w, x, y, z), w >= 0, of M; M v; M w; M F(t-h) / sF,
#   M T(t-h) / sT for h = 0..3, sF = max_h |F(t-h)|, sT = max_h |T(t-h)|.
# Targets: M (F(t+1) - 2 F(t) + F(t-1)) / sF and the torque alike -- the
# departure from linear extrapolation -- so F^ = 2 F(t) - F(t-1) + sF M^T y.

def quaternion(M):
    """Unit quaternion (w, x, y, z), w >= 0, with rotation matrix M.  The
    products q q^T are linear in M (the matrix entries of a unit quaternion's
    rotation are quadratic in q), so q is the principal eigenvector of that
    4 x 4 matrix."""
    M = np.asarray(M, dtype=np.float64).reshape(3, 3)
    tr = np.trace(M)
    Q = 0.25 * np.array([
        [1 + tr, M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]],
        [M[2, 1] - M[1, 2], 1 + M[0, 0] - M[1, 1] - M[2, 2], M[0, 1] + M[1, 0], M[0, 2] + M[2, 0]],
        [M[0, 2] - M[2, 0], M[0, 1] + M[1, 0], 1 - M[0, 0] + M[1, 1] - M[2, 2], M[1, 2] + M[2, 1]],
        [M[1, 0] - M[0, 1], M[0, 2] + M[2, 0], M[1, 2] + M[2, 1], 1 - M[0, 0] - M[1, 1] + M[2, 2]]])
    w, V = np.linalg.eigh(Q)
    q = V[:, np.argmax(w)]
    q = q / np.linalg.norm(q)
    return -q if q[0] < 0 else q


def scales(Fh, Th):
    sF = max(float(np.linalg.norm(f)) for f in Fh) or 1.0
    sT = max(float(np.linalg.norm(t)) for t in Th) or 1.0
    return sF, sT


def features(M, v, w, Fh, Th):
    """Inputs of the network: Fh, Th = lab-frame forces and torques at t, t-1,
    t-2, t-3 (newest first)."""
    M = np.asarray(M, dtype=np.float64).reshape(3, 3)
    sF, sT = scales(Fh, Th)
    out = [quaternion(M), M @ np.asarray(v, float), M @ np.asarray(w, float)]
    for h in range(4):
        out += [M @ np.asarray(Fh[h], float) / sF, M @ np.asarray(Th[h], float) / sT]
    return np.concatenate(out)


def target(M, Fh, Th, F_next, T_next):
    M = np.asarray(M, dtype=np.float64).reshape(3, 3)
    sF, sT = scales(Fh, Th)
    lin_F = 2 * np.asarray(Fh[0], float) - np.asarray(Fh[1], float)
    lin_T = 2 * np.asarray(Th[0], float) - np.asarray(Th[1], float)
    return np.concatenate([M @ (np.asarray(F_next, float) - lin_F) / sF, M @ (np.asarray(T_next, float) - lin_T) / sT])


def prediction(M, Fh, Th, y):
    """Lab-frame (F^, T^) from the network's outputs y [6]."""
    M = np.asarray(M, dtype=np.float64).reshape(3, 3)
    sF, sT = scales(Fh, Th)
    return (2 * np.asarray(Fh[0], float) - np.asarray(Fh[1], float) + sF * (M.T @ y[:3]),
            2 * np.asarray(Th[0], float) - np.asarray(Th[1], float) + sT * (M.T @ y[3:]))


LOG_REC = 32


def samples(log):
    """(x [n-4][34], y [n-4][6]) from n consecutive trajectory records
    [n][32] (d [9], v [3], w [3], F [3], T [3], step, ...)."""
    log = np.asarray(log, dtype=np.float64)
    xs, ys = [], []
    for j in range(log.shape[0] - 4):
        t = j + 3
        M = log[t, 0:9].reshape(3, 3)
        Fh = [log[t - h, 15:18] for h in range(4)]
        Th = [log[t - h, 18:21] for h in range(4)]
        xs.append(features(M, log[t, 9:12], log[t, 12:15], Fh, Th))
        ys.append(target(M, Fh, Th, log[t + 1, 15:18], log[t + 1, 18:21]))
    return np.array(xs), np.array(ys)
