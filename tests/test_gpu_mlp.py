"""The surrogate network's GPU kernels against the FP64 oracle: forward
outputs and every parameter gradient in the FP32 check mode (<= 1e-5) and
with BF16 tensor-core products (<= 2e-2), the fused inference kernel against
the training kernels, AdamW against the oracle's update, and a monotone
training loss on a fixed batch."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2408_15115_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, M.N_IN)) * rng.uniform(0.5, 3.0, M.N_IN) + rng.uniform(-2, 2, M.N_IN)
    y = np.tanh(x[:, :6] * 0.7) + 0.1 * x[:, 6:12] * x[:, 12:18] + 0.3
    return x, y


def _norm(x, y):
    mx, sx = M.standardisation(x)
    my, sy = M.standardisation(y)
    return mx, sx, my, sy


def _net(precision, p, norm, cap=512):
    from paper_2408_15115_gb300 import turret as T
    net = T.MLP(p.astype(np.float32), batch_cap=cap, precision=precision)
    net.set_norm(*[v.astype(np.float32) for v in norm])
    return net


def _oracle(p, x, y, norm):
    mx, sx, my, sy = norm
    # the oracle sees the float32 values the GPU sees
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    xs = (f(x) - f(mx)) / f(sx)
    ts = (f(y) - f(my)) / f(sy)
    out, _ = M.forward(f(p), xs)
    L, g = M.loss_and_grad(f(p), xs, ts)
    return out * f(sy) + f(my), L, g


def _per_tensor_err(g, ref):
    worst = 0.0
    for k, (o, s) in M.OFFSETS.items():
        n = int(np.prod(s))
        a, b = g[o:o + n], ref[o:o + n]
        worst = max(worst, float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)))
    return worst


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_forward_and_gradients_vs_oracle(precision, tol):
    # 300 rows: several 64-row tiles and a ragged tail
    x, y = _data(300, 1)
    norm = _norm(x, y)
    p = I.mlp_init_params(3)
    net = _net(precision, p, norm)
    want_y, want_L, want_g = _oracle(p, x, y, norm)
    got_y = net.forward(x).cpu().numpy().astype(np.float64)
    assert np.abs(got_y - want_y).max() / np.abs(want_y).max() < tol
    L, g = net.loss_grad(x, y)
    assert abs(L - want_L) / want_L < tol
    assert _per_tensor_err(g.cpu().numpy().astype(np.float64), want_g) < tol
    net.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_inference_kernel_matches_training_forward(precision):
    x, y = _data(37, 2)  # three blocks of 16 rows, ragged
    norm = _norm(x, y)
    net = _net(precision, I.mlp_init_params(4), norm)
    a = net.forward(x).cpu().numpy()
    b = net.infer(x).cpu().numpy()
    if precision == "bf16":
        # same BF16 operands and k order of the mma products
        assert np.array_equal(a, b)
    else:
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    net.close()


def test_adamw_step_vs_oracle():
    import torch
    x, y = _data(256, 5)
    norm = _norm(x, y)
    p = I.mlp_init_params(6).astype(np.float32).astype(np.float64)
    net = _net("fp32", p, norm)
    lr, wd = 1e-3, 0.01
    xt = torch.tensor(x, dtype=torch.float32, device="cuda:0")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda:0")
    torch.cuda.synchronize()
    net.train_step(xt, yt, lr=lr, weight_decay=wd)
    got = net.params().astype(np.float64)
    _, _, g = _oracle(p, x, y, norm)
    want, _, _ = M.adamw(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr, wd=wd)
    # the first step moves each parameter by lr g / (|g| + eps): compare where
    # the gradient is not vanishing (its sign is then unambiguous)
    sig = np.abs(g) > 1e-4 * np.abs(g).max()
    assert sig.mean() > 0.5
    assert np.abs(got - want)[sig].max() < 1e-6
    net.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_training_loss_is_monotone_on_a_fixed_batch(precision):
    import torch
    x, y = _data(512, 7)
    norm = _norm(x, y)
    net = _net(precision, I.mlp_init_params(8), norm)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda:0")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda:0")
    torch.cuda.synchronize()
    losses = [net.train_step(xt, yt, lr=3e-4) for _ in range(60)]
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0]
    net.close()
