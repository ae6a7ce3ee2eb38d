"""Training workflow of the force/torque surrogate (host orchestration only:
the trajectories come from the solver's own steps with a device log, the
training pairs from the library's sample builder, the updates from its
forward/backward/AdamW kernels)."""
import numpy as np

from . import inputs as I
from . import turret as T


def record(turret, steps, chunk=1000):
    """Step a Turret with a device trajectory log attached; returns the
    records in time order (the initial time level included when the log was
    attached before the surface was loaded)."""
    turret.set_log(steps + 1)
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        turret.step(k)
        done += k
    return turret.log_records()


def record_ensemble(cfgs, steps, chunk=500, device="cuda:0"):
    """Trajectories of many runs at once: the runs of `cfgs` (ensemble
    configurations) advanced together by one batch, each with its own device
    log; returns the records of every run in time order."""
    from . import configs
    runs = configs.load_ensemble(cfgs, device=device)
    for t in runs:
        t.set_log(steps + 1)
    b = T.Batch(runs, device=device)
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        b.step(k)
        done += k
    recs = [t.log_records() for t in runs]
    b.close()
    for t in runs:
        t.close()
    return recs


def dataset(record_sets):
    """Concatenated training pairs of several trajectories."""
    import torch
    xs, ys = zip(*[T.build_samples(r) for r in record_sets])
    return torch.cat(xs), torch.cat(ys)


def standardisation(x, y):
    """Per-column mean and standard deviation of the training pairs (host)."""
    xa = x.double().cpu().numpy()
    ya = y.double().cpu().numpy()
    sx = xa.std(0)
    sy = ya.std(0)
    sx[sx == 0] = 1.0
    sy[sy == 0] = 1.0
    return xa.mean(0), sx, ya.mean(0), sy


def validation_loss(net, x, y):
    """Mean squared error of standardised outputs on (x, y), in chunks."""
    tot, n = 0.0, x.shape[0]
    for s in range(0, n, net.cap):
        e = min(n, s + net.cap)
        L, _ = net.loss_grad(x[s:e], y[s:e])
        tot += L * (e - s)
    return tot / n


def train(x, y, epochs=30, batch=4096, lr=1e-3, weight_decay=1e-4, seed=0, precision="bf16", net=None,
          device="cuda:0", val=None):
    """Train (or continue training) a network on pairs (x, y); returns (net,
    per-epoch mean losses).  Minibatches are drawn by a seeded permutation.
    With val = (x_val, y_val), the parameters of the epoch with the lowest
    validation loss are kept (early stopping); history then holds
    (train loss, validation loss) pairs."""
    import torch
    n = x.shape[0]
    if net is None:
        net = T.MLP(I.mlp_init_params(seed), batch_cap=min(batch, n), precision=precision, device=device)
        net.set_norm(*standardisation(x, y))
    rng = np.random.default_rng(seed)
    bsz = min(batch, net.cap)
    history = []
    best = (validation_loss(net, *val), net.params()) if val is not None else None
    for _ in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=x.device)
        tot, cnt = 0.0, 0
        for s in range(0, n - bsz + 1, bsz):
            idx = perm[s:s + bsz]
            xb = x.index_select(0, idx).contiguous()
            yb = y.index_select(0, idx).contiguous()
            tot += net.train_step(xb, yb, lr=lr, weight_decay=weight_decay)
            cnt += 1
        if val is None:
            history.append(tot / max(cnt, 1))
        else:
            vl = validation_loss(net, *val)
            history.append((tot / max(cnt, 1), vl))
            if vl < best[0]:
                best = (vl, net.params())
    if val is not None:
        net.set_params(best[1])
    return net, history


def offline_errors(net, x, y):
    """Relative error |F^ - F(t+1)| / |F(t+1)| of one-step force predictions on
    pairs (x, y) (inputs and targets as built by build_samples) for: the
    network, linear extrapolation (target 0), and persistence F^ = F(t)."""
    xa = x.double().cpu().numpy()
    ya = y.double().cpu().numpy()
    lin = 2 * xa[:, 10:13] - xa[:, 16:19]   # linear extrapolation, body frame / sF
    fn = lin + ya[:, :3]                     # the next force, body frame / sF
    den = np.linalg.norm(fn, axis=1)
    out = {"linear": np.linalg.norm(ya[:, :3], axis=1) / den,
           "persistence": np.linalg.norm(xa[:, 10:13] - fn, axis=1) / den}
    if net is not None:
        pa = net.infer(x).double().cpu().numpy()
        out["network"] = np.linalg.norm(pa[:, :3] - ya[:, :3], axis=1) / den
    return out
