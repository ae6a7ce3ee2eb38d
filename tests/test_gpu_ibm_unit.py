"""GPU parity of the standalone spreading operator (Sec. 2.2, step l = 1)
with the oracle's dense loops, on a ragged grid, plus its domain check."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(seed=0, shape=(28, 20, 24), n=4):
    nz, ny, nx = shape
    V, T = I.icosphere(n, 5.5)
    rng = np.random.default_rng(seed)
    X = V + np.array([nx / 2 - 0.37, ny / 2 + 0.21, nz / 2 + 0.05]) + 0.1 * rng.standard_normal(3)
    h = 1e-3 * rng.standard_normal((X.shape[0], 3))
    dS = O.mesh_props(V, T)["dS"]
    return X, h, dS, shape


def _gpu_spread(X, h, dS, shape):
    import torch
    from paper_2408_15115_gb300 import turret as T
    dev = torch.device("cuda:0")
    Xt = torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device=dev)
    ht = torch.tensor(np.ascontiguousarray(h.T), dtype=torch.float32, device=dev)
    dt = torch.tensor(dS, dtype=torch.float32, device=dev)
    return T.ibm_spread(Xt, ht, dt, shape).cpu().numpy()


def test_spread_matches_oracle():
    X, h, dS, shape = _case()
    got = np.moveaxis(_gpu_spread(X, h, dS, shape), 0, -1).astype(np.float64)
    want = O.spread(h, X, dS, shape, (False, False, False))
    # FP32 weights and sums of at most ~30 terms per cell
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    # total force is conserved by the spreading (partition of unity)
    assert np.abs(got.reshape(-1, 3).sum(0) - (h * dS[:, None]).sum(0)).max() < 1e-5 * np.abs(h * dS[:, None]).sum()


def test_spread_is_reproducible():
    X, h, dS, shape = _case(seed=3)
    a = _gpu_spread(X, h, dS, shape)
    b = _gpu_spread(X, h, dS, shape)
    assert np.array_equal(a, b)


def test_spread_rejects_marker_outside_grid():
    from paper_2408_15115_gb300 import turret as T
    X, h, dS, shape = _case()
    X = X.copy()
    X[0] = (0.5, 5.0, 5.0)  # stencil starts at -1
    with pytest.raises(T.TurretError) as e:
        _gpu_spread(X, h, dS, shape)
    assert e.value.status == 7
