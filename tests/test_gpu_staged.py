"""The 16-bit collide+stream paths: the default one on x-adjacent cell pairs
with 4-byte accesses against the FP64 oracle, and the opt-in one with its
sources and results staged in shared memory by bulk tensor copies
(flags.staged_loads) against the default: bitwise equal
populations and particle state, on fluid-only periodic windows (every tile at
a periodic edge patched from the far side) and on coupled sliding windows
(far-cell tiles staged, tiles at the near region, the ring's wrap and the
boundary planes on the plain path), and against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

from cases import gpu_velocity, make_pair, rel_max

pytestmark = pytest.mark.gpu


def _pair_runs(build, steps):
    out = []
    for plain in (0, 1):
        t = build(plain)
        t.step(steps)
        out.append((t.populations().cpu().numpy(), t.state()))
        t.close()
    return out


@pytest.mark.parametrize("storage,sr", [("f16", 0), ("bf16", 0), ("bf16", 1)])
@pytest.mark.parametrize("shape", [(32, 32, 64), (64, 96, 32)])
def test_staged_fluid_window_is_bitwise_plain(storage, sr, shape):
    # fully periodic windows (nx = 32: both x edges in one tile), a seeded
    # smooth flow, 25 steps with the staged and with the plain loads
    from paper_2408_15115_gb300 import turret as T
    nz, ny, nx = shape
    rho, u = I.random_state(shape, u_amp=0.02, rho_amp=0.002, kmax=3, seed=21)

    def build(plain):
        t = T.Turret(nx, ny, nz, 0.02, storage=storage,
                     flags={"staged_loads": 1 - plain, "stochastic_rounding": sr, "ibm_cycles": 4})
        t.set_fields(rho, u)
        return t

    (pa, _), (pb, _) = _pair_runs(build, 25)
    assert np.array_equal(pa, pb)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_staged_coupled_sliding_window_is_bitwise_plain(storage):
    # a sphere in a 64 x 64 x 96 sliding window (pressure top with a sponge,
    # no-slip bottom) released seven cells below the window's anchor: the
    # window slides up to it over the first steps, so the ring's physical
    # wrap and the entering plane sit at interior planes; the near region
    # moves with the particle
    from paper_2408_15115_gb300 import turret as T
    V, Tr = I.sphere(6, 10.0)

    def build(plain):
        t = T.Turret(64, 64, 96, 0.02, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=8, slide=1, anchor_frac=0.45,
                     storage=storage, flags={"staged_loads": 1 - plain, "ibm_cycles": 4})
        t.load_surface(V, Tr, (31.3, 32.6, 36.2), v0=(0.0, 0.0, -0.05), w0=(0.0, 0.002, 0.0))
        return t

    (pa, sa), (pb, sb) = _pair_runs(build, 60)
    assert abs(sa["origin"][2]) >= 3  # the window slid
    assert np.array_equal(pa, pb)
    for k in ("r", "v", "w", "F", "T", "d"):
        assert np.array_equal(sa[k], sb[k]), k


def test_staged_fp16_window_vs_oracle():
    # the staged path against the FP64 oracle: a periodic 64 x 32 x 32 window
    # with a pressure top and sponge, 100 steps of a seeded flow, FP16 storage
    # (velocity bar of the 16-bit parity suite)
    shape = (32, 32, 64)
    O.set_threads(0)
    fields = I.random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=3, seed=9)
    t, s = make_pair(64, 32, 32, 0.03, (0, 0, 1, 2), sponge=4, storage="f16", fields=fields,
                     flags={"staged_loads": 1})
    t.step(100)
    s.fluid_step(100)
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < 2e-3
    t.close()


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_xpair_window_vs_oracle(storage, tol):
    # the default 16-bit path on a window its 64 x 2 x 2 tiles cover (x-adjacent
    # cell pairs, 4-byte accesses; boundary planes on the cell-pair path):
    # 64 x 32 x 32 with a no-slip bottom, a pressure top and a sponge, 100
    # steps of a seeded flow against the FP64 oracle
    shape = (32, 32, 64)
    O.set_threads(0)
    fields = I.random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=3, seed=17)
    t, s = make_pair(64, 32, 32, 0.03, (0, 0, 1, 2), sponge=4, storage=storage, fields=fields)
    t.step(100)
    s.fluid_step(100)
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < tol
    t.close()


@pytest.mark.parametrize("storage,tol_f,tol_v", [("f16", 2e-2, 2e-3), ("bf16", 5e-2, 2e-2)])
def test_xpair_coupled_sliding_window_vs_oracle(storage, tol_f, tol_v):
    # a coupled 64 x 64 x 96 sliding window in 16-bit storage: the far cells on
    # x-pairs, the near region and the boundary planes on the cell-pair path;
    # 40 steps against the FP64 oracle (force, body velocity, fluid velocity)
    V, Tr = I.sphere(6, 10.0)
    O.set_threads(0)
    r0 = (31.3, 32.6, 36.2)
    t, s = make_pair(64, 64, 96, 0.02, (0, 0, 1, 2), kappa=2.0, g=(0, 0, -1e-4), sponge=8, slide=1, anchor=0.45,
                     storage=storage, particle=(V, Tr, r0, (0.0, 0.0, -0.05), (0.0, 0.002, 0.0)))
    t.step(40)
    s.step(40)
    a, b = t.state(), s.state()
    assert abs(b["origin"][2]) >= 3
    assert np.array_equal(a["origin"], b["origin"].astype(np.int64))
    assert np.abs(a["F"] - b["F"]).max() / np.abs(b["F"]).max() < tol_f, (a["F"], b["F"])
    assert np.abs(a["v"] - b["v"]).max() / np.abs(b["v"]).max() < tol_v, (a["v"], b["v"])
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < tol_v
    t.close()
