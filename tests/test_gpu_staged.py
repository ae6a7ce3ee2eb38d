"""The 16-bit collide+stream with its sources and results staged in shared
memory by bulk tensor copies (flags.staged_loads) against the same kernel with
plain global loads and stores: bitwise equal
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
