"""GPU parity of the fused collide+stream kernel (through the C ABI) with the
FP64 oracle: periodic box, walls, constant-pressure top with sponge, ragged
tiles, reduced-precision storage, and the full 96x96x192 window."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_15115_gb300 import inputs as I

from cases import TOL_U_F32, gpu_velocity, make_pair, rel_max

pytestmark = pytest.mark.gpu

# 40 x 10 x 12 spans two 32-wide x tiles and three 4-high y tiles, all ragged
SHAPE = (12, 10, 40)


def _fields(shape, seed=1):
    return I.random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=3, seed=seed)


def test_initial_state_matches():
    nz, ny, nx = SHAPE
    t, s = make_pair(nx, ny, nz, 0.05, (0, 0, 0, 0), fields=_fields(SHAPE))
    u, rho = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < 1e-6
    fo = s.f()
    fg = t.populations().cpu().numpy()
    xi, w = O.lattice()
    dev_o = np.moveaxis(fo - w, -1, 0)
    assert np.abs(fg - dev_o).max() < 1e-8


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 0, 1, 2), (1, 0, 1, 2)])
def test_collide_stream_100_steps(bc):
    nz, ny, nx = SHAPE
    sponge = 4 if bc[3] == 2 else 0
    t, s = make_pair(nx, ny, nz, 0.03, bc, sponge=sponge, fields=_fields(SHAPE, 3))
    t.step(1)
    s.fluid_step(1)
    xi, w = O.lattice()
    fg = t.populations().cpu().numpy()
    assert np.abs(fg - np.moveaxis(s.f() - w, -1, 0)).max() < 2e-9
    t.step(99)
    s.fluid_step(99)
    u, rho = gpu_velocity(t)
    err = rel_max(u, s.velocity())
    assert err < TOL_U_F32, err


def test_graph_and_direct_launch_agree_bitwise():
    nz, ny, nx = SHAPE
    f = _fields(SHAPE, 5)
    a, _ = make_pair(nx, ny, nz, 0.05, (0, 0, 1, 2), sponge=3, fields=f)
    b, _ = make_pair(nx, ny, nz, 0.05, (0, 0, 1, 2), sponge=3, fields=f, flags={"no_graph": 1, "ibm_cycles": 4})
    a.step(7)
    b.step(7)
    assert np.array_equal(a.populations().cpu().numpy(), b.populations().cpu().numpy())


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_reduced_precision_storage(storage, tol):
    # deviations stored as q/w (x16 for FP16): per-step rounding ~2^-11 (FP16)
    # or 2^-8 (BF16) of q/w; velocity error after 100 steps stays at that level
    nz, ny, nx = SHAPE
    t, s = make_pair(nx, ny, nz, 0.03, (0, 0, 1, 2), sponge=4, storage=storage, fields=_fields(SHAPE, 4))
    t.step(100)
    s.fluid_step(100)
    u, _ = gpu_velocity(t)
    err = rel_max(u, s.velocity())
    assert err < tol, err


def test_periodic_mass_and_momentum_conservation():
    shape = (32, 32, 64)
    t, _ = make_pair(64, 32, 32, 0.02, (0, 0, 0, 0), fields=_fields(shape, 6))
    m0 = t.macro().double()
    M0 = m0[0].sum().item()
    J0 = (m0[0] * m0[1:]).sum(dim=(1, 2, 3))
    t.step(500)
    m1 = t.macro().double()
    assert abs(m1[0].sum().item() - M0) / M0 < 1e-6
    J1 = (m1[0] * m1[1:]).sum(dim=(1, 2, 3))
    assert (J1 - J0).abs().max().item() < 1e-6 * m0[0].numel() * 0.01


def test_full_size_window_one_step():
    # the 96 x 96 x 192 turret window, no-slip bottom, pressure top, 15-cell sponge
    shape = (192, 96, 96)
    O.set_threads(0)
    t, s = make_pair(96, 96, 192, 0.02, (0, 0, 1, 2), sponge=15, fields=_fields(shape, 7))
    t.step(2)
    s.fluid_step(2)
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < 1e-6


@pytest.mark.parametrize("storage,tol", [("f32", TOL_U_F32), ("f16", 2e-3)])
def test_moving_walls_100_steps(storage, tol):
    # shear between a bottom and a top wall moving in their planes (bc 3), on a
    # seeded random flow: the moving-wall bounce-back against the oracle
    nz, ny, nx = SHAPE
    walls = ((-0.02, 0.01, 0.0), (0.03, -0.005, 0.0))
    t, s = make_pair(nx, ny, nz, 0.03, (0, 0, 3, 3), fields=_fields(SHAPE, 5), walls=walls, storage=storage)
    t.step(100)
    s.fluid_step(100)
    u, _ = gpu_velocity(t)
    err = rel_max(u, s.velocity())
    assert err < tol, err


def test_moving_walls_reject_bad_velocities():
    from paper_2408_15115_gb300 import turret as T
    t = T.Turret(8, 8, 8, 0.1, 1.0, (0, 0, 0), 0, 0, 3, 3)
    with pytest.raises(T.TurretError):
        t.set_wall_velocity((0, 0, 0.01), (0, 0, 0))  # normal component
    with pytest.raises(T.TurretError):
        t.set_wall_velocity((0.5, 0, 0), (0, 0, 0))  # too fast
    with pytest.raises(T.TurretError):
        T.Turret(8, 8, 8, 0.1, 1.0, (0, 0, 0), 0, 0, 3, 2, slide=1, anchor_frac=0.3)  # no sliding window
    t.close()



def test_zero_and_negative_step_counts():
    # step(0) enqueues nothing; step(-1) is rejected (EINVAL) before any work
    # and the context stays usable: the next step still matches the oracle
    from paper_2408_15115_gb300 import turret as T
    nz, ny, nx = SHAPE
    t, s = make_pair(nx, ny, nz, 0.05, (0, 0, 0, 0), fields=_fields(SHAPE, 5))
    before = t.populations().cpu().numpy().copy()
    t.step(0)
    assert np.array_equal(t.populations().cpu().numpy(), before)
    with pytest.raises(T.TurretError) as e:
        t.step(-1)
    assert e.value.status == 1
    assert np.array_equal(t.populations().cpu().numpy(), before)
    t.step(1)
    s.fluid_step(1)
    xi, w = O.lattice()
    assert np.abs(t.populations().cpu().numpy() - np.moveaxis(s.f() - w, -1, 0)).max() < 2e-9
